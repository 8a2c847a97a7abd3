"""CPU check of Rader's-form planning (csrc/rader_plan.h, compiled by the host compiler) over every
prime up to the FP32 length limit: the pass schedule exists exactly for 13-smooth p - 1, multiplies
to p - 1 with radices the Rader kernel implements, the primitive root is one and the smallest, the
two transform buffers fit a CTA, and the thread count is a whole number of warps.  A few schedules
are pinned by hand from the rule (each 7, 5, 3 takes a factor 2, 2, 4 while any is left; 11 and
13 alone; the other powers of two in radix-16 passes and one last 8, 4 or 2), and the primitive
roots by the textbook values."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("rader_plan") / "rader_plan")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "rader_plan_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return subprocess.run([exe], capture_output=True, text=True, timeout=120)


def test_every_prime_up_to_the_limit_plans_correctly(report):
    assert report.returncode == 0 and report.stdout.splitlines()[-1] == "ok", report.stdout[-2000:]
    summary = [ln.split() for ln in report.stdout.splitlines() if ln.startswith("primes")][0]
    assert int(summary[1]) == 1608                  # pi(13601)
    assert int(summary[3]) >= 200                   # primes with 13-smooth p - 1


def test_schedules_and_roots_by_hand(report):
    got = {}
    for ln in report.stdout.splitlines():
        if ln.startswith("sched"):
            head, rad = ln.split("|")
            f = head.split()
            got[int(f[1])] = (int(f[3]), [int(r) for r in rad.split()])
    assert got[13] == (2, [12])                     # 12 = 2^2 3: the two 2s join the 3
    assert got[3001] == (14, [10, 10, 10, 3])       # 3000 = 2^3 3 5^3: the 2s go to the 5s
    assert got[3137] == (3, [16, 14, 14])           # 3136 = 2^6 7^2
    assert got[8191] == (17, [14, 13, 5, 3, 3])     # 8190 = 2 3^2 5 7 13
    assert got[12289] == (11, [16, 16, 12, 4])      # 12288 = 2^12 3
