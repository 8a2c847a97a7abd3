"""CPU check of the per-prime DFT tables every plan uploads (csrc/prime_tables.h, compiled by the
host compiler): the chirp form's chirp and filter spectrum and Rader's form's permutations and V
are combined on the host exactly as the kernels combine them, and the resulting length-p DFT
(eq. DFT_GKlam_Comp's measurements, E_c = (1/p) sum_k x_k e^{-2 pi i k c / p}) must match the
defining sum in long double to 1e-13 relative, for small, benchmark-sized and limit-sized primes;
the re-estimation twiddles must be the turns e^{-2 pi i n / p}."""
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
    exe = str(tmp_path_factory.mktemp("prime_tables") / "prime_tables")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "prime_tables_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return subprocess.run([exe], capture_output=True, text=True, timeout=300)


def test_both_forms_reproduce_the_dft(report):
    assert report.returncode == 0 and report.stdout.splitlines()[-1] == "ok", report.stdout[-2000:]
    rows = [ln.split() for ln in report.stdout.splitlines() if ln.startswith(("chirp", "rader"))]
    chirp = {int(r[1]): int(r[2]) for r in rows if r[0] == "chirp"}
    rader = {int(r[1]) for r in rows if r[0] == "rader"}
    assert chirp[3001] == 6144 and chirp[3079] == 7168 and chirp[8191] == 16384
    assert {3001, 3137, 12289, 13313} <= rader
    assert all(float(r[-1]) <= 1e-13 for r in rows)
