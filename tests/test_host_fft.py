"""CPU check of the plan's FP64 host FFTs (csrc/host_fft.h, compiled by the host compiler): the
chirp filter's spectrum is taken by host_fft at every chirp-convolution length r 2^k (r = 1, 3, 5,
7), Rader's V by host_fft_mixed at lengths p - 1, and both from the exactly reduced turns of
expi_turns and half_turn_twiddles.  Each is compared with the defining sum evaluated in long double
and must stay inside the rounding-error bound of its stage radices (Higham's analysis of the FFT);
a dropped term, a wrong sign or a wrong twiddle index gives an error of order 1."""
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
    exe = str(tmp_path_factory.mktemp("host_fft") / "host_fft")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "host_fft_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    rows = {}
    for ln in out.stdout.splitlines():
        f = ln.split()
        if len(f) == 4:
            rows[(f[0], int(f[1]))] = (float(f[2]), float(f[3]))
    return out, rows


def test_every_length_is_inside_its_error_bound(report):
    out, rows = report
    assert out.returncode == 0 and out.stdout.splitlines()[-1] == "ok", out.stdout[-3000:]
    for key, (err, bound) in rows.items():
        assert err <= bound, key


def test_every_chirp_length_and_the_rader_lengths_are_covered(report):
    _, rows = report
    chirp = {m for base in (64, 96, 640, 896) for m in (base << j for j in range(10)) if m <= 16384}
    assert chirp <= {M for kind, M in rows if kind == "chirp"}
    rader = {M for kind, M in rows if kind == "rader"}
    assert {4098, 4110, 13596} <= rader          # 4099 - 1 = 2 3 683: a large prime factor


def test_turns_are_accurate_to_a_few_ulp(report):
    _, rows = report
    err, bound = rows[("turns", 0)]
    assert err <= bound < 20                     # units of 2^-53
    for (kind, M), (err, bound) in rows.items():
        if kind == "twiddles" and M % 8 == 0:
            assert err <= bound < 3.4, M         # first octant only, the rest by exact symmetry
