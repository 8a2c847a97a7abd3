"""CPU check of the chirp-convolution FFT schedule (csrc/sft_internal.h, compiled by the host
compiler): for every admissible length r 2^k (r = 1, 3, 5, 7) the passes multiply up to M, no pass
holds more than 16 values per thread, the radix-2 pass splits evenly, the twiddle rows fit in M
entries, and the length chosen for each prime is the smallest admissible one >= 2p - 1."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_every_length_has_a_valid_schedule(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path / "fft_schedule")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "fft_schedule_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout[-2000:]
    lines = out.stdout.split("\n")
    assert "ok" in lines
    sched = {int(ln.split()[0]): [int(x) for x in ln.split("|")[0].split()[2:]]
             for ln in lines if "|" in ln}
    assert sched[8192] == [16, 16, 16]
    assert sched[7168] == [16, 16, 14]
    assert sched[6144] == [16, 16, 12]
    assert sched[12288] == [16, 16, 12, 2]
    assert sched[1280] == [16, 10, 4]
