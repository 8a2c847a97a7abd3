"""CPU check of the plan's integer helpers (csrc/int_math.h, compiled by the host compiler) against
brute force: primality (the moduli pools and caller-given primes), gcd (coprimality of the
moduli), modular inverses (the Garner constants of the residue reconstruction, bit-exact by
construction only if every inverse is right) and 13-smoothness (Rader's schedules)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_helpers_match_brute_force(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "int_math")
    subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "int_math_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout[-2000:]
