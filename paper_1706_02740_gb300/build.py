"""Builds libsft.so (the CUDA kernels and the C ABI of include/sft.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked as one shared library against
the CUDA runtime.  Output: paper_1706_02740_gb300/_build/libsft.so, and the checked build (index
checks compiled in, SFT_CHECKED) paper_1706_02740_gb300/_build_checked/libsft_checked.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsft.so")
# The checked build (every gather, bin and candidate index range-checked, faults recorded in the
# plan's status words): the same sources compiled with SFT_CHECKED into a library of its own.
OUT_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libsft_checked.so")
SOURCES = ["api.cu", "batch.cu", "plan.cpp", "server.cpp", "resample.cu", "bluestein.cu", "rader.cu",
           "identify.cu",
           "select.cu", "refine.cu", "energy.cu", "tuning_table.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _compile(src: str, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(OUT_CHECKED if checked else OUT, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + FLAGS
    if checked:
        cmd += ["-DSFT_CHECKED=1"]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _stale(lib: str, srcs: list) -> bool:
    if not os.path.exists(lib):
        return True
    lib_t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > lib_t for s in srcs)


def _link(objs: list, lib: str) -> None:
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile libsft.so and, unless checked=False, libsft_checked.so (all translation units of
    both in one parallel pool); returns the path of libsft.so."""
    os.makedirs(OUT, exist_ok=True)
    os.makedirs(OUT_CHECKED, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(os.path.dirname(HERE), "include", "sft.h"))
    jobs = []
    if force or _stale(LIB, srcs):
        jobs += [(s, False) for s in SOURCES]
    if checked and (force or _stale(LIB_CHECKED, srcs)):
        jobs += [(s, True) for s in SOURCES]
    if not jobs:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    plain = [o for o, j in zip(objs, jobs) if not j[1]]
    chk = [o for o, j in zip(objs, jobs) if j[1]]
    if plain:
        _link(plain, LIB)
    if chk:
        _link(chk, LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
