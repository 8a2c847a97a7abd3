"""The boundary used from a plain C program (gcc, libsft.so, the CUDA runtime; no Python in the
path): build tests/c_api_smoke.c against include/sft.h and run it on the GPU."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_program_recovers_a_sparse_spectrum(tmp_path):
    from paper_1706_02740_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "c_api_smoke")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-O2", "-std=c11", os.path.join(HERE, "c_api_smoke.c"), "-o", exe,
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           "-L", libdir, "-lsft", f"-Wl,-rpath,{libdir}",
           "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}",
           "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "C-ABI OK" in out.stdout
