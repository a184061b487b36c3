"""The C-ABI is usable from plain C: tests/c/capi_check.c compiles with a C compiler against
include/kdiag.h alone, links libkdiag.so and runs its host-side checks (no kernel is launched)."""
import os
import shutil
import subprocess

import pytest

from paper_1306_6291_gb300 import _build, kdiag as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    K.load()   # builds the library if needed
    libdir = os.path.dirname(_build.LIB)
    exe = tmp_path / "capi_check"
    cmd = [cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "capi_check.c"), "-L", libdir, "-lkdiag",
           f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr + r.stdout
    assert "capi_check: ok" in r.stdout


@pytest.mark.gpu
def test_plain_c_client_runs_the_kernels(tmp_path):
    """tests/c/capi_gpu.c runs the forward and the adjoint through the C-ABI with the CUDA
    runtime's C API alone and checks trace, orthogonality, reconstruction and the eigenvalue
    adjoint on 1000 matrices."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    K.load()
    libdir = os.path.dirname(_build.LIB)
    cudalib = _build._cuda_libdir(_build.nvcc())
    cudainc = os.path.join(os.path.dirname(cudalib), "include")
    exe = tmp_path / "capi_gpu"
    cmd = [cc, "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cudainc,
           os.path.join(ROOT, "tests", "c", "capi_gpu.c"), "-L", libdir, "-lkdiag", "-L", cudalib, "-lcudart",
           "-lm", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr + r.stdout
    assert "capi_gpu: ok" in r.stdout, r.stdout
