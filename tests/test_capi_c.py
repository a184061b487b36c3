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
