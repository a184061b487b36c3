"""kd_st_loss_fwd_noalloc: the structure-tensor loss forward for callers that cannot allocate
device memory (a plugin inside a host application that owns all GPU memory, or a loop where
cudaMalloc's implicit synchronisation is not allowed). It keeps its partial sums in a fixed
device array inside the library instead of a caller-supplied workspace.

This file is named to be collected last, so that a run stopping at the first failure has run
every other test before it. It also passes on its own in a fresh process: every call looks up the
array's address in the current context.
"""
import math
import os
import shutil
import subprocess

import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import _build, kdiag as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
WV = (1 / math.sqrt(3),) * 3
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _noalloc(A, dtype_code):
    out = torch.full((2,), float("nan"), device=DEV, dtype=torch.float64)
    n = A.shape[1]
    s = K.kd_st_loss_fwd_noalloc(A.data_ptr(), dtype_code, n, n, WV, out.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_OK, K.status_string(s)
    return out


def _check(A, code):
    got = _noalloc(A, code)
    ref = K.st_loss_fwd(A, WV)
    torch.cuda.synchronize()
    assert torch.isfinite(got).all()
    # both entry points run the same kernel; the tolerance allows for a different block split
    assert torch.allclose(got, ref, rtol=1e-6, atol=0.0), (got.tolist(), ref.tolist())


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    """Two calls in a row (a larger field, then a smaller one, so the second call runs over
    partials left by the first) give the sums of kd_st_loss_fwd within 1e-6 relative."""
    fields = [(W.structure_tensor_field((64, 64, 32), seed=11, device=DEV), K.KD_BF16),
              (W.structure_tensor_field((32, 32, 16), seed=12, device=DEV).float(), K.KD_F32)]
    for A, code in fields:
        _check(A, code)


def test_noalloc_ragged_sizes_and_growing_block_counts():
    """Sizes with a partial last block and block counts that are not powers of two, in an order
    where a call uses more blocks than the one before it and then fewer again."""
    big = W.structure_tensor_field((64, 64, 64), seed=13, device=DEV)   # 262,144 tensors
    for n, dt, code in ((3 * 16384 + 17, torch.bfloat16, K.KD_BF16), (5 * 16384 + 1, torch.float32, K.KD_F32),
                        (big.shape[1], torch.bfloat16, K.KD_BF16), (1000 + 37, torch.float32, K.KD_F32)):
        A = big[:, :n].to(dt).contiguous()
        _check(A, code)


def test_noalloc_rejects_n_beyond_its_capacity():
    A = torch.zeros(6, 16, device=DEV)
    out = torch.zeros(2, device=DEV, dtype=torch.float64)
    n = 8192 * 16384 + 1
    s = K.kd_st_loss_fwd_noalloc(A.data_ptr(), K.KD_F32, n, n, WV, out.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_ERR_TOO_LARGE
    assert "capacity" in K.status_string(s)


def test_noalloc_after_a_device_reset(tmp_path):
    """tests/c/noalloc_reset.c (a separate process, CUDA runtime C API only) calls the entry point,
    resets the device, and calls it twice more in the new context; every call must give the sums
    of kd_st_loss_fwd. A stale scratch address would fail this."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    K.load()
    libdir = os.path.dirname(_build.LIB)
    cudalib = _build._cuda_libdir(_build.nvcc())
    cudainc = os.path.join(os.path.dirname(cudalib), "include")
    exe = tmp_path / "noalloc_reset"
    cmd = [cc, "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cudainc,
           os.path.join(ROOT, "tests", "c", "noalloc_reset.c"), "-L", libdir, "-lkdiag", "-L", cudalib,
           "-lcudart", "-lm", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr + r.stdout
    assert "noalloc_reset: ok" in r.stdout, r.stdout
