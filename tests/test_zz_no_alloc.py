"""kd_st_loss_fwd_noalloc: the structure-tensor loss forward for callers that cannot allocate
device memory (a plugin inside a host application that owns all GPU memory, or a loop where
cudaMalloc's implicit synchronisation is not allowed). It keeps its partial sums in a fixed
device array inside the library instead of a caller-supplied workspace.

This file is named to be collected last, so that a run stopping at the first failure has run
every other test before it. It also passes on its own in a fresh process: the first call on the
device looks up the array's address.
"""
import math

import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import kdiag as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
WV = (1 / math.sqrt(3),) * 3


def _noalloc(A, dtype_code):
    out = torch.full((2,), float("nan"), device=DEV, dtype=torch.float64)
    n = A.shape[1]
    s = K.kd_st_loss_fwd_noalloc(A.data_ptr(), dtype_code, n, n, WV, out.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_OK, K.status_string(s)
    return out


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    """Two calls in a row (a larger field, then a smaller one, so the second call runs over
    partials left by the first) give the sums of kd_st_loss_fwd. The two entry points split the
    field into blocks differently, so the FP32 per-thread partial sums differ by rounding only:
    1e-6 relative."""
    fields = [(W.structure_tensor_field((64, 64, 32), seed=11, device=DEV), K.KD_BF16),
              (W.structure_tensor_field((32, 32, 16), seed=12, device=DEV).float(), K.KD_F32)]
    for A, code in fields:
        got = _noalloc(A, code)
        ref = K.st_loss_fwd(A, WV)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert torch.allclose(got, ref, rtol=1e-6, atol=0.0), (got.tolist(), ref.tolist())


def test_noalloc_rejects_n_beyond_its_capacity():
    A = torch.zeros(6, 16, device=DEV)
    out = torch.zeros(2, device=DEV, dtype=torch.float64)
    n = 8192 * 16384 + 1
    s = K.kd_st_loss_fwd_noalloc(A.data_ptr(), K.KD_F32, n, n, WV, out.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_ERR_TOO_LARGE
    assert "capacity" in K.status_string(s)
