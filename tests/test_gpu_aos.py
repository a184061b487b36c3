"""Array-of-structures batches (kd_opts.layout = KD_LAYOUT_AOS): the TMA-staged FP32 forward, the
tail and misaligned fallbacks, the FP64/BF16 paths and the adjoint give the structure-of-arrays
results; the bounded waits report through the library's fault word."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import kdiag as K
from parity import D_rows, definition_errors, planes_to_rows, summary

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rows(P):
    return P.t().contiguous()


def _check_close(aos, soa_planes, atol):
    assert torch.allclose(aos, soa_planes.t(), atol=atol, rtol=0), float((aos - soa_planes.t()).abs().max())


@pytest.mark.parametrize("n", [256, (1 << 16) + 37, 1 << 20])
def test_aos_fp32_forward_matches_soa(n):
    A, _ = W.sym3_precision(n, seed=n, device=DEV)
    l1, D1, a1, k1 = K.eig3(A, kase=True)
    R = _rows(A)
    assert R.data_ptr() % 16 == 0
    l2, D2, a2, k2 = K.eig3_aos(R, kase=True)
    assert torch.equal(k1, k2)
    scale = planes_to_rows(A).__abs__().max(1)
    lerr = (l2.double().cpu().numpy() - planes_to_rows(l1)) / scale[:, None]
    assert np.max(np.abs(lerr)) < 4e-6
    errs = summary(definition_errors(planes_to_rows(A), l2.double().cpu().numpy(),
                                     D2.double().cpu().numpy().reshape(-1, 3, 3)))
    assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6
    st, code = K.kd_device_fault()
    assert st == K.KD_OK and code == 0


def test_aos_misaligned_and_other_dtypes_use_the_plain_path():
    n = 5000
    A = W.sym3_normal(n, seed=1, device=DEV)
    R = _rows(A)
    buf = torch.empty(6 * n + 1, device=DEV)
    buf[1:] = R.reshape(-1)
    Rm = buf[1:].view(n, 6)                       # 4-byte aligned only: no TMA
    l1, D1, a1, _ = K.eig3_aos(R)
    l2, D2, a2, _ = K.eig3_aos(Rm)
    assert torch.allclose(l1, l2, atol=1e-5) and torch.allclose(a1, a2, atol=1e-4)
    l64, D64, _, _ = K.eig3_aos(R.double())
    l64s, _, _, _ = K.eig3(A.double())
    assert torch.allclose(l64, l64s.t(), rtol=0, atol=1e-13 * float(A.abs().max()) * 10)
    lb, _, _, _ = K.eig3_aos(R.to(torch.bfloat16))
    lbs, _, _, _ = K.eig3(A.to(torch.bfloat16))
    assert torch.allclose(lb, lbs.t(), atol=1e-5)


def test_aos_adjoint_matches_soa():
    n = 20000
    A = W.sym3_normal_gapped(n, seed=2, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(3)
    lb, Db, ab = (torch.randn(k, n, generator=g, device=DEV) for k in (3, 9, 3))
    ref = K.eig3_adjoint(A, lb, Db, ang_bar=ab)
    got = K.eig3_adjoint_aos(_rows(A), _rows(lb), _rows(Db), _rows(ab))
    rel = ((got - ref.t()).abs().amax(1) / ref.t().abs().amax(1)).cpu().numpy()
    assert np.quantile(rel, 0.999) < 1e-4


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = K.kd_selftest_wait_timeout(flag.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == K.KD_OK
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
    A = W.sym3_normal(4096, seed=4, device=DEV)
    lam, _, _, _ = K.eig3_aos(_rows(A))
    torch.cuda.synchronize()
    assert torch.isfinite(lam).all()
    st, code = K.kd_device_fault()
    assert st == K.KD_OK and code == 0
