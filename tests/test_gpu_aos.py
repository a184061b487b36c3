"""Array-of-structures batches (kd_opts.layout = KD_LAYOUT_AOS): the TMA-staged FP32 forward, the
tail and misaligned fallbacks, the FP64/BF16 paths and the adjoint against the oracles (and the
structure-of-arrays results); the bounded waits report through the library's fault word."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1306_6291_gb300 import kdiag as K
from parity import D_rows, definition_errors, planes_to_rows, summary

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rows(P):
    return P.t().contiguous()


def _check_close(aos, soa_planes, atol):
    assert torch.allclose(aos, soa_planes.t(), atol=atol, rtol=0), float((aos - soa_planes.t()).abs().max())


@pytest.mark.parametrize("n,inv", [(256, 0), ((1 << 16) + 37, 0), (1 << 20, 0), ((1 << 16) + 37, 2)])
def test_aos_fp32_forward_matches_soa(n, inv):
    A, _ = W.sym3_precision(n, seed=n, device=DEV)
    o = K.make_opts(invariants=inv)
    l1, D1, a1, k1 = K.eig3(A, o, kase=True)
    R = _rows(A)
    assert R.data_ptr() % 16 == 0
    l2, D2, a2, k2 = K.eig3_aos(R, o, kase=True)
    assert torch.equal(k1, k2)
    scale = planes_to_rows(A).__abs__().max(1)
    lerr = (l2.double().cpu().numpy() - planes_to_rows(l1)) / scale[:, None]
    assert np.max(np.abs(lerr)) < 4e-6
    errs = summary(definition_errors(planes_to_rows(A), l2.double().cpu().numpy(),
                                     D2.double().cpu().numpy().reshape(-1, 3, 3)))
    assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6
    st, code = K.kd_device_fault()
    assert st == K.KD_OK and code == 0


def _definition_check(Arows_f64, lam, D, what):
    """FP32 tolerances against the Jacobi definition oracle (lam (n, 3), D (n, 9) rows)."""
    e = summary(definition_errors(Arows_f64, lam.double().cpu().numpy(),
                                  D.double().cpu().numpy().reshape(-1, 3, 3)))
    print(f"AoS {what}: {e}")
    assert e["lam"] < 2e-6 and e["ev"] < 1e-5 and e["rec"] < 4e-6 and e["orth"] < 2e-6, e


def test_aos_misaligned_and_other_dtypes_use_the_plain_path():
    """The per-thread AoS fallbacks against the oracle: a 4-byte aligned FP32 batch (no TMA) and
    BF16 records against the Jacobi definition oracle at the FP32 tolerances; FP64 records against
    the method oracle at 1e-13 ||A||_F; all three also agree with their SoA counterparts."""
    n = 5000
    A = W.sym3_normal(n, seed=1, device=DEV)
    R = _rows(A)
    buf = torch.empty(6 * n + 1, device=DEV)
    buf[1:] = R.reshape(-1)
    Rm = buf[1:].view(n, 6)                       # 4-byte aligned only: no TMA
    assert Rm.data_ptr() % 16 != 0
    l2, D2, a2, _ = K.eig3_aos(Rm)
    _definition_check(planes_to_rows(A), l2, D2, "fp32 misaligned")
    l1, D1, a1, _ = K.eig3_aos(R)
    assert torch.allclose(l1, l2, atol=1e-5) and torch.allclose(a1, a2, atol=1e-4)
    # FP64 records: the plain FP64 form against the method oracle
    l64, D64, a64, k64 = K.eig3_aos(R.double(), kase=True)
    lo, Do, ao, ko = oracle.eig3(planes_to_rows(A))
    fro = np.linalg.norm(oracle.unpack3(planes_to_rows(A)), axis=(1, 2))
    same = (k64.cpu().numpy() == ko)
    lerr = np.abs(l64.cpu().numpy() - lo).max(1) / fro
    print(f"AoS fp64: max lam err {lerr.max():.3e}, kase agreement {same.mean():.5f}")
    assert same.mean() > 0.999 and np.max(lerr[same]) < 1e-13
    # BF16 records: the widened values against the definition oracle
    Rb = R.to(torch.bfloat16)
    lb, Db_, _, _ = K.eig3_aos(Rb)
    _definition_check(Rb.double().cpu().numpy(), lb, Db_, "bf16")
    lbs, _, _, _ = K.eig3(A.to(torch.bfloat16))
    assert torch.allclose(lb, lbs.t(), atol=1e-5)


def test_aos_adjoint_matches_oracle():
    """The AoS adjoint (per-thread records) against the oracle's analytic adjoint, scaled as in
    the SoA adjoint tests (the oracle's cotangents take the GPU D's column signs); it also agrees
    with the SoA adjoint."""
    n = 20000
    A = W.sym3_normal_gapped(n, seed=2, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(3)
    lb, Db, ab = (torch.randn(k, n, generator=g, device=DEV) for k in (3, 9, 3))
    got = K.eig3_adjoint_aos(_rows(A), _rows(lb), _rows(Db), _rows(ab))
    Ar = planes_to_rows(A)
    lo, Do, _, ko = oracle.eig3(Ar)
    _, D, _, kase = K.eig3(A, ang=False, kase=True)
    sign = np.sign(np.einsum("nik,nik->nk", D_rows(D), Do))
    lbr = planes_to_rows(lb)
    Dbr = planes_to_rows(Db).reshape(-1, 3, 3) * sign[:, None, :]
    same = (kase.cpu().numpy() == 0) & (ko == 0)
    # the angle cotangents are left out of the oracle comparison (they enter through the Euler
    # angles, whose representation the FP32 and FP64 paths pick alike only away from the range
    # ends); the AoS call with them is compared with the SoA call below
    got0 = K.eig3_adjoint_aos(_rows(A), _rows(lb), _rows(Db))
    ref = oracle.eig3_adjoint(Ar[same], lbr[same], Dbr[same], gap_mask=1e-6)
    fro = np.linalg.norm(oracle.unpack3(Ar[same]), axis=(1, 2))
    gmin = np.min(np.abs(lo[same][:, [0, 0, 1]] - lo[same][:, [1, 2, 2]]), 1) / fro
    err = np.abs(got0.double().cpu().numpy()[same] - ref).max(1)
    scale = (1 + np.abs(Dbr[same]).max((1, 2)) + np.abs(lbr[same]).max(1)) / gmin ** 2
    print(f"AoS adjoint: max err/scale {np.max(err / scale):.3e}")
    # the bound of the SoA adjoint tests (tests/test_gpu_adjoint.py)
    assert same.mean() > 0.99 and np.max(err / scale) < 2e-6
    ref_soa = K.eig3_adjoint(A, lb, Db, ang_bar=ab)
    rel = ((got - ref_soa.t()).abs().amax(1) / ref_soa.t().abs().amax(1)).cpu().numpy()
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
