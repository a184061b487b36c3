"""GPU parity of the 2x2 forward and adjoint (kd_eig2_sym, kd_eig2_sym_adjoint) against the oracle.

Tolerances: FP32 eigenvalues 2e-6 ||A||_F (label-exact: the sign rule of Section 3 fixes the
labels); phi within 1e-6 ||A||_F / |lam1 - lam2| (first-order: phi moves by e / gap for a
backward error e); FP64 eigenvalues 1e-14 ||A||_F, phi 1e-14 ||A||_F / gap. At A11 = A22 (a tenth of
the mixed workload) phi = +-pi/4 exactly by the sign(0) = +1 reading.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1306_6291_gb300 import kdiag as K
from parity import planes_to_rows

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _check(A, lam, phi, tol_lam, tol_phi):
    Ar = planes_to_rows(A)
    lo, po = oracle.eig2(Ar)
    lg, pg = planes_to_rows(lam), phi.double().cpu().numpy()
    fro = np.sqrt(Ar[:, 0] ** 2 + Ar[:, 1] ** 2 + 2 * Ar[:, 2] ** 2)
    fro = np.where(fro > 0, fro, 1)
    assert np.max(np.abs(lg - lo) / fro[:, None]) < tol_lam
    gap = np.abs(lo[:, 0] - lo[:, 1])
    ok = gap > 0
    assert np.max(np.abs(pg - po)[ok] * gap[ok] / fro[ok]) < tol_phi
    return Ar, lo, po, lg, pg


def test_eig2_f32_normal_with_ties():
    A = W.sym2_normal_ties(1 << 16, seed=0, device=DEV)
    lam, phi, D = K.eig2(A, D=True)
    Ar, lo, po, lg, pg = _check(A, lam, phi, 2e-6, 1e-6)
    tie = Ar[:, 0] == Ar[:, 1]
    assert tie.mean() > 0.08
    nz = tie & (Ar[:, 2] != 0)
    assert np.all(np.abs(np.abs(pg[nz]) - np.pi / 4) < 1e-7)
    # D = R(phi) (Eq. (2.5)) and it diagonalizes A (Eq. (3.4))
    Dg = planes_to_rows(D).reshape(-1, 2, 2)
    np.testing.assert_allclose(Dg[:, 0, 0], np.cos(pg), atol=2e-7)
    np.testing.assert_allclose(Dg[:, 1, 0], np.sin(pg), atol=2e-7)
    M = np.stack([Ar[:, 0], Ar[:, 2], Ar[:, 2], Ar[:, 1]], 1).reshape(-1, 2, 2)
    rec = np.einsum("nij,nj,nkj->nik", Dg, lg, Dg)
    fro = np.linalg.norm(M, axis=(1, 2))
    assert np.max(np.linalg.norm(rec - M, axis=(1, 2)) / fro) < 4e-6


def test_eig2_f64():
    A = W.sym2_normal_ties(1 << 16, seed=1, device=DEV).double()
    lam, phi, _ = K.eig2(A)
    _check(A, lam, phi, 1e-14, 1e-14)


def test_eig2_full_size_sampled():
    n = 1 << 25
    A = W.sym2_normal_ties(n, seed=0, device=DEV)
    lam, phi, _ = K.eig2(A)
    rng = np.random.default_rng(1)
    idx = torch.as_tensor(np.unique(np.concatenate([np.arange(1000), np.arange(n - 1000, n),
                                                    rng.integers(0, n, 20000)])), device=DEV)
    _check(A[:, idx], lam[:, idx], phi[idx], 2e-6, 1e-6)


def test_eig2_special_and_nonfinite():
    rows = np.array([[4, 4, 0], [2, 2, 1], [2, 2, -1], [1, 3, 0], [0, 0, 0], [1e30, -1e30, 1e29],
                     [np.nan, 1, 0], [1, np.inf, 0]])
    A = torch.as_tensor(rows.T.copy(), dtype=torch.float32, device=DEV)
    lam, phi, _ = K.eig2(A)
    l, p = planes_to_rows(lam), phi.double().cpu().numpy()
    np.testing.assert_allclose(l[:6], [[4, 4], [3, 1], [3, 1], [1, 3], [0, 0], l[5]], rtol=1e-6)
    np.testing.assert_allclose(p[:5], [0, np.pi / 4, -np.pi / 4, 0, 0], atol=1e-7)
    assert np.isnan(l[6:]).all() and np.isnan(p[6:]).all()


def test_eig2_ties_with_underflowing_a12():
    """A11 = A22 with A12 so small against them that 4 A12^2 is subnormal or zero (FP32: 1e-20 to
    1e-40 of the diagonal; FP64: 1e-160 to 1e-300): the tie rule still gives phi = sign(A12) pi/4
    with D = R(phi), and the eigenvalues are those of the oracle."""
    for dtype, exps, tol in ((torch.float32, (-20, -25, -30, -35, -40), 2e-7),
                             (torch.float64, (-160, -200, -250, -300), 1e-15)):
        rows = [[a, a, sg * 1.3 * 10.0 ** e] for e in exps for a, sg in ((1.0, 1), (-1.5, -1), (0.75, 1))]
        A = torch.as_tensor(np.array(rows).T.copy(), dtype=dtype, device=DEV)
        lam, phi, D = K.eig2(A, D=True)
        Ar = planes_to_rows(A)
        assert np.all(Ar[:, 2] != 0)
        p = phi.double().cpu().numpy()
        np.testing.assert_allclose(p, np.sign(Ar[:, 2]) * np.pi / 4, rtol=0, atol=tol)
        Dg = planes_to_rows(D).reshape(-1, 2, 2)
        np.testing.assert_allclose(Dg[:, 0, 0], np.cos(p), rtol=0, atol=tol)
        np.testing.assert_allclose(Dg[:, 1, 0], np.sin(p), rtol=0, atol=tol)
        lo, _ = oracle.eig2(Ar)
        np.testing.assert_allclose(planes_to_rows(lam), lo, rtol=tol, atol=0)


def test_eig2_adjoint_matches_oracle():
    A = W.sym2_normal_ties(1 << 14, seed=2, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(3)
    lb = torch.randn(2, A.shape[1], generator=g, device=DEV)
    pb = torch.randn(A.shape[1], generator=g, device=DEV)
    ab = K.eig2_adjoint(A, lb, pb)
    Ar = planes_to_rows(A)
    ref = oracle.eig2_adjoint(Ar, planes_to_rows(lb), pb.double().cpu().numpy(), gap_mask=1e-6)
    lo, _ = oracle.eig2(Ar)
    fro = np.sqrt(Ar[:, 0] ** 2 + Ar[:, 1] ** 2 + 2 * Ar[:, 2] ** 2)
    gap = np.abs(lo[:, 0] - lo[:, 1]) / fro
    ok = gap > 1e-3
    scale = np.abs(ref).max(1)
    err = np.abs(planes_to_rows(ab) - ref).max(1) / np.maximum(scale, 1e-30)
    # FP32 relative accuracy of phi's derivative ~ eps / relative gap
    assert np.max(err[ok] * gap[ok]) < 1e-5


def test_eig2_autograd_fp64_gradcheck():
    g = torch.Generator(device=DEV).manual_seed(4)
    A = torch.randn(3, 8, generator=g, device=DEV, dtype=torch.float64)
    A[0] += 3.0          # keep the two eigenvalues apart
    A.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: K.Eig2Fn.apply(X), (A,), eps=1e-6, atol=1e-7)


def test_eig2_64bit_plane_offsets_give_the_same_results():
    """Plane strides at or above 858,993,459 elements take the 2x2 kernels' 64-bit offset
    variants; results must equal those of a contiguous batch. About 34 GB of device memory."""
    n, ld = 50001, 858993459 + 5
    A = W.sym2_normal_ties(n, seed=7, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(8)
    lb, pb = torch.randn(2, n, generator=g, device=DEV), torch.randn(n, generator=g, device=DEV)
    lam, phi, D = K.eig2(A, D=True)
    ab = K.eig2_adjoint(A, lb, pb)
    h = torch.cuda.current_stream().cuda_stream
    big = torch.empty(10, ld, device=DEV)
    Ab, Lb, Pb, Db = big[0:3], big[3:5], big[5], big[6:10]
    Ab[:, :n] = A
    assert K.kd_eig2_sym(Ab.data_ptr(), K.KD_F32, n, ld, Lb.data_ptr(), Pb.data_ptr(), Db.data_ptr(), K.KD_F32, None,
                         h) == K.KD_OK
    assert torch.equal(Lb[:, :n], lam) and torch.equal(Pb[:n], phi) and torch.equal(Db[:, :n], D)
    Lb[:, :n] = lb
    Pb[:n] = pb
    out = big[6:9]
    assert K.kd_eig2_sym_adjoint(Ab.data_ptr(), K.KD_F32, n, ld, Lb.data_ptr(), Pb.data_ptr(), out.data_ptr(), None,
                                 h) == K.KD_OK
    assert torch.equal(out[:, :n], ab)
    del big
    torch.cuda.empty_cache()
