"""GPU parity of the 3x3 adjoint (kd_eig3_sym_adjoint) and the autograd wrapper.

The FP32 adjoint recomputes the precision-form decomposition and forms
A_bar = D (diag(lam_bar) + F o (D^T D_bar)) D^T. Against the oracle's analytic adjoint (FP64) on
the gapped workload (every eigen-gap >= 1e-3), with g the smallest eigen-gap over ||A||_F: the
precision form's eigenvectors err by at most dv = 7.1e-7 ||A||_F / gap and its eigenvalues by
dl = 4.2e-7 ||A||_F (the measured figures that tests/test_gpu_accuracy.py asserts with margin).
An entry of A_bar then errs by at most |lam_bar| 2 dv + |D_bar| (2 dv / gap + dl / gap^2), i.e.
err <= (2 * 7.1e-7 + 4.2e-7) (1 + |D_bar| + |lam_bar|) / g^2 = 1.8e-6 scale. The tests ask for
err / scale <= 2e-6 (measured: at most 6.8e-7) and print the largest ratio.
The oracle's adjoint is itself pinned by central finite differences (tests/test_oracle.py); the
FP64 plain GPU adjoint is also checked directly against central differences of the FP64 plain GPU
forward on 4,096 matrices.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1306_6291_gb300 import kdiag as K
from parity import D_rows, planes_to_rows

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _cotangents(n, seed, dtype=torch.float32):
    g = torch.Generator(device=DEV).manual_seed(seed)
    return (torch.randn(3, n, generator=g, device=DEV, dtype=dtype),
            torch.randn(9, n, generator=g, device=DEV, dtype=dtype))


# Bound on max over matrices of err / scale for the FP32 adjoint (see the module docstring).
ADJ32_BOUND = 2e-6


def _adj32_ratio(A, lb, Db, ab, opts=None, idx=None, what=""):
    """err / scale per matrix of an FP32 adjoint ab against the oracle's analytic adjoint, on the
    matrices the GPU and the oracle both take as general (idx: a sample of columns). The oracle's
    cotangents are given the GPU D's column signs. Prints the largest ratio."""
    Aw = A.float()
    if idx is not None:
        Aw, lb, Db, ab = Aw[:, idx], lb[:, idx], Db[:, idx], ab[:, idx]
    Ar = planes_to_rows(Aw)
    lo, Do, _, ko = oracle.eig3(Ar)
    Asel = A if idx is None else A[:, idx]
    _, D, _, kase = K.eig3(Asel.contiguous(), opts, ang=False, kase=True)
    sign = np.sign(np.einsum("nik,nik->nk", D_rows(D), Do))
    lbr = planes_to_rows(lb)
    Dbr = planes_to_rows(Db).reshape(-1, 3, 3) * sign[:, None, :]
    same = (kase.cpu().numpy() == 0) & (ko == 0)
    ref = oracle.eig3_adjoint(Ar[same], lbr[same], Dbr[same], gap_mask=1e-6)
    fro = np.linalg.norm(oracle.unpack3(Ar[same]), axis=(1, 2))
    gmin = np.min(np.abs(lo[same][:, [0, 0, 1]] - lo[same][:, [1, 2, 2]]), 1) / fro
    err = np.abs(planes_to_rows(ab.contiguous())[same] - ref).max(1)
    scale = (1 + np.abs(Dbr[same]).max((1, 2)) + np.abs(lbr[same]).max(1)) / gmin ** 2
    r = err / scale
    print(f"adjoint {what}: max err/scale {r.max():.3e} over {same.sum()} matrices "
          f"(99.9% {np.quantile(r, 0.999):.3e}), general on both sides {same.mean():.4f}")
    return r, same


def test_adjoint_f32_gapped_matches_oracle():
    n = 1 << 14
    A = W.sym3_normal_gapped(n, seed=0, device=DEV)
    lb, Db = _cotangents(n, 1)
    ab = K.eig3_adjoint(A, lb, Db)
    r, same = _adj32_ratio(A, lb, Db, ab, what="f32 gapped 2^14")
    assert same.mean() > 0.99
    assert np.max(r) < ADJ32_BOUND


@pytest.mark.parametrize("variant", ["inv64", "ff", "bf16", "aos"])
def test_adjoint_variants_match_oracle(variant):
    """The other FP32 adjoint instantiations against the oracle's analytic adjoint, as above: FP64
    invariants, float-float invariants, BF16 input (compared on the widened values) and
    array-of-structures records."""
    n = 1 << 13
    A = W.sym3_normal_gapped(n, seed=11, device=DEV)
    if variant == "bf16":
        A = A.to(torch.bfloat16)
    lb, Db = _cotangents(n, 12)
    opts = K.make_opts(invariants={"inv64": K.KD_INV_F64, "ff": K.KD_INV_FLOAT_FLOAT}.get(variant, K.KD_INV_F32))
    if variant == "aos":
        Aw = A.float()
        ab = K.eig3_adjoint_aos(Aw.t().contiguous(), lb.t().contiguous(), Db.t().contiguous(), opts=opts).t()
    else:
        ab = K.eig3_adjoint(A, lb, Db, opts)
    r, same = _adj32_ratio(A, lb, Db, ab, opts, what=variant)
    assert same.mean() > 0.99
    assert np.max(r) < ADJ32_BOUND


def test_adjoint_f64_plain_matches_finite_differences():
    n = 4096
    A = W.sym3_normal_gapped(n, seed=2, device=DEV).double()
    lb, Db = _cotangents(n, 3, torch.float64)
    ab = K.eig3_adjoint(A, lb, Db)
    h = 1e-6
    fd = torch.empty_like(ab)
    for j in range(6):
        Ap, Am = A.clone(), A.clone()
        Ap[j] += h
        Am[j] -= h
        lp, Dp, _, _ = K.eig3(Ap, ang=False)
        lm, Dm, _, _ = K.eig3(Am, ang=False)
        fd[j] = ((lb * (lp - lm)).sum(0) + (Db * (Dp - Dm)).sum(0)) / (2 * h)
    rel = ((fd - ab).abs().amax(0) / ab.abs().amax(0)).cpu().numpy()
    assert np.median(rel) < 1e-7
    assert np.quantile(rel, 0.999) < 1e-4


def test_adjoint_f64_plain_matches_oracle_adjoint():
    n = 4096
    A = W.sym3_normal_gapped(n, seed=4, device=DEV).double()
    lb, Db = _cotangents(n, 5, torch.float64)
    ab = planes_to_rows(K.eig3_adjoint(A, lb, Db))
    ref = oracle.eig3_adjoint(planes_to_rows(A), planes_to_rows(lb), planes_to_rows(Db).reshape(-1, 3, 3))
    rel = np.abs(ab - ref).max(1) / np.abs(ref).max(1)
    assert np.quantile(rel, 0.999) < 1e-7


def test_adjoint_full_size_sampled():
    """The differentiation workload at full size (2^26, gaps >= 1e-3), the launch the benchmark
    times; sampled entries against the oracle."""
    n = 1 << 26
    A = W.sym3_normal_gapped(n, seed=0, device=DEV)
    lb, Db = _cotangents(n, 6)
    ab = K.eig3_adjoint(A, lb, Db)
    rng = np.random.default_rng(2)
    idx = torch.as_tensor(np.unique(np.concatenate([np.arange(512), np.arange(n - 512, n),
                                                    rng.integers(0, n, 3000)])), device=DEV)
    r, same = _adj32_ratio(A, lb, Db, ab, idx=idx, what="f32 full size 2^26 sampled")
    assert same.mean() > 0.99
    assert np.max(r) < ADJ32_BOUND


def test_autograd_eig3_backward_is_the_adjoint():
    A = W.sym3_normal_gapped(2048, seed=7, device=DEV).requires_grad_(True)
    lam, D, ang = K.Eig3Fn.apply(A)
    lb, Db = _cotangents(2048, 8)
    ab = torch.randn(3, 2048, generator=torch.Generator(device=DEV).manual_seed(9), device=DEV)
    (lam * lb).sum().add((D * Db).sum()).add((ang * ab).sum()).backward()
    ref = K.eig3_adjoint(A.detach(), lb, Db, ang_bar=ab)
    assert torch.equal(A.grad, ref)


def test_autograd_eig3_fp64_gradcheck():
    A = W.sym3_normal_gapped(6, seed=9, device=DEV, min_gap=0.2).double().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: K.Eig3Fn.apply(X), (A,), eps=1e-6, atol=1e-6)


def _angle_safe(ang, lam, edge=0.05):
    """Matrices away from gimbal lock and from the ends of the angle ranges (where the returned
    representation jumps), with comfortable gaps."""
    gaps = np.min(np.abs(lam[:, [0, 0, 1]] - lam[:, [1, 2, 2]]), 1)
    return ((gaps > 0.05) & (np.abs(ang[:, 1]) < np.pi / 2 - 0.2) & (np.abs(ang[:, 0]) < np.pi / 2 - edge)
            & (np.abs(ang[:, 2]) < np.pi / 2 - edge))


def test_angle_adjoint_f64_plain_matches_finite_differences_and_oracle():
    n = 4096
    A = W.sym3_normal_gapped(n, seed=10, device=DEV).double()
    lam, _, ang, _ = K.eig3(A)
    keep = torch.as_tensor(_angle_safe(planes_to_rows(ang), planes_to_rows(lam)), device=DEV)
    A = A[:, keep].contiguous()
    m = A.shape[1]
    ab = torch.randn(3, m, generator=torch.Generator(device=DEV).manual_seed(11), device=DEV, dtype=torch.float64)
    g = K.eig3_adjoint(A, None, None, ang_bar=ab)
    h = 1e-6
    fd = torch.empty_like(g)
    for j in range(6):
        Ap, Am = A.clone(), A.clone()
        Ap[j] += h
        Am[j] -= h
        _, _, ap, _ = K.eig3(Ap, lam=False, D=False)
        _, _, am, _ = K.eig3(Am, lam=False, D=False)
        fd[j] = (ab * (ap - am)).sum(0) / (2 * h)
    rel = ((fd - g).abs().amax(0) / g.abs().amax(0)).cpu().numpy()
    assert np.median(rel) < 1e-7 and np.quantile(rel, 0.99) < 1e-4
    ref = oracle.eig3_adjoint(planes_to_rows(A), np.zeros((m, 3)), np.zeros((m, 3, 3)), ang_bar=planes_to_rows(ab))
    rel2 = np.abs(planes_to_rows(g) - ref).max(1) / np.abs(ref).max(1)
    assert np.quantile(rel2, 0.999) < 1e-7


def test_angle_adjoint_f32_matches_oracle():
    n = 1 << 14
    A = W.sym3_normal_gapped(n, seed=12, device=DEV)
    lam, D, ang, kase = K.eig3(A, kase=True)
    Ar = planes_to_rows(A)
    lo, Do, ao, ko = oracle.eig3(Ar)
    keep = _angle_safe(ao, lo) & (kase.cpu().numpy() == 0) & (ko == 0)
    ab = torch.randn(3, n, generator=torch.Generator(device=DEV).manual_seed(13), device=DEV)
    g = planes_to_rows(K.eig3_adjoint(A, None, None, ang_bar=ab))
    ref = oracle.eig3_adjoint(Ar[keep], np.zeros((keep.sum(), 3)), np.zeros((keep.sum(), 3, 3)),
                              ang_bar=planes_to_rows(ab)[keep], gap_mask=1e-6)
    fro = np.linalg.norm(oracle.unpack3(Ar[keep]), axis=(1, 2))
    gmin = np.min(np.abs(lo[keep][:, [0, 0, 1]] - lo[keep][:, [1, 2, 2]]), 1) / fro
    err = np.abs(g[keep] - ref).max(1) / np.abs(ref).max(1)
    # FP32: relative error ~ eps / gap^2 of the 1/(lam_k - lam_j) weights
    assert np.max(err * gmin ** 2) < 1e-5


def test_adjoint_null_cotangents_and_masking():
    A = torch.tensor([[2.0], [2.0], [5.0], [0.0], [0.0], [0.0]], device=DEV)   # two equal eigenvalues
    lb = torch.tensor([[1.0], [2.0], [3.0]], device=DEV)
    Db = torch.ones(9, 1, device=DEV)
    ab = K.eig3_adjoint(A, lb, Db)
    assert torch.isfinite(ab).all()
    ab0 = K.eig3_adjoint(A, None, None)
    assert torch.equal(ab0, torch.zeros_like(ab0))
