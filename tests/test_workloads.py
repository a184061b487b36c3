"""Host-side checks of the seeded input generators (shapes, determinism, the stated structure)."""
import torch

import workloads as W


def test_uniform_is_seeded_and_in_range():
    a = W.sym3_uniform(1000, seed=0)
    b = W.sym3_uniform(1000, seed=0)
    c = W.sym3_uniform(1000, seed=1)
    assert a.shape == (6, 1000) and a.dtype == torch.float64
    assert torch.equal(a, b) and not torch.equal(a, c)
    assert a.abs().max() <= 1


def test_precision_groups_have_the_stated_spectra():
    A, grp = W.sym3_precision(4000, seed=0)
    assert A.dtype == torch.float32 and A.shape == (6, 4000)
    assert grp.bincount().tolist() == [1000] * 4
    M = torch.stack([A[0], A[3], A[4], A[3], A[1], A[5], A[4], A[5], A[2]], 1).reshape(-1, 3, 3).double()
    w = torch.linalg.eigvalsh(M)
    spread = (w[:, 2] - w[:, 0]).abs()
    scale = w.abs().max(1).values
    gmin = torch.minimum(w[:, 1] - w[:, 0], w[:, 2] - w[:, 1])
    g1 = grp == 1
    # float32 rounding of A moves eigenvalues by ~6e-8 |A|, so the 1e-6 pair stays within ~2e-6
    assert (gmin[g1] / scale[g1]).max() < 3e-6
    g2 = grp == 2
    assert (spread[g2] / scale[g2]).max() < 1e-6
    g3 = grp == 3
    assert torch.all(A[3:, g3] == 0)
    mags = A.abs().amax(0)
    assert mags.max() > 1e10 and mags.min() < 1e-10


def test_ties_fraction_and_gapped_filter():
    B = W.sym2_normal_ties(20000, seed=3)
    frac = (B[0] == B[1]).float().mean().item()
    assert 0.09 < frac < 0.11
    C = W.sym3_normal_gapped(5000, seed=4, min_gap=1e-2)
    assert W.min_eigen_gap(C).min() >= 1e-2


def test_structure_tensor_field_is_symmetric_psd_and_bf16():
    S = W.structure_tensor_field((16, 16, 8), seed=0)
    assert S.shape == (6, 16 * 16 * 8) and S.dtype == torch.bfloat16
    M = torch.stack([S[0], S[3], S[4], S[3], S[1], S[5], S[4], S[5], S[2]], 1).reshape(-1, 3, 3).double()
    w = torch.linalg.eigvalsh(M)
    # a blurred outer product is positive semidefinite up to bf16 rounding
    assert (w[:, 0] / w[:, 2].clamp_min(1e-30)).min() > -0.05


def test_jacobi_gap_filter_matches_lapack():
    A = W.sym3_normal(3000, seed=9, dtype=torch.float64)
    M = torch.stack([A[0], A[3], A[4], A[3], A[1], A[5], A[4], A[5], A[2]], 1).reshape(-1, 3, 3)
    w = torch.linalg.eigvalsh(M)
    ref = torch.minimum(w[:, 1] - w[:, 0], w[:, 2] - w[:, 1])
    assert torch.max(torch.abs(W.min_eigen_gap(A) - ref)) < 1e-12
