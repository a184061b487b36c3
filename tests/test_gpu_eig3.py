"""GPU parity of the 3x3 forward (kd_eig3_sym through the C-ABI) against the CPU oracle.

Tolerances (relative to ||A||_F; definitions in tests/parity.py):
  FP32 precision form (mixed): eigenvalues 2e-6, eigenvectors 1e-5 / gap, reconstruction 4e-6;
    orthogonality 2e-6 and |det D - 1| 2e-6 (a few FP32 rotations, each exact to ~1 ulp).
  FP64 plain form: eigenvalues 1e-13 against both oracles; D against the method oracle in the
    same labels: the method recovers phi2 from cos^2 phi2 = v, so a rounding difference e in v
    becomes up to sqrt(e) in the angle near 0 or pi/2: with e ~ 1e-15 here, 1e-7 at worst.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1306_6291_gb300 import kdiag as K
from parity import D_rows, definition_errors, euler_D, planes_to_rows, summary, wrap_pi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run(A, **kw):
    opts = kw.pop("opts", None)
    return K.eig3(A, opts=opts, kase=True, **kw)


# ------------------------------------------------------------------------------------------ #
# Plain FP64 form: 65,536 matrices with entries U[-1, 1] from seed 0
# ------------------------------------------------------------------------------------------ #

def test_plain_f64_uniform_65536_matches_method_oracle():
    A = W.sym3_uniform(65536, seed=0, device=DEV)
    lam, D, ang, kase = run(A)
    Ar = planes_to_rows(A)
    lo, Do, ao, ko = oracle.eig3(Ar)
    lg, Dg, ag = planes_to_rows(lam), D_rows(D), planes_to_rows(ang)
    fro = np.linalg.norm(oracle.unpack3(Ar), axis=(1, 2))
    assert np.array_equal(kase.cpu().numpy(), ko.astype(np.uint8))
    assert np.max(np.abs(lg - lo) / fro[:, None]) < 1e-13
    assert np.max(np.abs(Dg - Do)) < 1e-7
    assert np.quantile(np.abs(Dg - Do).max((1, 2)), 0.999) < 1e-10
    assert np.max(np.abs(euler_D(ag) - Dg)) < 1e-13
    errs = summary(definition_errors(Ar, lg, Dg))
    assert errs["lam"] < 1e-13 and errs["rec"] < 1e-10 and errs["orth"] < 1e-14 and errs["det"] < 1e-14


# ------------------------------------------------------------------------------------------ #
# FP32 precision form on the four groups of the precision workload
# ------------------------------------------------------------------------------------------ #

@pytest.fixture(scope="module")
def precision_small():
    A, grp = W.sym3_precision(1 << 16, seed=0, device=DEV)
    return A, grp


@pytest.mark.parametrize("inv", [K.KD_INV_F32, K.KD_INV_F64, K.KD_INV_FLOAT_FLOAT])
def test_mixed_f32_precision_groups_vs_definition(precision_small, inv):
    A, grp = precision_small
    opts = K.make_opts(form=K.KD_FORM_MIXED, invariants=inv)
    lam, D, ang, kase = run(A, opts=opts)
    Ar = planes_to_rows(A)
    g = grp.cpu().numpy()
    lg, Dg = planes_to_rows(lam), D_rows(D)
    errs = definition_errors(Ar, lg, Dg)
    for k in range(4):
        s = {name: float(np.max(np.abs(v[g == k] - (1 if name == "det" else 0)))) for name, v in errs.items()}
        assert s["lam"] < 2e-6, (W.GROUPS[k], s)
        assert s["ev"] < 1e-5, (W.GROUPS[k], s)
        assert s["rec"] < 4e-6, (W.GROUPS[k], s)
        assert s["orth"] < 2e-6 and s["det"] < 2e-6, (W.GROUPS[k], s)
    # the Euler angles rebuild D (Eq. (6.5))
    assert np.max(np.abs(euler_D(planes_to_rows(ang)) - Dg)) < 2e-6


def test_mixed_f32_labels_and_angles_match_method_oracle():
    """Where both sides take the general branch, eigen-gaps are comfortable and the angles are
    away from the edges at which the paper calls a sign arbitrary, the FP32 form returns the
    method's labels and angles."""
    A = W.sym3_normal(1 << 16, seed=3, device=DEV)
    lam, D, ang, kase = run(A)
    Ar = planes_to_rows(A)
    lo, Do, ao, ko = oracle.eig3(Ar)
    lg, ag, kg = planes_to_rows(lam), planes_to_rows(ang), kase.cpu().numpy()
    fro = np.linalg.norm(oracle.unpack3(Ar), axis=(1, 2))
    gaps = np.min(np.abs(lo[:, [0, 0, 1]] - lo[:, [1, 2, 2]]), 1) / fro
    edge = 2e-2
    ok = ((kg == 0) & (ko == 0) & (gaps > 1e-2) & (np.abs(ao[:, 0]) < math.pi / 2 - edge)
          & (np.abs(ao[:, 1]) < math.pi / 2 - edge) & (np.abs(ao[:, 2]) < math.pi / 2 - edge))
    assert ok.mean() > 0.5
    assert np.max(np.abs(lg[ok] - lo[ok]) / fro[ok, None]) < 2e-6
    assert np.max(np.abs(wrap_pi(ag[ok] - ao[ok]))) < 1e-4


def test_fp32_euler_angles_match_float64_atan2_of_D():
    """The FP32 kernels evaluate atan2 with their own minimax polynomial (relative error 1.5e-8
    on [0, 1]) after range reduction; the angles they return agree with float64 atan2 of the same
    D to a few FP32 ulp of pi."""
    A = W.sym3_normal(1 << 16, seed=12, device=DEV)
    lam, D, ang, kase = run(A)
    Dg, ag = D_rows(D), planes_to_rows(ang)
    c2 = np.hypot(Dg[:, 1, 2], Dg[:, 2, 2])
    phi1 = np.arctan2(-Dg[:, 1, 2], Dg[:, 2, 2])
    phi2 = np.arctan2(Dg[:, 0, 2], c2)
    c1, s1 = Dg[:, 2, 2] / c2, -Dg[:, 1, 2] / c2
    phi3 = np.arctan2(c1 * Dg[:, 1, 0] + s1 * Dg[:, 2, 0], c1 * Dg[:, 1, 1] + s1 * Dg[:, 2, 1])
    ref = np.stack([phi1, phi2, phi3], 1)
    ok = c2 > 1e-3          # away from gimbal lock, where phi1 and phi3 are not individually defined
    assert np.max(np.abs(wrap_pi(ag[ok] - ref[ok]))) < 1e-6
    assert np.max(np.abs(ag[:, 1] - phi2)) < 1e-6


@pytest.mark.parametrize("inv", [K.KD_INV_F64, K.KD_INV_FLOAT_FLOAT])
def test_plain_f32_with_accurate_invariants(inv):
    """The plain FP32 form (no refinement) with FP64 or compensated float-float invariants: the
    discriminant no longer loses its digits to cancellation, so where the method takes the
    general branch its FP32 eigenvalues are accurate to a few FP32 ulps of ||A||_F (with FP32
    invariants they err by up to 5e-5, test_plain_f32_is_the_method_in_fp32). D keeps the
    sqrt(eps_32) sensitivity of the angle formulas, which only the refinement removes."""
    A = W.sym3_normal(1 << 15, seed=4, device=DEV)
    lam, D, ang, kase = run(A, opts=K.make_opts(form=K.KD_FORM_PLAIN, invariants=inv))
    errs = definition_errors(planes_to_rows(A), planes_to_rows(lam), D_rows(D))
    k = kase.cpu().numpy()
    lam32, _, _, k32 = run(A, opts=K.make_opts(form=K.KD_FORM_PLAIN))
    e32 = definition_errors(planes_to_rows(A), planes_to_rows(lam32), D_rows(D))["lam"]
    g = (k == 0) & (k32.cpu().numpy() == 0)
    print(f"plain FP32, invariants {inv}: general-case lam error {errs['lam'][k == 0].max():.2e} "
          f"(FP32 invariants {e32[g].max():.2e}), rec {errs['rec'].max():.2e}")
    assert np.max(errs["lam"][k == 0]) < 1e-6
    assert np.max(errs["lam"][k == 1]) < 2e-3
    assert np.max(errs["rec"]) < 3e-3
    assert np.max(errs["orth"]) < 2e-6


def test_plain_f32_is_the_method_in_fp32():
    """The plain FP32 form (no refinement) is the paper's method in FP32. Its D carries the
    sqrt(eps_32) sensitivity of phi = arccos(sqrt(v)) (reconstruction up to ~1e-3), and with two
    eigenvalues closer than tau2 = 3e-3 of the spread it returns their mean for both (the
    paper's lam1 = lam2 = lam), off by up to tau2 / 2 of the spread. The refinement of the
    precision form removes both."""
    A = W.sym3_normal(1 << 15, seed=4, device=DEV)
    lam, D, ang, kase = run(A, opts=K.make_opts(form=K.KD_FORM_PLAIN))
    errs = definition_errors(planes_to_rows(A), planes_to_rows(lam), D_rows(D))
    k = kase.cpu().numpy()
    assert np.max(errs["lam"][k == 0]) < 5e-5
    assert np.max(errs["lam"][k == 1]) < 2e-3
    assert np.max(errs["rec"]) < 3e-3
    assert np.max(errs["orth"]) < 2e-6


# ------------------------------------------------------------------------------------------ #
# The precision workload at full size (2^24), as the benchmark launches it
# ------------------------------------------------------------------------------------------ #

def _gpu_properties(A, lam, D, chunk=1 << 22):
    """Reconstruction and orthogonality of every matrix, computed on the GPU in float64."""
    n = A.shape[1]
    worst_rec, worst_orth = 0.0, 0.0
    I = torch.eye(3, device=A.device, dtype=torch.float64)
    for s in range(0, n, chunk):
        a = A[:, s:s + chunk].double()
        M = torch.stack([a[0], a[3], a[4], a[3], a[1], a[5], a[4], a[5], a[2]], 1).reshape(-1, 3, 3)
        Dm = D[:, s:s + chunk].double().t().reshape(-1, 3, 3)
        l = lam[:, s:s + chunk].double().t()
        rec = torch.einsum("nij,nj,nkj->nik", Dm, l, Dm)
        fro = torch.linalg.matrix_norm(M)
        worst_rec = max(worst_rec, float((torch.linalg.matrix_norm(rec - M) / fro).max()))
        worst_orth = max(worst_orth, float((Dm.transpose(1, 2) @ Dm - I).abs().amax()))
    return worst_rec, worst_orth


def test_mixed_f32_precision_full_size_sampled():
    n = 1 << 24
    A, grp = W.sym3_precision(n, seed=0, device=DEV)
    lam, D, ang, kase = run(A)
    rec, orth = _gpu_properties(A, lam, D)
    assert rec < 4e-6 and orth < 2e-6
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([np.arange(2048), np.arange(n - 2048, n),
                                    rng.integers(0, n, 12000)]))
    it = torch.as_tensor(idx, device=DEV)
    errs = summary(definition_errors(planes_to_rows(A[:, it]), planes_to_rows(lam[:, it]), D_rows(D[:, it])))
    assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6


# ------------------------------------------------------------------------------------------ #
# Edge cases
# ------------------------------------------------------------------------------------------ #

@pytest.mark.parametrize("n", [1, 31, 257, 100003])
def test_ragged_sizes(n):
    A = W.sym3_normal(n, seed=n, device=DEV)
    lam, D, ang, kase = run(A)
    errs = summary(definition_errors(planes_to_rows(A), planes_to_rows(lam), D_rows(D)))
    assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6


def test_empty_batch():
    A = torch.empty(6, 0, device=DEV)
    lam, D, ang, kase = run(A)
    assert lam.shape == (3, 0)


def test_special_inputs():
    rows = np.array([
        [0, 0, 0, 0, 0, 0],                    # zero matrix: three equal eigenvalues
        [2.5, 2.5, 2.5, 0, 0, 0],              # alpha I
        [3, 1, 2, 0, 0, 0],                    # diagonal, distinct
        [2, 2, 5, 0, 0, 0],                    # diagonal, two equal
        [1e30, -2e30, 3e29, 1e29, 0, -5e29],   # huge entries
        [1e-30, -2e-30, 3e-29, 1e-29, 0, -5e-31],  # tiny entries
        [1, 1, 1, 1, 1, 1],                    # rank one
        [1, 2, 3, 1e-20, 2e-20, -1e-20],       # nearly diagonal
    ], dtype=np.float64)
    A = torch.as_tensor(rows.T.copy(), dtype=torch.float32, device=DEV)
    lam, D, ang, kase = run(A)
    Ar = planes_to_rows(A)
    errs = summary(definition_errors(Ar, planes_to_rows(lam), D_rows(D)))
    assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6, errs
    k = kase.cpu().numpy()
    assert k[0] == 2 and k[1] == 2 and k[3] == 1
    np.testing.assert_array_equal(D_rows(D)[1], np.eye(3))
    np.testing.assert_allclose(planes_to_rows(lam)[1], [2.5, 2.5, 2.5], rtol=0, atol=0)


def test_e1_block_matrices():
    """A12 = A13 = 0 (f1 = 0, the paper's conjecture (2) case): e1 is an eigenvector. Inputs with
    A11 above, between and below the eigenvalues of the (A22, A33, A23) block, equal to one of them
    (two equal) or to both (three equal), and diagonal ones; the decomposition, the paper's labels
    (general: lam1 >= lam3 >= lam2) and det D = +1 are checked."""
    rng = np.random.default_rng(14)
    rows = []
    for _ in range(2000):
        b = rng.normal(size=3)
        m, r = 0.5 * (b[0] + b[1]), np.hypot(b[0] - b[1], 2 * b[2]) / 2
        for a11 in (m + r + abs(rng.normal()) + 0.1, m, m - r - abs(rng.normal()) - 0.1, m + r, m - r):
            rows.append([a11, b[0], b[1], 0.0, 0.0, b[2]])
        rows.append([b[0], b[1], b[2], 0.0, 0.0, 0.0])
    rows.append([2.0, 2.0, 2.0, 0.0, 0.0, 0.0])
    Ar = np.array(rows)
    A = torch.as_tensor(Ar.T.copy(), dtype=torch.float32, device=DEV)
    lam, D, ang, kase = run(A)
    Af = planes_to_rows(A)
    errs = definition_errors(Af, planes_to_rows(lam), D_rows(D))
    s = summary(errs)
    assert s["lam"] < 2e-6 and s["ev"] < 1e-5 and s["rec"] < 4e-6 and s["orth"] < 2e-6 and s["det"] < 2e-6, s
    lg, k = planes_to_rows(lam), kase.cpu().numpy()
    g = k == 0
    assert np.all(lg[g, 0] >= lg[g, 2]) and np.all(lg[g, 2] >= lg[g, 1])
    assert k[-1] == 2
    assert np.max(np.abs(euler_D(planes_to_rows(ang)) - D_rows(D))) < 2e-6


def test_nonfinite_inputs_give_nan_and_kase_255():
    A = W.sym3_normal(64, seed=5, device=DEV)
    A[0, 3] = float("nan")
    A[4, 10] = float("inf")
    A[2, 20] = -float("inf")
    lam, D, ang, kase = run(A)
    k = kase.cpu().numpy()
    assert k[3] == 255 and k[10] == 255 and k[20] == 255
    bad = [3, 10, 20]
    assert torch.isnan(lam[:, bad]).all() and torch.isnan(D[:, bad]).all() and torch.isnan(ang[:, bad]).all()
    good = np.setdiff1d(np.arange(64), bad)
    assert torch.isfinite(lam[:, good]).all()


def test_strided_planes_and_output_masks():
    n, ld = 1000, 1024
    base = W.sym3_normal(n, seed=6, device=DEV)
    Ap = torch.zeros(6, ld, device=DEV)
    Ap[:, :n] = base
    lam = torch.empty(3, ld, device=DEV)
    s = K.kd_eig3_sym(Ap.data_ptr(), K.KD_F32, n, ld, lam.data_ptr(), None, None, K.KD_F32, None, None,
                      torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_OK
    ref, _, _, _ = run(base)
    torch.cuda.synchronize()
    assert torch.equal(lam[:, :n], ref)


def test_bf16_input_equals_fp32_of_rounded_values():
    """BF16 planes are widened exactly, so the BF16 kernel and the FP32 kernel on the widened
    values compute the same decomposition; the two instantiations may round differently (FMA
    contraction), so they agree to the FP32 tolerances, not bit for bit."""
    A = W.sym3_normal(20000, seed=7, device=DEV)
    Ab = A.to(torch.bfloat16)
    l1, D1, a1, k1 = run(Ab)
    l2, D2, a2, k2 = run(Ab.float())
    Ar = planes_to_rows(Ab.float())
    fro = np.linalg.norm(__import__("oracle").unpack3(Ar), axis=(1, 2))
    assert np.max(np.abs(planes_to_rows(l1) - planes_to_rows(l2)) / fro[:, None]) < 4e-6
    for lam, D in ((l1, D1), (l2, D2)):
        errs = summary(definition_errors(Ar, planes_to_rows(lam), D_rows(D)))
        assert errs["lam"] < 2e-6 and errs["ev"] < 1e-5 and errs["rec"] < 4e-6


def _expected_counts(k):
    base = np.where(k == 255, 255, k & 15)
    unconv = (k != 255) & ((k & 16) != 0)
    return [int(np.sum(base == 0)), int(np.sum(base == 1)), int(np.sum(base == 2)), int(np.sum(base == 255)),
            int(np.sum(unconv))]


def test_stats_counters():
    A, grp = W.sym3_precision(4096, seed=8, device=DEV)
    A[0, 5] = float("nan")
    stats = torch.zeros(5, dtype=torch.int64, device=DEV)
    lam, D, ang, kase = run(A, opts=K.make_opts(stats=stats))
    k = kase.cpu().numpy().astype(np.int64)
    expect = _expected_counts(k)
    assert stats.cpu().tolist() == expect
    assert expect[3] == 1 and expect[2] >= 1024 and expect[4] == 0


@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_unconverged_refinement_is_reported(layout):
    """With max_sweeps = 0 no refinement step runs: every matrix whose D^T A D has an
    off-diagonal above conv_kappa ||A||_F gets kase bit 16 and is counted in stats[4]; with
    max_sweeps = 1 the matrices whose one sweep did not converge are flagged and counted the same
    way; with the default 4 sweeps nothing on the precision workload is. The flagged matrices'
    D^T A D (formed here in float64 from the returned D) is indeed off-diagonal beyond the
    threshold (half of it, for the FP32 rounding of D); the others are within twice it."""
    A, grp = W.sym3_precision(1 << 16, seed=21, device=DEV)
    Ar = planes_to_rows(A)
    M = oracle.unpack3(Ar)
    fro = np.linalg.norm(M, axis=(1, 2))
    seen = {}
    for sweeps in (0, 1, 4):
        stats = torch.zeros(5, dtype=torch.int64, device=DEV)
        o = K.make_opts(max_sweeps=sweeps, stats=stats, layout=K.KD_LAYOUT_AOS if layout == "aos" else K.KD_LAYOUT_SOA)
        if layout == "aos":
            _, Dt, _, kt = K.eig3_aos(A.t().contiguous(), o, kase=True)
            Dm = Dt.double().cpu().numpy().reshape(-1, 3, 3)
        else:
            _, Dt, _, kt = K.eig3(A, o, kase=True)
            Dm = D_rows(Dt)
        k = kt.cpu().numpy().astype(np.int64)
        assert stats.cpu().tolist() == _expected_counts(k)
        flagged = (k != 255) & ((k & 16) != 0)
        B = np.einsum("nji,njk,nkl->nil", Dm, M, Dm)
        off = np.max(np.abs(B[:, [0, 0, 1], [1, 2, 2]]), 1) / fro
        seen[sweeps] = int(flagged.sum())
        if flagged.any():
            assert np.min(off[flagged]) > 0.5 * 3e-7
        # general matrices take the first-order step or converge; both leave O(eps) off-diagonals
        assert np.quantile(off[~flagged], 0.999) < 1e-6
    print(f"unconverged ({layout}): {seen}")
    assert seen[0] > 1000 and seen[1] < seen[0] and seen[4] == 0


def test_host_pipeline_matches_device_calls():
    """kdiag.eig3_host on host planes (several chunks over rotating streams, ragged last chunk)
    returns what the device calls return."""
    n = 100003
    A = W.sym3_normal(n, seed=15, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(16)
    lb, Db = torch.randn(3, n, generator=g, device=DEV), torch.randn(9, n, generator=g, device=DEV)
    out = K.eig3_host(A.cpu().pin_memory(), lb.cpu().pin_memory(), Db.cpu().pin_memory(), chunk=16384, streams=3)
    lam, D, ang, _ = K.eig3(A)
    ab = K.eig3_adjoint(A, lb, Db)
    assert torch.equal(out["lam"], lam.cpu()) and torch.equal(out["D"], D.cpu()) and torch.equal(out["ang"], ang.cpu())
    assert torch.equal(out["A_bar"], ab.cpu())
    # lam alone runs another kernel instantiation: equal up to FP32 rounding of the Rayleigh quotients
    only = K.eig3_host(A.cpu(), outputs=("lam",), chunk=30000, streams=2)
    assert set(only) == {"lam"}
    torch.testing.assert_close(only["lam"], lam.cpu(), rtol=1e-6, atol=1e-6 * float(lam.abs().max()))


def test_host_pipeline_other_dtypes_and_checks():
    """kd_eig3_sym_host with FP64 and BF16 input, angle cotangents and a workspace that is too
    small (rejected before anything is enqueued)."""
    n = 40001
    A64 = W.sym3_uniform(n, seed=2, device=DEV)
    out = K.eig3_host(A64.cpu().pin_memory(), chunk=8192, streams=4)
    lam, D, ang, _ = K.eig3(A64)
    assert torch.equal(out["lam"], lam.cpu()) and torch.equal(out["D"], D.cpu()) and torch.equal(out["ang"], ang.cpu())
    Ab16 = W.sym3_normal(n, seed=4, device=DEV).to(torch.bfloat16)
    g = torch.Generator(device=DEV).manual_seed(5)
    ab = torch.randn(3, n, generator=g, device=DEV)
    out = K.eig3_host(Ab16.cpu().pin_memory(), ang_bar=ab.cpu().pin_memory(), outputs=(), chunk=5000, streams=2)
    assert set(out) == {"A_bar"}
    ref = K.eig3_adjoint(Ab16, None, None, ang_bar=ab)
    assert torch.equal(out["A_bar"], ref.cpu())
    ws = torch.empty(1024, dtype=torch.uint8, device=DEV)
    hA = A64.cpu()
    hl = torch.empty(3, n, dtype=torch.float64)
    st = K.kd_eig3_sym_host(hA.data_ptr(), K.KD_F64, n, None, None, None, hl.data_ptr(), None, None, None, 4096,
                            ws.data_ptr(), ws.numel(), None, [torch.cuda.current_stream().cuda_stream], 1)
    assert st == K.KD_ERR_INVALID_ARG



def test_64bit_plane_offsets_give_the_same_results():
    """Plane strides at or above 429,496,729 elements take the kernels' 64-bit offset variants
    (10 planes of that stride pass 2^32 elements). The same matrices through a contiguous batch
    (32-bit offsets) must give identical forward bits; the adjoint instantiations may contract
    different products into FMAs, so its results agree to FP32 rounding (eigen-gaps >= 1e-3 keep
    the 1/gap weights tame). About 40 GB of device memory."""
    n, ld = 70001, 429496729 + 7
    A = W.sym3_normal_gapped(n, seed=21, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(22)
    lb, Db = torch.randn(3, n, generator=g, device=DEV), torch.randn(9, n, generator=g, device=DEV)
    lam, D, ang, _ = K.eig3(A)
    ab = K.eig3_adjoint(A, lb, Db)
    h = torch.cuda.current_stream().cuda_stream
    big = torch.empty(6 + 3 + 9 + 3, ld, device=DEV)
    Ab, Lb, Bb, Gb = big[0:6], big[6:9], big[9:18], big[18:21]
    Ab[:, :n] = A
    st = K.kd_eig3_sym(Ab.data_ptr(), K.KD_F32, n, ld, Lb.data_ptr(), Bb.data_ptr(), Gb.data_ptr(), K.KD_F32, None,
                       None, h)
    assert st == K.KD_OK
    assert torch.equal(Lb[:, :n], lam) and torch.equal(Bb[:, :n], D) and torch.equal(Gb[:, :n], ang)
    # adjoint: A (6), lam_bar (3), D_bar (9) in, A_bar (6) out, all with the same stride
    big2 = torch.empty(6, ld, device=DEV)
    Lb[:, :n] = lb
    Bb[:, :n] = Db
    st = K.kd_eig3_sym_adjoint(Ab.data_ptr(), K.KD_F32, n, ld, Lb.data_ptr(), Bb.data_ptr(), None, big2.data_ptr(),
                               None, h)
    assert st == K.KD_OK
    torch.testing.assert_close(big2[:, :n], ab, rtol=1e-4, atol=1e-4 * float(ab.abs().max()))
    del big, big2
    torch.cuda.empty_cache()


@pytest.mark.parametrize("want", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)])
def test_every_output_set_agrees_with_the_full_call(want):
    """Each subset of (lam, D, angles) runs its own kernel instantiation (the common ones without
    run-time output checks); all must agree with the full call (with kase requested, the generic
    instantiation) on a ragged batch. The instantiations round differently, so the bound is the
    precision form's own accuracy: eigenvalues ~1e-7 ||A||, eigenvectors ~1e-6 ||A|| / gap (here
    gaps >= 0.1 with ||A|| ~ 3: a few 1e-5), angles the same divided by cos(phi2) for phi1, phi3."""
    n = 100003
    A = W.sym3_normal_gapped(n, seed=31, device=DEV, min_gap=0.1)
    lam0, D0, ang0, k0 = K.eig3(A, kase=True)
    lam, D, ang, _ = K.eig3(A, lam=bool(want[0]), D=bool(want[1]), ang=bool(want[2]))
    if lam is not None:
        torch.testing.assert_close(lam, lam0, rtol=0, atol=1e-6 * float(lam0.abs().max()))
    if D is not None:
        torch.testing.assert_close(D, D0, rtol=0, atol=5e-5)
    if ang is not None:
        # phi1 and phi3 in (-pi, pi] wrap around at +-pi
        c2 = torch.cos(ang0[1]).abs().clamp_min(1e-6)
        tol = torch.stack([5e-5 / c2, torch.full_like(c2, 5e-5), 5e-5 / c2])
        d = torch.remainder(ang.double() - ang0.double() + math.pi, 2 * math.pi) - math.pi
        assert bool((d.abs() <= tol).all()), float((d.abs() / tol).max())
    assert int((k0 == 255).sum()) == 0


def test_gpu_angles_satisfy_the_rotation_identities():
    """The paper's identities g1 = R(phi1) f1 and g2 = R(2 phi1) f2 (f from A, g from the
    eigenvalues and phi2, phi3; Eqs. (5.5)-(5.8)) for the FP32 precision form's eigenvalues and
    angles on well-separated spectra, to FP32 accuracy; and exactly as for the oracle for the
    FP64 plain form."""
    n = 20000
    for dtype, tol in ((torch.float32, 2e-5), (torch.float64, 1e-9)):
        A = W.sym3_normal_gapped(n, seed=41, device=DEV, min_gap=0.1)
        if dtype == torch.float64:
            A = A.double()
        lam, _, ang, kase = K.eig3(A, D=False, kase=True)
        Ar, lr, ar = planes_to_rows(A), planes_to_rows(lam), planes_to_rows(ang)
        l1, l2, l3, p1, p2, p3 = lr[:, 0], lr[:, 1], lr[:, 2], ar[:, 0], ar[:, 1], ar[:, 2]
        v, w = np.cos(p2) ** 2, np.cos(p3) ** 2
        f1 = np.stack([Ar[:, 3], -Ar[:, 4]], 1)
        f2 = np.stack([Ar[:, 1] - Ar[:, 2], -2 * Ar[:, 5]], 1)
        g1 = np.stack([0.5 * (l1 - l2) * np.cos(p2) * np.sin(2 * p3), 0.5 * ((l1 - l2) * w + l2 - l3) * np.sin(2 * p2)], 1)
        g2 = np.stack([(l1 - l2) * (1 + (v - 2) * w) + (l2 - l3) * v, (l1 - l2) * np.sin(p2) * np.sin(2 * p3)], 1)

        def rot(phi, x):
            return np.stack([np.cos(phi) * x[:, 0] - np.sin(phi) * x[:, 1], np.sin(phi) * x[:, 0] + np.cos(phi) * x[:, 1]], 1)

        fro = np.linalg.norm(oracle.unpack3(Ar), axis=(1, 2))[:, None]
        gen = kase.cpu().numpy() == 0
        assert gen.mean() > 0.99
        assert np.max((np.abs(rot(p1, f1) - g1) / fro)[gen]) < tol
        assert np.max((np.abs(rot(2 * p1, f2) - g2) / fro)[gen]) < tol


def test_entries_spanning_sixty_decades():
    """Entries N(0,1) x 10^u, u ~ U[-30, 30] drawn per entry. After the power-of-two prescale most
    entries of such a matrix are tiny or flush to zero, so the e1-block path with blocks far below
    A11, refinement rotations of pairs whose squares underflow, and rotations within 2^-50 of
    gimbal lock all occur (before the fixes about one matrix in 2,000 lost orthogonality or had
    angles that did not reproduce D). The first rows are such inputs: a pair coupled at 1e-26 with
    a subnormal diagonal gap (the Jacobi tangent must stay in [-1, 1]), an e1 block 1e-22 below
    A11 (the block's squares must not underflow) and near-lock rotations whose cos(phi2)^2
    underflows (the lock rule)."""
    rng = np.random.default_rng(60)
    n = 1 << 18
    Ar = rng.normal(size=(n, 6)) * 10.0 ** rng.uniform(-30, 30, (n, 6))
    Ar[:5] = [[8.920158700839299e-27, -7.124747206779165e+26, -4.382763166645388e-30, 4.733062351840665e+23,
               -3.8575240302887875e-17, 29212.787109375],
              [-3.7426050076045676e+27, 3.1435804942797295e-29, -286875.03125, -4.594969238803889e-20,
               -5.675832756048558e-23, 3.3766763715091076e-18],
              [181639888.0, -0.9293251633644104, 4.1694198094077706e-10, -1.1247333375018023e-28,
               -2.2457428576266522e-14, 9690.4365234375],
              [82280292352.0, -1.4883186758088719e-19, -1.4388906017033423e-18, 9.18916071707132e-12,
               -3.055289347319122e-25, 16032855.0],
              [-1.1423410286669195e+25, -3.556236333679408e-05, -5336.9609375, 1039.0908203125,
               2.078493742302198e-22, 9.68210644309892e+21]]
    A = torch.as_tensor(Ar.T.astype(np.float32).copy(), device=DEV)
    lam, D, ang, kase = run(A)
    Af = planes_to_rows(A)
    errs = definition_errors(Af, planes_to_rows(lam), D_rows(D))
    s = summary(errs)
    assert s["lam"] < 2e-6 and s["ev"] < 1e-5 and s["rec"] < 4e-6 and s["orth"] < 2e-6 and s["det"] < 2e-6, s
    assert np.max(np.abs(euler_D(planes_to_rows(ang)) - D_rows(D))) < 2e-6
    for adj_ang in (False, True):
        g = torch.Generator(device=DEV).manual_seed(3)
        lb, Db, ab = (torch.randn(k, n, generator=g, device=DEV) for k in (3, 9, 3))
        Ab = K.eig3_adjoint(A, lb, Db, ang_bar=ab if adj_ang else None)
        assert bool(torch.isfinite(Ab).all())
