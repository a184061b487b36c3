"""Pins of the CPU oracle against facts fixed by the paper and by mathematics, not by itself.

Each test names what pins it: an independent library (LAPACK eigh, scipy's Euler rotations),
hand-worked cases (tests/golden/handworked.json), inputs built from known angles and
eigenvalues, invariants of A = D Lambda D^T (Eq. (2.1)), the symmetries stated in Sections 3
and 4, and central finite differences for the adjoints.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handworked.json")


def _rng(seed):
    return np.random.default_rng(seed)


def _fro(A):
    return np.linalg.norm(oracle.unpack3(A), axis=(1, 2))


def _build_from(R, lam):
    """A = R diag(lam) R^T packed (n, 6)."""
    M = np.einsum("nij,nj,nkj->nik", R, lam, R)
    return np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]], 1)


# ------------------------------------------------------------------------------------------ #
# Eigenvalues (Section 4) against LAPACK and against the Jacobi definition oracle
# ------------------------------------------------------------------------------------------ #

def test_eig3_eigenvalues_match_lapack_uniform():
    A = _rng(0).uniform(-1, 1, (50000, 6))
    lam, D, ang, kase = oracle.eig3(A)
    ref = np.linalg.eigvalsh(oracle.unpack3(A))
    err = np.abs(np.sort(lam, 1) - ref) / _fro(A)[:, None]
    assert err.max() < 1e-13          # the FP64 eigenvalue tolerance of the plain form
    assert np.all(kase == 0)


def test_eig3_label_order_is_max_min_mid():
    A = _rng(1).normal(size=(20000, 6))
    lam, _, _, kase = oracle.eig3(A)
    g = kase == 0
    assert np.all(lam[g, 0] >= lam[g, 2]) and np.all(lam[g, 2] >= lam[g, 1])   # Eqs. (4.10)-(4.12)


def test_jacobi_definition_oracle_matches_lapack():
    A = _rng(2).normal(size=(3000, 6)) * 10.0 ** _rng(3).uniform(-5, 5, (3000, 1))
    lam, V, sweeps = oracle.jacobi3(A)
    M = oracle.unpack3(A)
    w, U = np.linalg.eigh(M)
    fro = _fro(A)
    assert np.max(np.abs(lam[:, ::-1] - w) / fro[:, None]) < 1e-14
    # eigenvectors up to sign
    dots = np.abs(np.einsum("nik,nik->nk", V[:, :, ::-1], U))
    assert np.max(1 - dots) < 1e-12
    # A V = V Lambda and V^T V = I
    res = np.einsum("nij,njk->nik", M, V) - V * lam[:, None, :]
    assert np.max(np.linalg.norm(res, axis=(1, 2)) / fro) < 1e-14
    assert np.max(np.abs(np.einsum("nji,njk->nik", V, V) - np.eye(3))) < 1e-14
    assert sweeps.max() < 20


def test_eig3_matches_jacobi_definition_on_normal_inputs():
    A = _rng(4).normal(size=(20000, 6))
    lam, D, _, kase = oracle.eig3(A)
    lj, V, _ = oracle.jacobi3(A)
    fro = _fro(A)
    assert np.max(np.abs(np.sort(lam, 1)[:, ::-1] - lj) / fro[:, None]) < 1e-13


# ------------------------------------------------------------------------------------------ #
# Invariants of A = D Lambda D^T (Eq. (2.1)), D a rotation (Section 2)
# ------------------------------------------------------------------------------------------ #

def test_eig3_decomposition_invariants():
    rng = _rng(5)
    A = rng.uniform(-1, 1, (20000, 6)) * 10.0 ** rng.uniform(-8, 8, (20000, 1))
    lam, D, ang, kase = oracle.eig3(A)
    M = oracle.unpack3(A)
    fro = _fro(A)
    rec = np.einsum("nij,nj,nkj->nik", D, lam, D)
    assert np.max(np.linalg.norm(rec - M, axis=(1, 2)) / fro) < 1e-10
    assert np.max(np.abs(np.einsum("nji,njk->nik", D, D) - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(D) - 1)) < 1e-14
    tr = M[:, 0, 0] + M[:, 1, 1] + M[:, 2, 2]
    assert np.max(np.abs(lam.sum(1) - tr) / fro) < 1e-14
    assert np.max(np.abs(np.prod(lam, 1) - np.linalg.det(M)) / fro ** 3) < 1e-14
    assert np.max(np.abs(np.sum(lam ** 2, 1) - fro ** 2) / fro ** 2) < 1e-14


# ------------------------------------------------------------------------------------------ #
# Angles (Sections 5 and 6)
# ------------------------------------------------------------------------------------------ #

def test_euler_angles_rebuild_D_like_scipy_intrinsic_xyz():
    """Eq. (6.5): D = R1(phi1) R2(phi2) R3(phi3) is the intrinsic X-Y'-Z'' Euler sequence with
    angles (phi1, phi2, phi3); scipy's 'XYZ' (upper case = intrinsic) builds the same matrix."""
    A = _rng(6).normal(size=(5000, 6))
    lam, D, ang, kase = oracle.eig3(A)
    R = Rotation.from_euler("XYZ", ang).as_matrix()
    assert np.max(np.abs(R - D)) < 1e-14


def test_eig3_recovers_known_angles_and_labels():
    """A = R1 R2 R3 diag(lam) (R1 R2 R3)^T with lam1 > lam3 > lam2 and angles inside the ranges
    the method returns (phi1 in (-pi/2, pi/2], phi2, phi3 in [-pi/2, pi/2]) gives back the
    same angles and labels, away from the edges where the paper says a sign is arbitrary."""
    rng = _rng(7)
    n = 20000
    edge = 1e-2
    ang = rng.uniform(-math.pi / 2 + edge, math.pi / 2 - edge, (n, 3))
    R = Rotation.from_euler("XYZ", ang).as_matrix()
    l = np.sort(rng.normal(size=(n, 3)), 1)[:, ::-1]
    keep = np.minimum(l[:, 0] - l[:, 1], l[:, 1] - l[:, 2]) > 1e-2
    lam = np.stack([l[:, 0], l[:, 2], l[:, 1]], 1)[keep]          # paper labels: max, min, mid
    R, ang = R[keep], ang[keep]
    A = _build_from(R, lam)
    lo, D, ao, kase = oracle.eig3(A)
    assert np.all(kase == 0)
    assert np.max(np.abs(lo - lam)) < 1e-12
    assert np.max(np.abs(ao - ang)) < 1e-7
    assert np.quantile(np.abs(ao - ang).max(1), 0.99) < 1e-10
    assert np.max(np.abs(D - R)) < 1e-7


def test_eig3_recovers_pythagorean_rotation_exactly():
    """Rotations with rational cosines (3-4-5, 5-12-13, 4-3-5 triangles) give an A whose entries
    are exact rationals; the angles are atan2 of the triangle's legs."""
    c1, s1 = Fraction(4, 5), Fraction(3, 5)
    c2, s2 = Fraction(12, 13), Fraction(5, 13)
    c3, s3 = Fraction(3, 5), Fraction(4, 5)
    R1 = [[1, 0, 0], [0, c1, -s1], [0, s1, c1]]
    R2 = [[c2, 0, s2], [0, 1, 0], [-s2, 0, c2]]
    R3 = [[c3, -s3, 0], [s3, c3, 0], [0, 0, 1]]

    def mm(X, Y):
        return [[sum(X[i][k] * Y[k][j] for k in range(3)) for j in range(3)] for i in range(3)]

    Dq = mm(mm(R1, R2), R3)
    lam = [Fraction(7), Fraction(-2), Fraction(3)]                 # lam1 > lam3 > lam2
    Mq = [[sum(Dq[i][k] * lam[k] * Dq[j][k] for k in range(3)) for j in range(3)] for i in range(3)]
    A = np.array([[float(Mq[0][0]), float(Mq[1][1]), float(Mq[2][2]),
                   float(Mq[0][1]), float(Mq[0][2]), float(Mq[1][2])]])
    lo, D, ao, kase = oracle.eig3(A)
    assert kase[0] == 0
    np.testing.assert_allclose(lo[0], [7, -2, 3], atol=1e-13)
    np.testing.assert_allclose(ao[0], [math.atan2(3, 4), math.atan2(5, 12), math.atan2(4, 3)], atol=1e-12)
    np.testing.assert_allclose(D[0], np.array(Dq, dtype=float), atol=1e-13)


def _paper_f_g(A, lam, ang):
    """f1, f2 (Eqs. (5.5)-(5.6)) from the packed matrix and g1, g2 (Eqs. (5.7)-(5.8)) from the
    paper's labels (lam1, lam2, lam3) and the angles phi2, phi3, as (n, 2) arrays."""
    l1, l2, l3 = lam[:, 0], lam[:, 1], lam[:, 2]
    p2, p3 = ang[:, 1], ang[:, 2]
    v, w = np.cos(p2) ** 2, np.cos(p3) ** 2
    f1 = np.stack([A[:, 3], -A[:, 4]], 1)
    f2 = np.stack([A[:, 1] - A[:, 2], -2 * A[:, 5]], 1)
    g1 = np.stack([0.5 * (l1 - l2) * np.cos(p2) * np.sin(2 * p3),
                   0.5 * ((l1 - l2) * w + l2 - l3) * np.sin(2 * p2)], 1)
    g2 = np.stack([(l1 - l2) * (1 + (v - 2) * w) + (l2 - l3) * v,
                   (l1 - l2) * np.sin(p2) * np.sin(2 * p3)], 1)
    return f1, f2, g1, g2


def _rot2(phi, x):
    c, s = np.cos(phi), np.sin(phi)
    return np.stack([c * x[:, 0] - s * x[:, 1], s * x[:, 0] + c * x[:, 1]], 1)


def test_selected_angles_satisfy_the_rotation_identities():
    """Pin of the sign search and phi1 (Eqs. (5.9)-(5.15)): for the angles the method returns,
    the paper's two identities g1 = R(phi1) f1 and g2 = R(2 phi1) f2 (its computer-algebra
    results) hold, with f from A and g from the eigenvalues and phi2, phi3. A wrong sign of phi2
    or phi3, or a phi1 off by pi/2, breaks at least one of them."""
    A = _rng(21).uniform(-1, 1, (4000, 6))
    lam, _, ang, kase = oracle.eig3(A)
    f1, f2, g1, g2 = _paper_f_g(A, lam, ang)
    fro = _fro(A)[:, None]
    gen = kase == 0
    assert gen.mean() > 0.99
    e1 = np.abs(_rot2(ang[:, 0], f1) - g1)[gen] / fro[gen]
    e2 = np.abs(_rot2(2 * ang[:, 0], f2) - g2)[gen] / fro[gen]
    assert np.max(e1) < 1e-9 and np.max(e2) < 1e-9
    # and the identities are not vacuous: flipping the sign of phi3 breaks them for most matrices
    flipped = ang.copy()
    flipped[:, 2] = -flipped[:, 2]
    _, _, g1f, g2f = _paper_f_g(A, lam, flipped)
    bad = np.maximum(np.abs(_rot2(ang[:, 0], f1) - g1f).max(1), np.abs(_rot2(2 * ang[:, 0], f2) - g2f).max(1))
    assert np.mean(bad[gen] / fro[gen, 0] > 1e-3) > 0.9


def test_q_sign_symmetry():
    """Section 4: flipping the sign of q (A -> -A) flips the leading signs, so the largest
    eigenvalue of -A is minus the smallest of A: labels (lam1, lam2, lam3) -> (-lam2, -lam1, -lam3)."""
    A = _rng(8).normal(size=(20000, 6))
    lp, _, _, kp = oracle.eig3(A)
    lm, _, _, km = oracle.eig3(-A)
    g = (kp == 0) & (km == 0)
    fro = _fro(A)[g, None]
    assert np.max(np.abs(lm[g] - np.stack([-lp[g, 1], -lp[g, 0], -lp[g, 2]], 1)) / fro) < 1e-14


def test_two_equal_special_case_relabels_and_keeps_distinct_vector():
    """Eqs. (5.20)-(5.25): with a double eigenvalue the method relabels lam1 = lam2 = lam, lam3
    the distinct one, and column 3 of D is the distinct eigenvector."""
    rng = _rng(9)
    n = 5000
    R = Rotation.random(n, random_state=10).as_matrix()
    a = rng.normal(size=n)
    b = a + np.sign(rng.normal(size=n)) * rng.uniform(0.5, 2.0, n)
    A = _build_from(R, np.stack([a, a, b], 1))
    lam, D, ang, kase = oracle.eig3(A)
    assert np.all(kase == 1)
    fro = _fro(A)
    assert np.max(np.abs(lam[:, 0] - a) / fro) < 1e-12
    assert np.max(np.abs(lam[:, 1] - a) / fro) < 1e-12
    assert np.max(np.abs(lam[:, 2] - b) / fro) < 1e-13
    dots = np.abs(np.einsum("ni,ni->n", D[:, :, 2], R[:, :, 2]))
    assert np.max(1 - dots) < 1e-6      # the pair mean model error is ~sqrt(eps) in the angle
    rec = np.einsum("nij,nj,nkj->nik", D, lam, D)
    assert np.max(np.linalg.norm(rec - oracle.unpack3(A), axis=(1, 2)) / fro) < 1e-7
    assert np.max(np.abs(ang[:, 2])) == 0.0          # phi3 = 0 (Eq. (5.23))


def test_triple_special_case():
    """Section 5, p = 0: lam1 = lam2 = lam3 and all angles 0."""
    alpha = _rng(11).normal(size=1000) * 10.0 ** _rng(12).uniform(-10, 10, 1000)
    A = np.zeros((1000, 6))
    A[:, :3] = alpha[:, None]
    lam, D, ang, kase = oracle.eig3(A)
    assert np.all(kase == 2)
    np.testing.assert_allclose(lam, np.repeat(alpha[:, None], 3, 1), rtol=1e-15)
    assert np.all(ang == 0) and np.all(D == np.eye(3))


def test_conjecture2_rotation_in_e2_e3_plane():
    """Section 5, conjecture (2) example: A12 = A13 = 0 means a rotation in the e2-e3 plane;
    with e1 the eigenvector of the largest eigenvalue the angles are (phi, 0, 0), phi mod pi."""
    rng = _rng(13)
    n = 3000
    phi = rng.uniform(-math.pi / 2 + 1e-3, math.pi / 2 - 1e-3, n)
    l23 = rng.normal(size=(n, 2))
    lam1 = np.max(l23, 1) + rng.uniform(0.5, 2, n)
    lo, hi = np.min(l23, 1), np.max(l23, 1)
    keep = hi - lo > 1e-3
    R = Rotation.from_euler("XYZ", np.stack([phi, 0 * phi, 0 * phi], 1)).as_matrix()
    A = _build_from(R, np.stack([lam1, lo, hi], 1))[keep]
    lam, D, ang, kase = oracle.eig3(A)
    d = np.abs(np.angle(np.exp(2j * (ang[:, 0] - phi[keep])))) / 2
    assert np.max(d) < 1e-8
    # v = w = 1 here; a rounding error e of v becomes arccos(sqrt(1 - e)) ~ sqrt(e) in the angle,
    # with e ~ eps / (relative gap) <= ~2e-13 for gaps above 1e-3
    assert np.max(np.abs(ang[:, 1:])) < 2e-6


def test_long_double_run_agrees_with_double():
    A = _rng(14).normal(size=(5000, 6))
    l1, D1, a1, k1 = oracle.eig3(A, precision="f64")
    l2, D2, a2, k2 = oracle.eig3(A, precision="ld")
    assert np.all(k1 == k2)
    assert np.max(np.abs(l1 - l2) / _fro(A)[:, None]) < 1e-14
    assert np.quantile(np.abs(D1 - D2).max((1, 2)), 0.99) < 1e-10


def test_nonfinite_input_gives_nan_and_flag():
    A = np.array([[1, 2, 3, np.nan, 0, 0], [np.inf, 1, 1, 0, 0, 0]], dtype=float)
    lam, D, ang, kase = oracle.eig3(A)
    assert np.all(kase == -1) and np.all(np.isnan(lam)) and np.all(np.isnan(D))


# ------------------------------------------------------------------------------------------ #
# Hand-worked fixtures
# ------------------------------------------------------------------------------------------ #

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden()["eig3"], ids=lambda c: c["name"])
def test_golden_eig3(case):
    lam, D, ang, kase = oracle.eig3(np.array([case["A"]], dtype=float))
    assert kase[0] == case["kase"]
    np.testing.assert_allclose(lam[0], case["lam"], atol=1e-13)
    np.testing.assert_allclose(ang[0], case["ang"], atol=max(case["ang_tol"], 1e-15))
    np.testing.assert_allclose(D[0], np.array(case["D"], dtype=float), atol=max(case["ang_tol"], 1e-15))


@pytest.mark.parametrize("case", _golden()["eig3_spectrum_only"], ids=lambda c: c["name"])
def test_golden_eig3_spectrum(case):
    lam, D, ang, kase = oracle.eig3(np.array([case["A"]], dtype=float))
    assert kase[0] == case["kase"]
    np.testing.assert_allclose(lam[0], case["lam"], atol=1e-13)
    if "D_col3_abs" in case:
        np.testing.assert_allclose(np.abs(D[0][:, 2]), case["D_col3_abs"], atol=1e-7)
    if "D_abs" in case:
        np.testing.assert_allclose(np.abs(D[0]), np.array(case["D_abs"]), atol=1e-7)
    rec = D[0] @ np.diag(lam[0]) @ D[0].T
    np.testing.assert_allclose(rec, oracle.unpack3(np.array([case["A"]], dtype=float))[0], atol=1e-12)


@pytest.mark.parametrize("case", _golden()["eig2"], ids=lambda c: c["name"])
def test_golden_eig2(case):
    lam, phi = oracle.eig2(np.array([case["A"]], dtype=float))
    np.testing.assert_allclose(lam[0], case["lam"], atol=1e-14)
    assert abs(phi[0] - case["phi"]) < 1e-15


# ------------------------------------------------------------------------------------------ #
# 2x2 (Section 3)
# ------------------------------------------------------------------------------------------ #

def test_eig2_recovers_known_angle_and_sign_convention():
    rng = _rng(15)
    n = 20000
    phi = rng.uniform(-math.pi / 4, math.pi / 4, n)
    l = rng.normal(size=(n, 2))                     # either order: the sign rule follows A11-A22
    c, s = np.cos(phi), np.sin(phi)
    A = np.stack([l[:, 0] * c * c + l[:, 1] * s * s, l[:, 0] * s * s + l[:, 1] * c * c,
                  (l[:, 0] - l[:, 1]) * c * s], 1)
    lam, ph = oracle.eig2(A)
    assert np.max(np.abs(lam - l)) < 1e-14 * 10
    gap = np.abs(l[:, 0] - l[:, 1])
    good = gap > 1e-3
    assert np.max(np.abs(ph - phi)[good]) < 1e-12 / 1e-3


def test_eig2_char_equation_and_reconstruction():
    """The eigenvalues solve lam^2 - lam (A11 + A22) + A11 A22 - A12^2 = 0 (the characteristic
    equation of Section 3 with the printed A12 in the linear term read as A22), and
    R(phi) diag(lam) R(phi)^T reproduces A (Eq. (3.4))."""
    A = _rng(16).normal(size=(20000, 3))
    lam, phi = oracle.eig2(A)
    for k in range(2):
        resid = lam[:, k] ** 2 - lam[:, k] * (A[:, 0] + A[:, 1]) + A[:, 0] * A[:, 1] - A[:, 2] ** 2
        assert np.max(np.abs(resid) / (1 + np.sum(A ** 2, 1))) < 1e-14
    c, s = np.cos(phi), np.sin(phi)
    rec = np.stack([lam[:, 0] * c * c + lam[:, 1] * s * s, lam[:, 0] * s * s + lam[:, 1] * c * c,
                    (lam[:, 0] - lam[:, 1]) * c * s], 1)
    assert np.max(np.abs(rec - A)) < 1e-13
    ref = np.linalg.eigvalsh(np.stack([A[:, 0], A[:, 2], A[:, 2], A[:, 1]], 1).reshape(-1, 2, 2))
    assert np.max(np.abs(np.sort(lam, 1) - ref)) < 1e-14 * 10


def test_eig2_swap_symmetry():
    """Section 3: swapping A11 and A22 swaps lam1 and lam2 and changes the sign of phi."""
    A = _rng(17).normal(size=(20000, 3))
    l1, p1 = oracle.eig2(A)
    l2, p2 = oracle.eig2(A[:, [1, 0, 2]])
    assert np.max(np.abs(l1[:, ::-1] - l2)) < 1e-14
    assert np.max(np.abs(p1 + p2)) == 0.0


# ------------------------------------------------------------------------------------------ #
# Adjoints against central finite differences (double precision)
# ------------------------------------------------------------------------------------------ #

def _fd3(A, lb, Db, h=1e-6):
    fd = np.zeros_like(A)
    for j in range(6):
        E = np.zeros(6)
        E[j] = h
        lp, Dp, _, _ = oracle.eig3(A + E)
        lm, Dm, _, _ = oracle.eig3(A - E)
        fd[:, j] = (np.sum(lb * (lp - lm), 1) + np.sum(Db * (Dp - Dm), (1, 2))) / (2 * h)
    return fd


def test_eig3_adjoint_matches_finite_differences():
    rng = _rng(18)
    A = rng.normal(size=(2000, 6))
    lam, _, _, _ = oracle.eig3(A)
    gaps = np.min(np.abs(lam[:, [0, 0, 1]] - lam[:, [1, 2, 2]]), 1)
    A = A[gaps > 0.05]
    lb = rng.normal(size=(A.shape[0], 3))
    Db = rng.normal(size=(A.shape[0], 3, 3))
    g = oracle.eig3_adjoint(A, lb, Db)
    fd = _fd3(A, lb, Db)
    rel = np.abs(fd - g).max(1) / np.abs(g).max(1)
    assert np.median(rel) < 1e-8
    assert np.quantile(rel, 0.999) < 1e-5


def test_eig3_angle_adjoint_matches_finite_differences():
    """The Euler-angle cotangents (through the body angular velocity of D = R1 R2 R3) against
    central differences of the oracle's angles, away from gimbal lock and from the angle ranges'
    edges (where the representation jumps)."""
    rng = _rng(22)
    A = rng.normal(size=(3000, 6))
    lam, _, ang, _ = oracle.eig3(A)
    gaps = np.min(np.abs(lam[:, [0, 0, 1]] - lam[:, [1, 2, 2]]), 1)
    edge = 0.05
    keep = ((gaps > 0.05) & (np.abs(ang[:, 1]) < np.pi / 2 - 0.2) & (np.abs(ang[:, 0]) < np.pi / 2 - edge)
            & (np.abs(ang[:, 2]) < np.pi / 2 - edge))
    A = A[keep]
    ab = rng.normal(size=(A.shape[0], 3))
    zl, zD = np.zeros((A.shape[0], 3)), np.zeros((A.shape[0], 3, 3))
    g = oracle.eig3_adjoint(A, zl, zD, ang_bar=ab)
    h = 1e-6
    fd = np.zeros_like(A)
    for j in range(6):
        E = np.zeros(6)
        E[j] = h
        _, _, ap, _ = oracle.eig3(A + E)
        _, _, am, _ = oracle.eig3(A - E)
        fd[:, j] = np.sum(ab * (ap - am), 1) / (2 * h)
    rel = np.abs(fd - g).max(1) / np.abs(g).max(1)
    assert np.median(rel) < 1e-7
    assert np.quantile(rel, 0.99) < 1e-4


def test_eig3_adjoint_eigenvalue_part_is_sum_of_projectors():
    """With D_bar = 0 the gradient is sum_k lam_bar_k v_k v_k^T (first-order perturbation)."""
    rng = _rng(19)
    A = rng.normal(size=(2000, 6))
    lb = rng.normal(size=(2000, 3))
    lj, V, _ = oracle.jacobi3(A)
    lam, D, _, _ = oracle.eig3(A)
    g = oracle.eig3_adjoint(A, lb, np.zeros((2000, 3, 3)))
    G = np.einsum("nik,nk,njk->nij", D, lb, D)
    packed = np.stack([G[:, 0, 0], G[:, 1, 1], G[:, 2, 2], 2 * G[:, 0, 1], 2 * G[:, 0, 2], 2 * G[:, 1, 2]], 1)
    assert np.max(np.abs(packed - g)) < 1e-12
    # the same projectors from the Jacobi eigenvectors, matched by eigenvalue
    order = np.argsort(-lam, 1)
    lb_sorted = np.take_along_axis(lb, order, 1)
    Gj = np.einsum("nik,nk,njk->nij", V, lb_sorted, V)
    pj = np.stack([Gj[:, 0, 0], Gj[:, 1, 1], Gj[:, 2, 2], 2 * Gj[:, 0, 1], 2 * Gj[:, 0, 2], 2 * Gj[:, 1, 2]], 1)
    assert np.quantile(np.abs(pj - g).max(1), 0.99) < 1e-9


def test_eig2_adjoint_matches_finite_differences():
    rng = _rng(20)
    A = rng.normal(size=(3000, 3))
    lb = rng.normal(size=(3000, 2))
    pb = rng.normal(size=3000)
    lam, _ = oracle.eig2(A)
    A, lb, pb = A[np.abs(lam[:, 0] - lam[:, 1]) > 0.05], lb[np.abs(lam[:, 0] - lam[:, 1]) > 0.05], pb[np.abs(lam[:, 0] - lam[:, 1]) > 0.05]
    g = oracle.eig2_adjoint(A, lb, pb)
    h = 1e-6
    fd = np.zeros_like(A)
    for j in range(3):
        E = np.zeros(3)
        E[j] = h
        lp, pp = oracle.eig2(A + E)
        lm, pm = oracle.eig2(A - E)
        fd[:, j] = (np.sum(lb * (lp - lm), 1) + pb * (pp - pm)) / (2 * h)
    rel = np.abs(fd - g).max(1) / np.abs(g).max(1)
    assert np.quantile(rel, 0.999) < 1e-6


def test_st_loss_gradient_matches_finite_differences():
    rng = _rng(21)
    A = rng.normal(size=(1500, 6))
    lam, _, _, _ = oracle.eig3(A)
    gaps = np.min(np.abs(lam[:, [0, 0, 1]] - lam[:, [1, 2, 2]]), 1)
    A = A[gaps > 0.05]
    w = np.ones(3) / math.sqrt(3)
    terms, g = oracle.st_loss(A, w)
    h = 1e-6
    fd = np.zeros_like(A)
    for j in range(6):
        E = np.zeros(6)
        E[j] = h
        tp = oracle.st_loss(A + E, w, grad=False).sum(1)
        tm = oracle.st_loss(A - E, w, grad=False).sum(1)
        fd[:, j] = (tp - tm) / (2 * h)
    rel = np.abs(fd - g).max(1) / np.abs(g).max(1)
    assert np.quantile(rel, 0.999) < 1e-5
    # the anisotropy term against LAPACK eigenvalues
    ev = np.linalg.eigvalsh(oracle.unpack3(A))
    assert np.max(np.abs(terms[:, 0] - (ev[:, 2] - ev[:, 0]) ** 2)) < 1e-12
