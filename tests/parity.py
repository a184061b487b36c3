"""Comparison helpers for the GPU-vs-oracle parity tests (numpy, float64).

Definitions used by the tolerances (all relative to ||A||_F of each matrix):
  * eigenvalue error   max_k |lam_k - lam_k^ref|, eigenvalues compared as sorted sets;
  * eigenvector error  for each column k of D, matched to the reference eigenvalue closest to
                       lam_k: min(|v - v_ref|, |v + v_ref|) * gap_k / ||A||_F, gap_k the distance
                       of lam_k^ref to the other reference eigenvalues (first-order perturbation:
                       a backward error e moves v_k by at most e / gap_k);
  * reconstruction     |D diag(lam) D^T - A|_F / |A|_F.
"""
import numpy as np

import oracle


def planes_to_rows(P):
    """(k, n) torch/numpy planes -> (n, k) float64 numpy rows."""
    if hasattr(P, "detach"):
        P = P.detach().double().cpu().numpy()
    return np.ascontiguousarray(np.asarray(P, dtype=np.float64).T)


def D_rows(Dp):
    """(9, n) planes -> (n, 3, 3)."""
    return planes_to_rows(Dp).reshape(-1, 3, 3)


def fro3(A):
    return np.linalg.norm(oracle.unpack3(A), axis=(1, 2))


def definition_errors(A, lam, D, ref=None):
    """Errors of a decomposition (lam (n,3), D (n,3,3)) of packed A (n,6) against the Jacobi
    definition oracle. Returns dict of per-matrix arrays."""
    lj, V, _ = ref if ref is not None else oracle.jacobi3(A)
    M = oracle.unpack3(A)
    fro = np.linalg.norm(M, axis=(1, 2))
    fro_safe = np.where(fro > 0, fro, 1.0)
    n = A.shape[0]
    lam_err = np.abs(np.sort(lam, 1)[:, ::-1] - lj).max(1) / fro_safe
    ev_err = np.zeros(n)
    idx_all = np.arange(n)
    for k in range(3):
        idx = np.argmin(np.abs(lj - lam[:, k:k + 1]), 1)
        vref = V[idx_all, :, idx]
        lref = lj[idx_all, idx]
        others = np.abs(lj - lref[:, None])
        others[idx_all, idx] = np.inf
        gap = others.min(1)
        err = np.minimum(np.linalg.norm(D[:, :, k] - vref, axis=1), np.linalg.norm(D[:, :, k] + vref, axis=1))
        ev_err = np.maximum(ev_err, np.minimum(err, 2.0) * gap / fro_safe)
    rec = np.einsum("nij,nj,nkj->nik", D, lam, D)
    rec_err = np.linalg.norm(rec - M, axis=(1, 2)) / fro_safe
    orth = np.abs(np.einsum("nji,njk->nik", D, D) - np.eye(3)).max((1, 2))
    det = np.linalg.det(D)
    return {"lam": lam_err, "ev": ev_err, "rec": rec_err, "orth": orth, "det": det}


def summary(errs):
    return {k: float(np.max(np.abs(v - (1 if k == "det" else 0)))) for k, v in errs.items()}


def euler_D(ang):
    """R1(phi1) R2(phi2) R3(phi3) for (n, 3) angles, written out from the rotation matrices."""
    c1, s1 = np.cos(ang[:, 0]), np.sin(ang[:, 0])
    c2, s2 = np.cos(ang[:, 1]), np.sin(ang[:, 1])
    c3, s3 = np.cos(ang[:, 2]), np.sin(ang[:, 2])
    z, o = np.zeros_like(c1), np.ones_like(c1)
    R1 = np.stack([o, z, z, z, c1, -s1, z, s1, c1], 1).reshape(-1, 3, 3)
    R2 = np.stack([c2, z, s2, z, o, z, -s2, z, c2], 1).reshape(-1, 3, 3)
    R3 = np.stack([c3, -s3, z, s3, c3, z, z, z, o], 1).reshape(-1, 3, 3)
    return R1 @ R2 @ R3


def wrap_pi(x):
    """Angle difference wrapped to (-pi, pi]."""
    return np.angle(np.exp(1j * x))
