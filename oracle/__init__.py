"""CPU oracle for Kronenburg's closed-form diagonalization of 2x2 / 3x3 real symmetric matrices.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package. The GPU library never loads it and shares no code with it.

The oracle itself is plain C (``kd_oracle.c`` + ``method_body.h``) built with gcc into
``oracle/_build/libkd_oracle.so`` on first use (or by ``__graft_entry__.build()``). This module
only marshals numpy arrays into it. Layouts are array-of-structures float64:

* 3x3 input ``(n, 6)`` = (A11, A22, A33, A12, A13, A23); 2x2 input ``(n, 3)`` = (A11, A22, A12)
* ``lam`` ``(n, 3)`` in the paper's labels (lam1 >= lam3 >= lam2; two-equal case lam1 = lam2)
* ``D`` ``(n, 3, 3)``, column k the eigenvector of ``lam[:, k]``; ``ang`` ``(n, 3)`` = (phi1, phi2, phi3)

Functions follow the paper: Section 3 (2x2), Section 4 (3x3 eigenvalues), Section 5 (angles),
Section 6 (Euler angles). ``jacobi3`` is the definition oracle (Eq. (2.1) by cyclic Jacobi).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "kd_oracle.c"), os.path.join(_HERE, "method_body.h")]
_SO = os.path.join(_HERE, "_build", "libkd_oracle.so")

# Numerical readings of the paper's exact tests (q^2 = 4p^3, p = 0) for the double-precision
# method oracle. Near a double root the arccos of Eq. (4.9) gives the pair's split g (relative to
# the spread) with a relative error ~eps/g^2, which Eqs. (5.1)-(5.2) pass on to v and w; the
# equal-pair formulas (5.21)-(5.25) instead make a model error ~g. The two cross over at
# g = eps^(1/3) ~ 6e-6 for eps = 2^-52, so two eigenvalues count as equal when their difference is
# <= TAU2 * spread; all three are equal when the spread is <= TAU3 * ||A||_F.
TAU2 = 5e-6
TAU3 = 1e-12

# Default adjoint gap mask, relative to ||A||_F.
GAP_MASK = 1e-12

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent). Returns the path of the shared library."""
    newest = max(os.path.getmtime(s) for s in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_SO))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
    P = ctypes.c_void_p
    lib.kdo_eig3_f64.argtypes = [i64, P, d, d, P, P, P, P]
    lib.kdo_eig3_ld.argtypes = [i64, P, d, d, P, P, P, P]
    lib.kdo_eig2_f64.argtypes = [i64, P, P, P]
    lib.kdo_jacobi3_ld.argtypes = [i64, P, P, P, P]
    lib.kdo_eig3_adjoint_f64.argtypes = [i64, P, P, P, P, d, d, d, P]
    lib.kdo_eig2_adjoint_f64.argtypes = [i64, P, P, P, d, P]
    lib.kdo_st_loss_f64.argtypes = [i64, P, P, d, d, d, P, P]
    lib.kdo_set_threads.argtypes = [ctypes.c_int]
    lib.kdo_get_threads.restype = ctypes.c_int
    for f in ("kdo_eig3_f64", "kdo_eig3_ld", "kdo_eig2_f64", "kdo_jacobi3_ld", "kdo_eig3_adjoint_f64",
              "kdo_eig2_adjoint_f64", "kdo_st_loss_f64", "kdo_set_threads"):
        getattr(lib, f).restype = None
    _lib = lib
    return lib


def _arr(x, cols):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if x.ndim == 1:
        x = x.reshape(1, -1)
    if x.shape[1] != cols:
        raise ValueError(f"expected (n, {cols}) array, got {x.shape}")
    return x


def _p(x):
    return None if x is None else x.ctypes.data


def set_threads(n: int) -> None:
    _load().kdo_set_threads(int(n))


def get_threads() -> int:
    return int(_load().kdo_get_threads())


def eig3(A, tau2: float = TAU2, tau3: float = TAU3, precision: str = "f64"):
    """Method oracle for packed 3x3 inputs (n, 6). Returns lam (n,3), D (n,3,3), ang (n,3),
    kase (n,) with 0 general, 1 two equal eigenvalues, 2 three equal, -1 non-finite input."""
    A = _arr(A, 6)
    n = A.shape[0]
    lam = np.empty((n, 3))
    D = np.empty((n, 3, 3))
    ang = np.empty((n, 3))
    kase = np.empty(n, dtype=np.int32)
    fn = {"f64": _load().kdo_eig3_f64, "ld": _load().kdo_eig3_ld}[precision]
    fn(n, _p(A), tau2, tau3, _p(lam), _p(D), _p(ang), _p(kase))
    return lam, D, ang, kase


def eig2(A):
    """Method oracle for packed 2x2 inputs (n, 3). Returns lam (n, 2), phi (n,)."""
    A = _arr(A, 3)
    n = A.shape[0]
    lam = np.empty((n, 2))
    phi = np.empty(n)
    _load().kdo_eig2_f64(n, _p(A), _p(lam), _p(phi))
    return lam, phi


def jacobi3(A):
    """Definition oracle: eigenvalues descending (n, 3), eigenvectors as columns (n, 3, 3) and
    the sweep count, by cyclic Jacobi in long double."""
    A = _arr(A, 6)
    n = A.shape[0]
    lam = np.empty((n, 3))
    V = np.empty((n, 3, 3))
    sw = np.empty(n, dtype=np.int32)
    _load().kdo_jacobi3_ld(n, _p(A), _p(lam), _p(V), _p(sw))
    return lam, V, sw


def eig3_adjoint(A, lam_bar, D_bar, ang_bar=None, gap_mask: float = GAP_MASK, tau2: float = TAU2,
                 tau3: float = TAU3):
    """Packed gradient (n, 6) of L(lam, D, angles) through the method oracle, given cotangents
    lam_bar (n, 3), D_bar (n, 3, 3) and optionally ang_bar (n, 3), in the paper's labels."""
    A = _arr(A, 6)
    n = A.shape[0]
    lb = np.ascontiguousarray(np.asarray(lam_bar, dtype=np.float64).reshape(n, 3))
    Db = np.ascontiguousarray(np.asarray(D_bar, dtype=np.float64).reshape(n, 9))
    ab = None if ang_bar is None else np.ascontiguousarray(np.asarray(ang_bar, dtype=np.float64).reshape(n, 3))
    out = np.empty((n, 6))
    _load().kdo_eig3_adjoint_f64(n, _p(A), _p(lb), _p(Db), _p(ab), gap_mask, tau2, tau3, _p(out))
    return out


def eig2_adjoint(A, lam_bar, phi_bar=None, gap_mask: float = GAP_MASK):
    """Packed gradient (n, 3) of L(lam1, lam2, phi) through the 2x2 formulas of Section 3."""
    A = _arr(A, 3)
    n = A.shape[0]
    lb = np.ascontiguousarray(np.asarray(lam_bar, dtype=np.float64).reshape(n, 2))
    pb = None if phi_bar is None else np.ascontiguousarray(np.asarray(phi_bar, dtype=np.float64).reshape(n))
    out = np.empty((n, 3))
    _load().kdo_eig2_adjoint_f64(n, _p(A), _p(lb), _p(pb), gap_mask, _p(out))
    return out


def st_loss(A, w, gap_mask: float = GAP_MASK, tau2: float = TAU2, tau3: float = TAU3, grad: bool = True):
    """Structure-tensor loss per matrix: terms (n, 2) = ((lam_max - lam_min)^2, (v_max . w)^2)
    and, if grad, the packed gradient (n, 6) of their sum."""
    A = _arr(A, 6)
    n = A.shape[0]
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(3))
    terms = np.empty((n, 2))
    a_bar = np.empty((n, 6)) if grad else None
    _load().kdo_st_loss_f64(n, _p(A), _p(w), gap_mask, tau2, tau3, _p(terms), _p(a_bar))
    return (terms, a_bar) if grad else terms


def unpack3(A):
    """(n, 6) packed -> (n, 3, 3) full symmetric matrices (no arithmetic beyond copying)."""
    A = _arr(A, 6)
    M = np.empty((A.shape[0], 3, 3))
    M[:, 0, 0], M[:, 1, 1], M[:, 2, 2] = A[:, 0], A[:, 1], A[:, 2]
    M[:, 0, 1] = M[:, 1, 0] = A[:, 3]
    M[:, 0, 2] = M[:, 2, 0] = A[:, 4]
    M[:, 1, 2] = M[:, 2, 1] = A[:, 5]
    return M
