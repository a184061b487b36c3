"""The compensated float-float invariants of the FP32 kernels (KD_INV_FLOAT_FLOAT, csrc/kd_method.cuh
`invariants_ff`), replayed step by step in FP32 on the host (numpy float32 for every rounding, a
fused multiply-add rounded once from the exact product) and compared with exact rational
arithmetic. No GPU: this checks the formulas and their error, not the kernel.

* S9 = 9 tr(B^2) and Q27 = 27 det(B) of B = A - (tr A / 3) I are the right invariants: checked in
  exact arithmetic against tr(B^2) and det(B) formed from B itself.
* The float-float evaluation of X = S9^3 - 54 Q27^2 (27^2 * 4 * 54 times the discriminant p'^3 -
  q'^2) stays within 2^-44 of S9^3 of the exact X on rotated spectra whose relative gaps go down to
  1e-7, where FP32 arithmetic would lose every digit of X.
"""
from fractions import Fraction as F

import numpy as np

f32 = np.float32


def _add(a, b):
    return f32(f32(a) + f32(b))


def _sub(a, b):
    return f32(f32(a) - f32(b))


def _mul(a, b):
    return f32(f32(a) * f32(b))


def _fma(a, b, c):
    return f32(float(F(float(a)) * F(float(b)) + F(float(c))))


def _two_sum(a, b):
    s = _add(a, b)
    bb = _sub(s, a)
    return s, _add(_sub(a, _sub(s, bb)), _sub(b, bb))


def _fast_two_sum(a, b):
    s = _add(a, b)
    return s, _sub(b, _sub(s, a))


def _two_prod(a, b):
    p = _mul(a, b)
    return p, _fma(a, b, -p)


def _uadd(x, y):
    s, e = _two_sum(x[0], y[0])
    return s, _add(e, _add(x[1], y[1]))


def _umul(x, y):
    p, e = _two_prod(x[0], y[0])
    return p, _fma(x[0], y[1], _fma(x[1], y[0], e))


def _umul_f(x, c):
    p, e = _two_prod(x[0], c)
    return p, _fma(x[1], c, e)


def _usqr(x):
    p, e = _two_prod(x[0], x[0])
    return p, _fma(_add(x[0], x[0]), x[1], e)


def _norm(x):
    return _fast_two_sum(x[0], x[1])


def _neg(x):
    return -x[0], -x[1]


def ff_invariants(a11, a22, a33, a12, a13, a23):
    """The kernel's steps: exact differences, power-of-two scale of B, S9, Q27, X (scaled units)."""
    e12, e13, e23 = _two_sum(a11, -a22), _two_sum(a11, -a33), _two_sum(a22, -a33)
    bm = max(abs(float(v)) for v in (e12[0], e13[0], e23[0], a12, a13, a23))
    sc = f32(2.0 ** -np.floor(np.log2(bm))) if bm > 0 else f32(1)
    e12, e13, e23 = [(_mul(e[0], sc), _mul(e[1], sc)) for e in (e12, e13, e23)]
    a12, a13, a23 = _mul(a12, sc), _mul(a13, sc), _mul(a23, sc)
    d1, d2, d3 = _uadd(e12, e13), _uadd(e23, _neg(e12)), _neg(_uadd(e13, e23))
    s12, s13, s23 = _two_prod(a12, a12), _two_prod(a13, a13), _two_prod(a23, a23)
    o = _uadd(_uadd(s12, s13), s23)
    S9 = _norm(_uadd(_uadd(_usqr(d1), _usqr(d2)), _uadd(_usqr(d3), _umul_f(o, f32(18)))))
    t1 = _umul(_umul(d1, d2), d3)
    t2 = _umul_f(_umul_f(_two_prod(a12, a13), a23), f32(54))
    t3 = _uadd(_uadd(_umul(d1, s23), _umul(d2, s13)), _umul(d3, s12))
    Q27 = _norm(_uadd(_uadd(t1, t2), _neg(_umul_f(t3, f32(9)))))
    X = _uadd(_umul(_usqr(S9), S9), _neg(_umul_f(_usqr(Q27), f32(54))))
    return sc, S9, Q27, X


def _exact_s9_q27(a):
    a11, a22, a33, a12, a13, a23 = [F(float(v)) for v in a]
    d1, d2, d3 = 2 * a11 - a22 - a33, 2 * a22 - a11 - a33, 2 * a33 - a11 - a22
    S9 = d1 * d1 + d2 * d2 + d3 * d3 + 18 * (a12 ** 2 + a13 ** 2 + a23 ** 2)
    Q27 = d1 * d2 * d3 + 54 * a12 * a13 * a23 - 9 * (d1 * a23 ** 2 + d2 * a13 ** 2 + d3 * a12 ** 2)
    return S9, Q27


def _rotated(lam, rng):
    q = rng.standard_normal(4)
    w, x, y, z = q / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    M = R @ np.diag(lam) @ R.T
    a = [f32(v) for v in (M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2])]
    m = max(abs(float(v)) for v in a)
    s = f32(2.0 ** -np.floor(np.log2(m)))
    return [_mul(v, s) for v in a]        # the kernels' exact power-of-two prescale


def test_s9_q27_are_nine_tr_b2_and_27_det_b():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = [f32(v) for v in rng.standard_normal(6)]
        a11, a22, a33, a12, a13, a23 = [F(float(v)) for v in a]
        m = (a11 + a22 + a33) / 3
        B = [[a11 - m, a12, a13], [a12, a22 - m, a23], [a13, a23, a33 - m]]
        tr2 = sum(B[i][j] * B[j][i] for i in range(3) for j in range(3))
        det = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0])
               + B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]))
        S9, Q27 = _exact_s9_q27(a)
        assert S9 == 9 * tr2 and Q27 == 27 * det


def test_float_float_discriminant_is_accurate_on_nearly_degenerate_spectra():
    rng = np.random.default_rng(0)
    worst_ff = worst_f32 = 0.0
    for t in range(240):
        lam = rng.standard_normal(3)
        if t % 3 == 1:    # a close pair
            lam[1] = lam[0] * (1 + 10.0 ** rng.uniform(-7, -3))
        elif t % 3 == 2:  # nearly three equal
            lam = lam[0] * (1 + 10.0 ** rng.uniform(-6, -2) * rng.uniform(-1, 1, 3))
        a = _rotated(lam, rng)
        sc, S9, Q27, X = ff_invariants(*a)
        S9e, Q27e = _exact_s9_q27(a)
        Xe = S9e ** 3 - 54 * Q27e ** 2
        sc6 = F(float(sc)) ** 6
        got = (F(float(X[0])) + F(float(X[1]))) / sc6
        worst_ff = max(worst_ff, float(abs(got - Xe) / S9e ** 3))
        # the same difference from FP32 values of S9 and Q27 (what FP32 invariants can resolve)
        s9, q27 = f32(float(S9e * F(float(sc)) ** 2)), f32(float(Q27e * F(float(sc)) ** 3))
        x32 = F(float(_sub(_mul(_mul(s9, s9), s9), _mul(f32(54), _mul(q27, q27))))) / sc6
        worst_f32 = max(worst_f32, float(abs(x32 - Xe) / S9e ** 3))
    print(f"|X - X_exact| / S9^3: float-float {worst_ff:.2e}, FP32 {worst_f32:.2e}")
    assert worst_ff < 2.0 ** -44
    assert worst_f32 > 1e-8      # FP32 alone cannot resolve X on these spectra
