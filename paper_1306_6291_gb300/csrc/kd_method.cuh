// Device implementation of Kronenburg's closed-form diagonalization (arXiv:1306.6291) for the
// CUDA path: one thread per matrix, everything in registers.
//
// Equation numbers are the paper's: Eqs. (2.6)-(2.9) D = R1 R2 R3; Section 3 (2x2); Eqs.
// (4.5)-(4.12) the cubic's trigonometric roots; Eqs. (5.1)-(5.15) the angles; Eqs. (5.20)-(5.25)
// the two-equal special case; Eq. (6.5) the Euler angles.
//
// Restatements made for the GPU (the mathematics is the paper's):
//  * p and q of Eqs. (4.5)-(4.6) depend only on eigenvalue differences, so they are formed from
//    the trace-free part B = A - (tr A / 3) I, whose diagonal is built from the exact differences
//    A11-A22, A11-A33, A22-A33: p' = p/9 = tr(B^2)/6 (the paper's expanded p, a sum of squares)
//    and q' = q/54 = det(B)/2.
//  * Delta = arccos(q / 2 sqrt(p^3)) (Eq. (4.9)) is evaluated as atan2(sqrt(p'^3 - q'^2), q'),
//    the same angle without arccos's loss of accuracy near +-1; the three cosines of
//    Eqs. (4.10)-(4.12) come from one sincos of Delta/3 and the angle-addition formula.
//  * The sign search of Eqs. (5.13)-(5.15) is done without trigonometry: writing 2-vectors as
//    complex numbers, u1 = g1 conj(f1) has argument phi1(1) and u2 = g2 conj(f2) has argument
//    2 phi1(2). The sign pairs (s2, s3) and (-s2, -s3) differ only by phi1(1) -> phi1(1) + pi, so
//    the pair class is the one maximising Re(u1^2 conj(u2)) (best agreement of phi1(1) and
//    phi1(2) modulo pi; the two classes' scores differ by -2 Im(g1^2 conj g2) Im(conj(f1)^2 f2)) and the member is the one with Re(u1 conj(sqrt(u2))) >= 0 (agreement
//    modulo 2 pi, sqrt the principal root). Ties go to the first pair of the order
//    (+,+), (+,-), (-,+), (-,-). cos and sin of phi1 are the normalised u1 (|f1| >= |f2|) or
//    sqrt(u2) (otherwise); cos and sin of phi2, phi3 are sqrt(v), sqrt(1-v), sqrt(w), sqrt(1-w).
//  * Every matrix is first scaled by an exact power of two so its largest entry is in [1, 2);
//    eigenvalues are scaled back, D and the angles are scale-free.
//  * Precision form (MIXED): B = D^T A D is formed; unless it is already diagonal to conv_kappa,
//    D gets a first-order correction (all coefficients <= 3e-4) or cyclic Jacobi sweeps. The
//    eigenvalues are the diagonal of B (Rayleigh quotients) and the angles are read back from
//    the refined D.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kd {

// --------------------------------------------------------------------------------------------
// precision-generic helpers
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ float k_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double k_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float k_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double k_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float k_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double k_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float k_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double k_abs(double x) { return fabs(x); }
__device__ __forceinline__ float k_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double k_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float k_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double k_min(double a, double b) { return fmin(a, b); }
// quotient used for initial estimates that the refinement corrects (fast in FP32)
__device__ __forceinline__ float k_qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double k_qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float k_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double k_rcp(double x) { return 1.0 / x; }

template <bool FAST>
__device__ __forceinline__ void k_sincos(float x, float *s, float *c) {
    if (FAST) __sincosf(x, s, c); else sincosf(x, s, c);
}
template <bool FAST>
__device__ __forceinline__ void k_sincos(double x, double *s, double *c) { sincos(x, s, c); }

// Square root. FAST (FP32 precision form): the PTX approximate square root (relative error
// ~2^-23), used where the refinement corrects the result or only a threshold depends on it.
template <bool FAST> __device__ __forceinline__ float k_sqrtT(float x) {
    if constexpr (FAST) {
        float r;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return sqrtf(x);
    }
}
template <bool FAST> __device__ __forceinline__ double k_sqrtT(double x) { return sqrt(x); }

// atan(t) for |t| <= 1 (a few ulps beyond are harmless): t P(t^2) with the degree-8 minimax
// polynomial of fit_atan_minimax.py (relative error <= 1.5e-8 on [0, 1]).
// Its coefficients, highest degree first (called with constant i: they become immediates).
__device__ __forceinline__ constexpr float k_atan_coef(int i) {
    constexpr float c[9] = {0.0028498894309480277f, -0.016068628213143348f, 0.04269151809456388f,
                            -0.07504294445536913f, 0.10640933987480042f, -0.1420364446019658f,
                            0.1999261939185979f, -0.33333073345185465f, 0.9999999847657909f};
    return c[i];
}
__device__ __forceinline__ float k_atan_unit(float t) {
    const float q = t * t;
    float p = k_atan_coef(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) p = fmaf(p, q, k_atan_coef(i));
    return t * p;
}

// Angle in [-pi, pi] of the vector (c, s) of length r (= atan2(s, c)). FAST (FP32): by the
// tangent half-angle identity, psi = 2 atan(s / (r + |c|)) is the angle of (|c|, s), in
// [-pi/2, pi/2], and its tangent argument is already in [-1, 1], so the polynomial needs no range
// reduction; for c < 0 the angle is copysign(pi, s) - psi. r must be |(c, s)| up to rounding
// (1 for the unit vectors of a rotation); r + |c| = 0 only for the zero vector, which callers
// exclude. POSC: c >= 0 is known, so there is no reflection. Non-FAST: the library's atan2.
template <bool FAST, bool POSC = false>
__device__ __forceinline__ float k_angle(float s, float c, float r) {
    if constexpr (FAST) {
        const float psi = 2.f * k_atan_unit(__fdividef(s, r + fabsf(c)));
        if constexpr (POSC) return psi;
        return c < 0.f ? copysignf(3.141592653589793f, s) - psi : psi;
    } else {
        return atan2f(s, c);
    }
}
template <bool FAST, bool POSC = false>
__device__ __forceinline__ double k_angle(double s, double c, double) { return atan2(s, c); }

// Precision form: clamp to [0, 1] and take values within 8 ulps of 0 or 1 as 0 or 1 (a rounding
// error e there would become an angle error sqrt(e), ~3e-4 in FP32, for the refinement to remove;
// on the boundary, as for diagonal and block-diagonal inputs, D comes out exact). x is finite
// here: the quotients' denominators are bounded away from 0 by the two-equal test.
template <typename T> __device__ __forceinline__ T snap01(T x) {
    const T tiny = T(8) * T(1.1920928955078125e-07);
    return x < tiny ? T(0) : (x > T(1) - tiny ? T(1) : x);
}

template <typename T> __device__ __forceinline__ T clamp01(T x) {
    // NaN -> 0 (fmax returns the non-NaN operand)
    const T y = k_max(x, T(0));
    return y < T(1) ? y : T(1);
}

template <typename T> struct Lim;
// big(): the largest finite value; norm_floor(): a squared norm at or above it (2^-100 in FP32,
// 2^-900 in FP64) leaves the squares of its components far from underflow.
template <> struct Lim<float> {
    static __device__ __forceinline__ float big() { return 3.4028234e38f; }
    static __device__ __forceinline__ float norm_floor() { return 7.888609052210118e-31f; }
};
template <> struct Lim<double> {
    static __device__ __forceinline__ double big() { return 1.7976931348623157e308; }
    static __device__ __forceinline__ double norm_floor() { return 1.1830521861667747e-271; }
};

// Largest |entry| of the six packed entries; false if any entry is NaN or infinite. For FP32
// the maximum is taken over the bit patterns with the sign cleared (ordered like the values,
// with Inf and NaN above every finite number).
__device__ __forceinline__ bool finite_amax6(float a, float b, float c, float d, float e, float f, float &amax) {
    const int m = max(max(max(__float_as_int(a) & 0x7fffffff, __float_as_int(b) & 0x7fffffff),
                          max(__float_as_int(c) & 0x7fffffff, __float_as_int(d) & 0x7fffffff)),
                      max(__float_as_int(e) & 0x7fffffff, __float_as_int(f) & 0x7fffffff));
    amax = __int_as_float(m);
    return m < 0x7f800000;
}
__device__ __forceinline__ bool finite_amax6(double a, double b, double c, double d, double e, double f,
                                             double &amax) {
    const double BIG = 1.7976931348623157e308;
    if (!(fabs(a) <= BIG && fabs(b) <= BIG && fabs(c) <= BIG && fabs(d) <= BIG && fabs(e) <= BIG &&
          fabs(f) <= BIG))
        return false;
    amax = fmax(fmax(fmax(fabs(a), fabs(b)), fmax(fabs(c), fabs(d))), fmax(fabs(e), fabs(f)));
    return true;
}

// Exact power-of-two scale s with amax * s in [1, 2), and inv = 1/s (both normal numbers): with
// the exponent field clamped to [1, 253], inv is amax with its mantissa cleared and s has the
// exponent field 254 - e.
__device__ __forceinline__ void pow2_scale(float amax, float &s, float &inv) {
    const int eb = min(max(__float_as_int(amax) & 0x7f800000, 0x00800000), 0x7e800000);
    s = __int_as_float(0x7f000000 - eb);
    inv = __int_as_float(eb);
}
__device__ __forceinline__ void pow2_scale(double amax, double &s, double &inv) {
    int e = (__double2hiint(amax) >> 20) & 0x7ff;
    e = min(max(e, 1), 2045);
    s = __hiloint2double((2046 - e) << 20, 0);
    inv = __hiloint2double(e << 20, 0);
}

// --------------------------------------------------------------------------------------------
// Float-float arithmetic (a value is hi + lo, two FP32 numbers, about 48 significant bits) from
// the error-free transformations TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|) and TwoProd
// through a fused multiply-add. The _rn intrinsics keep the compiler from contracting a product
// and a sum into one FMA, which would break the exactness these rely on.
// --------------------------------------------------------------------------------------------
struct ffloat {
    float h, l;
};
__device__ __forceinline__ ffloat ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ffloat ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ffloat ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ffloat ff_neg(ffloat a) { return {-a.h, -a.l}; }
// The operations below leave their result unnormalised (the low part may exceed half an ulp of
// the high part; hi + lo is the value): each is one error-free transformation of the high parts
// plus the low-order terms folded in by FMAs, and ff_norm renormalises where a value feeds a
// squaring or the final difference. Dropped: the product of two low parts (2^-48 relative).
__device__ __forceinline__ ffloat ff_uadd(ffloat a, ffloat b) {
    const ffloat s = ff_two_sum(a.h, b.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ ffloat ff_umul(ffloat a, ffloat b) {
    const ffloat p = ff_two_prod(a.h, b.h);
    return {p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l))};
}
__device__ __forceinline__ ffloat ff_umul_f(ffloat a, float b) {
    const ffloat p = ff_two_prod(a.h, b);
    return {p.h, fmaf(a.l, b, p.l)};
}
__device__ __forceinline__ ffloat ff_usqr(ffloat a) {
    const ffloat p = ff_two_prod(a.h, a.h);
    return {p.h, fmaf(__fadd_rn(a.h, a.h), a.l, p.l)};
}
__device__ __forceinline__ ffloat ff_norm(ffloat a) { return ff_fast_two_sum(a.h, a.l); }

// Invariant modes of the FP32 forms: where p', q' and the discriminant N = p'^3 - q'^2 of
// Eqs. (4.5)-(4.9) are evaluated.
constexpr int INV_F32 = 0, INV_F64 = 1, INV_FF = 2;

// Float-float invariants of the trace-free part B = A - (tr A / 3) I, compensated: with the
// exact-difference matrix 3B (diagonal d1 = e12 + e13, d2 = e23 - e12, d3 = -(e13 + e23), each
// e an exact difference of two diagonal entries held as a TwoSum pair),
//   S9  = 9 tr(B^2)  = d1^2 + d2^2 + d3^2 + 18 (A12^2 + A13^2 + A23^2),
//   Q27 = 27 det(B)  = d1 d2 d3 + 54 A12 A13 A23 - 9 (d1 A23^2 + d2 A13^2 + d3 A12^2),
// so p' = S9 / 54, q' = Q27 / 54 and N = (S9^3 - 54 Q27^2) / 54^3: the high parts' products are
// FMA-exact TwoProds and their sums TwoSums, the low parts are folded in by FMAs (unnormalised
// between steps), and the cancellation S9^3 - 54 Q27^2 (where the spectrum is nearly degenerate)
// is taken in float-float before the one rounding to FP32: X comes out within about 2^-45 of
// S9^3 of its exact value (tests/test_ff_invariants.py replays this arithmetic against exact
// rational arithmetic on rotated spectra with relative gaps down to 1e-7). B is first scaled by an
// exact power of two sc so that its largest entry is in [1, 2) (S9^3 would otherwise leave the
// normal range for nearly equal eigenvalues); p, q, N come back in those units (p' sc^2, q' sc^3,
// N sc^6) with isc = 1/sc.
__device__ __forceinline__ void invariants_ff(float a11, float a22, float a33, float a12, float a13, float a23,
                                              float &p, float &q, float &N, float &isc) {
    ffloat e12 = ff_two_sum(a11, -a22), e13 = ff_two_sum(a11, -a33), e23 = ff_two_sum(a22, -a33);
    float bm = fmaxf(fmaxf(fmaxf(fabsf(e12.h), fabsf(e13.h)), fmaxf(fabsf(e23.h), fabsf(a12))),
                     fmaxf(fabsf(a13), fabsf(a23)));
    float sc;
    pow2_scale(bm, sc, isc);   // B = 0 gives p = q = N = 0 in any units (the three-equal case)
    e12 = {e12.h * sc, e12.l * sc};
    e13 = {e13.h * sc, e13.l * sc};
    e23 = {e23.h * sc, e23.l * sc};
    a12 *= sc; a13 *= sc; a23 *= sc;
    const ffloat d1 = ff_uadd(e12, e13), d2 = ff_uadd(e23, ff_neg(e12)), d3 = ff_neg(ff_uadd(e13, e23));
    const ffloat s12 = ff_two_prod(a12, a12), s13 = ff_two_prod(a13, a13), s23 = ff_two_prod(a23, a23);
    const ffloat o = ff_uadd(ff_uadd(s12, s13), s23);
    const ffloat S9 =
        ff_norm(ff_uadd(ff_uadd(ff_usqr(d1), ff_usqr(d2)), ff_uadd(ff_usqr(d3), ff_umul_f(o, 18.f))));
    const ffloat t1 = ff_umul(ff_umul(d1, d2), d3);
    const ffloat t2 = ff_umul_f(ff_umul_f(ff_two_prod(a12, a13), a23), 54.f);
    const ffloat t3 = ff_uadd(ff_uadd(ff_umul(d1, s23), ff_umul(d2, s13)), ff_umul(d3, s12));
    const ffloat Q27 = ff_norm(ff_uadd(ff_uadd(t1, t2), ff_neg(ff_umul_f(t3, 9.f))));
    const ffloat X = ff_uadd(ff_umul(ff_usqr(S9), S9), ff_neg(ff_umul_f(ff_usqr(Q27), 54.f)));
    p = (S9.h + S9.l) * (1.f / 54.f);
    q = (Q27.h + Q27.l) * (1.f / 54.f);
    N = fmaxf(X.h + X.l, 0.f) * (1.f / 157464.f);
}

// --------------------------------------------------------------------------------------------
// Packed FP32 pairs: on this GPU fma / mul / add on .f32x2 operands perform two FP32 operations
// in one instruction (one issue slot, the FMA pipes doing both lanes), so pairing independent FP32
// products halves their issue cost in these issue-bound kernels. Each lane rounds exactly as the
// scalar instruction would. Broadcasting one FP32 value into both lanes costs nothing measurable;
// pairing two different values may cost a move, so the pairs below are formed where one operand is
// a broadcast or a pair that is reused.
// --------------------------------------------------------------------------------------------
struct fp2 {
    unsigned long long v;
};
__device__ __forceinline__ fp2 fp2_make(float lo, float hi) {
    fp2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ fp2 fp2_bcast(float x) { return fp2_make(x, x); }
__device__ __forceinline__ float fp2_lo(fp2 a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
    return lo;
}
__device__ __forceinline__ float fp2_hi(fp2 a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
    return hi;
}
__device__ __forceinline__ fp2 fp2_fma(fp2 a, fp2 b, fp2 c) {
    fp2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ fp2 fp2_mul(fp2 a, fp2 b) {
    fp2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// B = D^T A D of a symmetric A (a11..a23) and row-major D: the six distinct entries. FP32: the
// first two columns of A D and of B are formed as pairs (rows of D paired by column, entries of A
// broadcast): 18 paired and 12 scalar instructions instead of 45.
template <typename T>
__device__ __forceinline__ void dtad(T a11, T a22, T a33, T a12, T a13, T a23, const T D[9], T &b00, T &b11,
                                     T &b22, T &b01, T &b02, T &b12) {
    if constexpr (sizeof(T) == 4) {
        const fp2 d0 = fp2_make(D[0], D[1]), d1 = fp2_make(D[3], D[4]), d2 = fp2_make(D[6], D[7]);
        // rows of A D: X_r = (AD_r0, AD_r1), Y_r = AD_r2
        const fp2 X0 = fp2_fma(fp2_bcast(a13), d2, fp2_fma(fp2_bcast(a12), d1, fp2_mul(fp2_bcast(a11), d0)));
        const fp2 X1 = fp2_fma(fp2_bcast(a23), d2, fp2_fma(fp2_bcast(a22), d1, fp2_mul(fp2_bcast(a12), d0)));
        const fp2 X2 = fp2_fma(fp2_bcast(a33), d2, fp2_fma(fp2_bcast(a23), d1, fp2_mul(fp2_bcast(a13), d0)));
        const float Y0 = a11 * D[2] + a12 * D[5] + a13 * D[8];
        const float Y1 = a12 * D[2] + a22 * D[5] + a23 * D[8];
        const float Y2 = a13 * D[2] + a23 * D[5] + a33 * D[8];
        // (b00, b01) = sum_r D_r0 X_r, (b02, b12) = sum_r (D_r0, D_r1) Y_r
        const fp2 P0 = fp2_fma(fp2_bcast(D[6]), X2, fp2_fma(fp2_bcast(D[3]), X1, fp2_mul(fp2_bcast(D[0]), X0)));
        const fp2 P2 = fp2_fma(d2, fp2_bcast(Y2), fp2_fma(d1, fp2_bcast(Y1), fp2_mul(d0, fp2_bcast(Y0))));
        b00 = fp2_lo(P0);
        b01 = fp2_hi(P0);
        b02 = fp2_lo(P2);
        b12 = fp2_hi(P2);
        b11 = D[1] * fp2_hi(X0) + D[4] * fp2_hi(X1) + D[7] * fp2_hi(X2);
        b22 = D[2] * Y0 + D[5] * Y1 + D[8] * Y2;
    } else {
        T AD[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            AD[c] = a11 * D[c] + a12 * D[3 + c] + a13 * D[6 + c];
            AD[3 + c] = a12 * D[c] + a22 * D[3 + c] + a23 * D[6 + c];
            AD[6 + c] = a13 * D[c] + a23 * D[3 + c] + a33 * D[6 + c];
        }
        b00 = D[0] * AD[0] + D[3] * AD[3] + D[6] * AD[6];
        b11 = D[1] * AD[1] + D[4] * AD[4] + D[7] * AD[7];
        b22 = D[2] * AD[2] + D[5] * AD[5] + D[8] * AD[8];
        b01 = D[0] * AD[1] + D[3] * AD[4] + D[6] * AD[7];
        b02 = D[0] * AD[2] + D[3] * AD[5] + D[6] * AD[8];
        b12 = D[1] * AD[2] + D[4] * AD[5] + D[7] * AD[8];
    }
}

// Runtime parameters of a call (thresholds already resolved to their defaults).
template <typename T> struct Params {
    T tau2;        // two equal eigenvalues: gap <= tau2 * spread
    T tau3;        // three equal: spread <= tau3 * ||A||_F
    T kappa;       // refinement converged: max |off-diagonal of D^T A D| <= kappa * ||A||_F
    T gap_mask;    // adjoint: |lam_k - lam_j| <= gap_mask * ||A||_F drops the 1/(lam_k - lam_j) term
    int max_sweeps;
};

// Result of one 3x3 decomposition, in scaled units (multiply lam by inv_s to undo the prescale).
template <typename T> struct Eig3 {
    T lam[3];
    T D[9];      // row-major, column k = eigenvector of lam[k]
    T s, inv_s;  // prescale and its inverse
    T fro;       // ||A||_F of the scaled matrix
    int kase;    // 0 general, 1 two equal, 2 three equal, 255 non-finite
    bool unconv; // precision form: the refinement stopped with an off-diagonal of D^T A D still
                 // above conv_kappa ||A||_F (max_sweeps sweeps ran out, or max_sweeps = 0)
};

// The per-matrix code of the kase output: kase, plus 16 when the refinement did not converge.
template <typename T> __device__ __forceinline__ int kase_code(const Eig3<T> &E) {
    return E.kase | (E.unconv ? 16 : 0);
}

// One cyclic-Jacobi rotation in the (i, j) plane of the symmetric B (bii, bjj, bij, and the two
// entries bik, bjk coupling i, j to the third index k), accumulated into the columns i, j of D:
// t = tan(angle) is the root of t^2 + 2 tau t - 1 = 0 of smaller modulus, tau = (bjj-bii)/(2 bij),
// written without the quotient so that bij = 0 gives t = 0. |t| <= 1 since r >= 2 |bij|; the clamp
// keeps it so when d^2 + 4 bij^2 underflows (a pair some 19 orders of magnitude below the scaled
// matrix), where r would come out 0, t would overflow 1 + t^2 and c = s = 0 would wipe two columns.
template <typename T, bool FAST>
__device__ __forceinline__ void jacobi_rot(T &bii, T &bjj, T &bij, T &bik, T &bjk,
                                           T &d0i, T &d1i, T &d2i, T &d0j, T &d1j, T &d2j) {
    T d = bjj - bii;
    T r = k_sqrtT<FAST>(d * d + T(4) * bij * bij);
    T den = k_abs(d) + r;
    T num = (d < T(0)) ? -T(2) * bij : T(2) * bij;
    T t = den > T(0) ? k_min(k_max(k_qdiv(num, den), T(-1)), T(1)) : T(0);
    T c = k_rsqrt(T(1) + t * t);
    T s = t * c;
    bii -= t * bij;
    bjj += t * bij;
    bij = T(0);
    T xik = c * bik - s * bjk, xjk = s * bik + c * bjk;
    bik = xik;
    bjk = xjk;
    T y;
    y = c * d0i - s * d0j; d0j = s * d0i + c * d0j; d0i = y;
    y = c * d1i - s * d1j; d1j = s * d1i + c * d1j; d1i = y;
    y = c * d2i - s * d2j; d2j = s * d2i + c * d2j; d2i = y;
}

// A12 = A13 = 0 (f1 = 0): e1 is an eigenvector and the rest is the 2x2 block (A22, A33, A23), the
// rotation in the e2-e3 plane that the paper discusses under conjecture (2) of Section 5. The
// block is diagonalized by the 2x2 formulas of Section 3 (eigenvalues m +- r/2, eigenvectors
// (0, c, s) and (0, -s, c) at the half angle of (A22 - A33, 2 A23)); the three eigenpairs are then
// labelled as the method labels them (general: max, min, middle; two equal: the pair, larger
// first, then the distinct one; three equal: D = I) and the third column is negated when the
// labelling is an odd permutation, so that det D = +1. Inputs already scaled.
template <typename T, bool FAST>
__device__ __forceinline__ void eig3_block_e1(T a11, T a22, T a33, T a23, const Params<T> &P, Eig3<T> &R) {
    R.fro = k_sqrtT<FAST>(a11 * a11 + a22 * a22 + a33 * a33 + T(2) * a23 * a23);
    // (d, e) = (A22 - A33, 2 A23) is taken times an exact power of two, so that its squares cannot
    // underflow when the block is many orders of magnitude below A11 (the scaled r stays exact).
    const T d = a22 - a33, e = T(2) * a23;
    T sc, isc;
    pow2_scale(k_max(k_abs(d), k_abs(e)), sc, isc);
    const T dn = d * sc, en = e * sc;
    const T rn = k_sqrtT<FAST>(dn * dn + en * en);
    const T r = rn * isc;
    const T m = T(0.5) * (a22 + a33);
    const T mp = m + T(0.5) * r, mm = m - T(0.5) * r;
    T c = T(1), sn = T(0);
    if (rn > T(0)) {
        const T ir = k_rcp(rn);
        const T ct = dn * ir, st = en * ir;      // cos, sin of the double angle
        if (ct >= T(0)) {
            c = k_sqrtT<FAST>(T(0.5) * (T(1) + ct));
            sn = st * T(0.5) * k_rcp(c);
        } else {
            const T as = k_sqrtT<FAST>(T(0.5) * (T(1) - ct));
            sn = st < T(0) ? -as : as;
            c = st * T(0.5) * k_rcp(sn);
        }
    }
    // 0: (a11, e1), 1: (mp, (0, c, sn)), 2: (mm, (0, -sn, c)); mp >= mm
    const int imax = a11 >= mp ? 0 : 1;
    const int imin = a11 < mm ? 0 : 2;
    const int imid = 3 - imax - imin;
    auto pick = [&](int q) { return q == 0 ? a11 : (q == 1 ? mp : mm); };
    const T vmax = pick(imax), vmin = pick(imin), vmid = pick(imid);
    const T spread = vmax - vmin;
    if (!(spread > P.tau3 * R.fro)) {
        const T mean = (a11 + a22 + a33) * (T(1) / T(3));
        R.lam[0] = R.lam[1] = R.lam[2] = mean;
        R.D[0] = T(1); R.D[1] = T(0); R.D[2] = T(0);
        R.D[3] = T(0); R.D[4] = T(1); R.D[5] = T(0);
        R.D[6] = T(0); R.D[7] = T(0); R.D[8] = T(1);
        R.kase = 2;
        return;
    }
    int p0, p1, p2;
    const T g13 = vmax - vmid, g32 = vmid - vmin;
    if (g13 <= P.tau2 * spread || g32 <= P.tau2 * spread) {
        R.kase = 1;
        if (g32 <= g13) { p0 = imid; p1 = imin; p2 = imax; }
        else            { p0 = imax; p1 = imid; p2 = imin; }
    } else {
        R.kase = 0;
        p0 = imax; p1 = imin; p2 = imid;
    }
    const int odd = ((p0 > p1) + (p0 > p2) + (p1 > p2)) & 1;
    const int pk[3] = {p0, p1, p2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = pk[k];
        const T sg = (k == 2 && odd) ? T(-1) : T(1);
        R.lam[k] = pick(q);
        R.D[k] = q == 0 ? sg : T(0);
        R.D[3 + k] = q == 0 ? T(0) : (q == 1 ? sg * c : -sg * sn);
        R.D[6 + k] = q == 0 ? T(0) : (q == 1 ? sg * sn : sg * c);
    }
}

// --------------------------------------------------------------------------------------------
// 3x3: Sections 4-6. T is the arithmetic type. MIXED adds the Jacobi refinement; INV selects where
// p', q' and the discriminant are formed for T = float: INV_F32, INV_F64 (FP64 arithmetic) or
// INV_FF (compensated float-float, invariants_ff).
// --------------------------------------------------------------------------------------------
template <typename T, bool MIXED, int INV, bool FAST_TRIG>
__device__ __forceinline__ void eig3_method(T a11, T a22, T a33, T a12, T a13, T a23,
                                            const Params<T> &P, Eig3<T> &R) {
    const T third = T(1) / T(3);
    R.unconv = false;
    T amax;
    if (!finite_amax6(a11, a22, a33, a12, a13, a23, amax)) {
        const T nan = T(0) / T(0);
        for (int k = 0; k < 3; ++k) R.lam[k] = nan;
        for (int k = 0; k < 9; ++k) R.D[k] = nan;
        R.s = R.inv_s = T(1);
        R.fro = nan;
        R.kase = 255;
        return;
    }
    pow2_scale(amax, R.s, R.inv_s);
    a11 *= R.s; a22 *= R.s; a33 *= R.s; a12 *= R.s; a13 *= R.s; a23 *= R.s;
    if constexpr (MIXED) {
        if (a12 == T(0) && a13 == T(0)) {
            eig3_block_e1<T, FAST_TRIG>(a11, a22, a33, a23, P, R);
            return;
        }
    }

    // Section 4: invariants of the trace-free part (see the header comment).
    const T e12 = a11 - a22, e13 = a11 - a33, e23 = a22 - a33;
    const T m = (a11 + a22 + a33) * third;
    const T o = a12 * a12 + a13 * a13 + a23 * a23;
    T p, q, N, isc = T(1);   // isc: the units of p, q, N are those of B / isc (INV_FF scales B)
    if constexpr (INV == INV_FF && sizeof(T) == 4) {
        invariants_ff(a11, a22, a33, a12, a13, a23, p, q, N, isc);
    } else if constexpr (INV == INV_F64) {
        const double E12 = (double)a11 - (double)a22, E13 = (double)a11 - (double)a33,
                     E23 = (double)a22 - (double)a33;
        const double A12 = a12, A13 = a13, A23 = a23;
        const double b1 = (E12 + E13) * (1.0 / 3), b2 = (E23 - E12) * (1.0 / 3),
                     b3 = -(E13 + E23) * (1.0 / 3);
        const double pd = (E12 * E12 + E13 * E13 + E23 * E23) * (1.0 / 18) +
                          (A12 * A12 + A13 * A13 + A23 * A23) * (1.0 / 3);
        const double qd = 0.5 * (b1 * (b2 * b3 - A23 * A23) + A12 * (2.0 * A13 * A23 - A12 * b3) -
                                 b2 * A13 * A13);
        p = (T)pd;
        q = (T)qd;
        N = (T)fmax(pd * pd * pd - qd * qd, 0.0);
    } else {
        const T b1 = (e12 + e13) * third, b2 = (e23 - e12) * third, b3 = -(e13 + e23) * third;
        p = (e12 * e12 + e13 * e13 + e23 * e23) * (T(1) / T(18)) + o * third;
        q = T(0.5) * (b1 * (b2 * b3 - a23 * a23) + a12 * (T(2) * a13 * a23 - a12 * b3) - b2 * a13 * a13);
        N = k_max(p * p * p - q * q, T(0));
    }
    R.fro = k_sqrtT<FAST_TRIG>(a11 * a11 + a22 * a22 + a33 * a33 + T(2) * o);

    // Eqs. (4.9)-(4.12): Delta = 3 theta; lam1 >= lam3 >= lam2.
    // Delta = atan2(sqrt N, q) = pi/2 - angle of (sqrt N, q), a vector of length p'^(3/2)
    // (N + q'^2 = p'^3). p = 0 (N = q = 0) makes theta NaN and the test below takes the
    // three-equal branch, which does not use theta.
    const T sps = k_sqrtT<FAST_TRIG>(p);
    const T th = (T(1.5707963267948966) - k_angle<FAST_TRIG, true>(q, k_sqrtT<FAST_TRIG>(N), p * sps)) * third;
    const T sp = sps * isc;
    T sn, cs;
    k_sincos<FAST_TRIG>(th, &sn, &cs);
    const T SQ3 = T(1.7320508075688772);
    T l1 = m + T(2) * sp * cs;
    T l2 = m - sp * (cs + SQ3 * sn);
    T l3 = m - sp * (cs - SQ3 * sn);
    const T spread = l1 - l2;

    // Section 5, p = 0: three equal eigenvalues, all angles 0.
    if (!(spread > P.tau3 * R.fro)) {
        R.lam[0] = R.lam[1] = R.lam[2] = m;
        R.D[0] = T(1); R.D[1] = T(0); R.D[2] = T(0);
        R.D[3] = T(0); R.D[4] = T(1); R.D[5] = T(0);
        R.D[6] = T(0); R.D[7] = T(0); R.D[8] = T(1);
        R.kase = 2;
        return;
    }

    T L1, L2, L3, v, w;
    const T g13 = l1 - l3, g32 = l3 - l2;
    if (g13 <= P.tau2 * spread || g32 <= P.tau2 * spread) {
        // q^2 = 4 p^3: relabel lam1 = lam2 = lam (the pair's mean), lam3 the distinct one
        // (Eq. (5.20)); s = cos^2 phi2 (Eq. (5.21)), phi3 = 0 (Eq. (5.23)). With lam1 = lam2 and
        // w = 1 the general g1, g2 below reduce to Eqs. (5.24)-(5.25).
        const bool low = g32 <= g13;
        const T lp = low ? T(0.5) * (l3 + l2) : T(0.5) * (l1 + l3);
        const T ld = low ? l1 : l2;
        L1 = lp; L2 = lp; L3 = ld;
        v = k_qdiv(a11 - ld, lp - ld);
        v = MIXED ? snap01(v) : clamp01(v);
        w = T(1);
        R.kase = 1;
    } else {
        // Eqs. (5.1)-(5.2); v = 0 gives w = 1.
        L1 = l1; L2 = l2; L3 = l3;
        v = k_qdiv(a12 * a12 + a13 * a13 + (a11 - l3) * (a11 + l3 - l1 - l2), (l2 - l3) * (l3 - l1));
        v = MIXED ? snap01(v) : clamp01(v);
        w = v > T(0) ? k_qdiv(a11 - l3 + (l3 - l2) * v, (l1 - l2) * v) : T(1);
        w = MIXED ? snap01(w) : clamp01(w);
        R.kase = 0;
    }
    // Eqs. (5.3)-(5.4): |cos|, |sin| of phi2, phi3 (signs chosen below).
    const T c2 = k_sqrtT<FAST_TRIG>(v), s2 = k_sqrtT<FAST_TRIG>(T(1) - v), c3 = k_sqrtT<FAST_TRIG>(w), s3 = k_sqrtT<FAST_TRIG>(T(1) - w);
    // Eqs. (5.7)-(5.8) for the sign pair (+,+): g1 = (G11, G12), g2 = (G21, G22). The pair
    // (s2, s3) gives g1 = (s3 G11, s2 G12), g2 = (G21, s2 s3 G22).
    const T d12 = L1 - L2, d23 = L2 - L3;
    const T G11 = d12 * c2 * c3 * s3;
    const T G12 = (d12 * w + d23) * c2 * s2;
    const T G21 = d12 * (T(1) + (v - T(2)) * w) + d23 * v;
    const T G22 = T(2) * d12 * s2 * s3 * c3;
    // f1 = (A12, -A13), f2 = (A22 - A33, -2 A23) (Eqs. (5.5)-(5.6)). The plain form scales each by
    // a positive constant (angles are unchanged) so that the products below cannot underflow; in
    // the precision form an underflow only happens when f1 or f2 is negligible, where the paper's
    // conjecture (2) makes every sign pair acceptable and the refinement absorbs the difference.
    const T nf1 = a12 * a12 + a13 * a13, nf2 = e23 * e23 + T(4) * a23 * a23;
    T if1 = T(1), if2 = T(1);
    if constexpr (!MIXED) {
        // without the refinement an underflowed score could pick a wrong sign pair
        const T mf1 = k_max(k_abs(a12), k_abs(a13)), mf2 = k_max(k_abs(e23), k_abs(T(2) * a23));
        if1 = mf1 > T(0) ? k_rcp(mf1) : T(0);
        if2 = mf2 > T(0) ? k_rcp(mf2) : T(0);
    }
    const T f1x = a12 * if1, f1y = -a13 * if1, f2x = e23 * if2, f2y = -T(2) * a23 * if2;
    // Class sigma = s2 s3 (s2 = +1): with u1 = g1 conj(f1) and u2 = g2 conj(f2), the class score
    // is Re(u1^2 conj(u2)). For sigma = -1, g1 -> -conj(g1) and g2 -> conj(g2), so with
    // b = g1^2 conj(g2) and a = conj(f1)^2 f2 the two scores are Re(b a) and Re(conj(b) a), and
    // their difference is -2 Im(b) Im(a): sigma = +1 wins (ties included) when Im(b) Im(a) <= 0.
    const T imb = T(2) * G11 * G12 * G21 - (G11 * G11 - G12 * G12) * G22;
    const T ima = (f1x * f1x - f1y * f1y) * f2y - T(2) * f1x * f1y * f2x;
    const bool plus = imb * ima <= T(0);
    const T G11s = plus ? G11 : -G11, G22s = plus ? G22 : -G22;
    T u1x = G11s * f1x + G12 * f1y, u1y = G12 * f1x - G11s * f1y;
    const T u2x = G21 * f2x + G22s * f2y, u2y = G22s * f2x - G21 * f2y;
    // principal square root of u2 (direction only): argument phi1(2) in (-pi/2, pi/2]
    const T r2 = k_sqrtT<FAST_TRIG>(u2x * u2x + u2y * u2y);
    T hx, hy;
    if (u2x >= T(0)) { hx = r2 + u2x; hy = u2y; }
    else { hx = k_abs(u2y); hy = (u2y < T(0)) ? -(r2 - u2x) : (r2 - u2x); }
    // member of the class: phi1(1) within pi/2 of phi1(2)
    const T sg2 = (u1x * hx + u1y * hy >= T(0)) ? T(1) : T(-1);
    u1x *= sg2; u1y *= sg2;
    const T S2 = sg2 * s2, S3 = (plus ? sg2 : -sg2) * s3;
    // Eq. (5.15): phi1 = phi1(1) if |f1| >= |f2|, else phi1(2)
    T zx = nf1 >= nf2 ? u1x : hx, zy = nf1 >= nf2 ? u1y : hy;
    T c1 = T(1), s1 = T(0);
    const T nz = zx * zx + zy * zy;
    if (nz >= Lim<T>::norm_floor()) {
        // |z|^2 is well inside the normal range: normalise directly
        const T rz = k_rsqrt(nz);
        c1 = zx * rz; s1 = zy * rz;
    } else {
        const T mz = k_max(k_abs(zx), k_abs(zy));
        if (mz > T(0)) {
            // scale first so that the squares cannot underflow
            const T im = k_rcp(mz);
            zx *= im; zy *= im;
            const T rz = k_rsqrt(zx * zx + zy * zy);
            c1 = zx * rz; s1 = zy * rz;
        }
    }
    // Eq. (2.6): D = R1(phi1) R2(phi2) R3(phi3), multiplied out.
    T *D = R.D;
    D[0] = c2 * c3;                 D[1] = -c2 * S3;                D[2] = S2;
    D[3] = c1 * S3 + s1 * S2 * c3;  D[4] = c1 * c3 - s1 * S2 * S3;  D[5] = -s1 * c2;
    D[6] = s1 * S3 - c1 * S2 * c3;  D[7] = s1 * c3 + c1 * S2 * S3;  D[8] = c1 * c2;

    if constexpr (!MIXED) {
        R.lam[0] = L1; R.lam[1] = L2; R.lam[2] = L3;
        return;
    } else {
    // Refinement: B = D^T A D, cyclic Jacobi sweeps, eigenvalues = diag(B).
    T b00, b11, b22, b01, b02, b12;
    dtad(a11, a22, a33, a12, a13, a23, D, b00, b11, b22, b01, b02, b12);
    const T kap = P.kappa * R.fro;
    const bool off_large = k_max(k_abs(b01), k_max(k_abs(b02), k_abs(b12))) > kap;
    R.unconv = off_large && P.max_sweeps == 0;
    if (P.max_sweeps > 0 && off_large) {
        // First-order eigenvector correction v_k += sum_j v_j b_jk / (b_kk - b_jj) when every
        // coefficient is <= 3e-4: the error left (and the loss of orthogonality) is O(e^2) <=
        // 1e-7. A pair with a larger coefficient (two close eigenvalues, the two-equal case, or
        // the sqrt(eps) tail of the angle formulas) is first rotated exactly by one Jacobi
        // rotation, the pair with the largest coefficient; if the other two coefficients are then
        // small the rest is corrected to first order, otherwise cyclic Jacobi sweeps run until the
        // off-diagonal is below conv_kappa.
        const T lim = T(3e-4);
        T e01 = b01 * k_rcp(b11 - b00), e02 = b02 * k_rcp(b22 - b00), e12 = b12 * k_rcp(b22 - b11);
        if (!(k_abs(e01) <= lim && k_abs(e02) <= lim && k_abs(e12) <= lim)) {
            const T x01 = k_abs(e01), x02 = k_abs(e02), x12 = k_abs(e12);
            if (x01 >= x02 && x01 >= x12) {
                jacobi_rot<T, FAST_TRIG>(b00, b11, b01, b02, b12, D[0], D[3], D[6], D[1], D[4], D[7]);
                e01 = T(0);
                e02 = b02 * k_rcp(b22 - b00);
                e12 = b12 * k_rcp(b22 - b11);
            } else if (x02 >= x12) {
                jacobi_rot<T, FAST_TRIG>(b00, b22, b02, b01, b12, D[0], D[3], D[6], D[2], D[5], D[8]);
                e02 = T(0);
                e01 = b01 * k_rcp(b11 - b00);
                e12 = b12 * k_rcp(b22 - b11);
            } else {
                jacobi_rot<T, FAST_TRIG>(b11, b22, b12, b01, b02, D[1], D[4], D[7], D[2], D[5], D[8]);
                e12 = T(0);
                e01 = b01 * k_rcp(b11 - b00);
                e02 = b02 * k_rcp(b22 - b00);
            }
        }
        if (k_abs(e01) <= lim && k_abs(e02) <= lim && k_abs(e12) <= lim) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const T v0 = D[3 * r], v1 = D[3 * r + 1], v2 = D[3 * r + 2];
                D[3 * r] = v0 - e01 * v1 - e02 * v2;
                D[3 * r + 1] = v1 + e01 * v0 - e12 * v2;
                D[3 * r + 2] = v2 + e02 * v0 + e12 * v1;
            }
        } else {
            bool conv = false;
            for (int it = 0; it < P.max_sweeps; ++it) {
                jacobi_rot<T, FAST_TRIG>(b00, b11, b01, b02, b12, D[0], D[3], D[6], D[1], D[4], D[7]);
                jacobi_rot<T, FAST_TRIG>(b00, b22, b02, b01, b12, D[0], D[3], D[6], D[2], D[5], D[8]);
                jacobi_rot<T, FAST_TRIG>(b11, b22, b12, b01, b02, D[1], D[4], D[7], D[2], D[5], D[8]);
                if (k_max(k_abs(b01), k_abs(b02)) <= kap) {   // b12 is 0 after the last rotation
                    conv = true;
                    break;
                }
            }
            R.unconv = !conv;
        }
    }
    R.lam[0] = b00; R.lam[1] = b11; R.lam[2] = b22;
    }
}

// k_atan_unit of two arguments at once, in packed FP32 pairs: each lane is bit for bit the scalar
// polynomial (the same FMAs in the same order); the constants are broadcast immediates.
__device__ __forceinline__ void k_atan_unit_pair(float ta, float tb, float &ra, float &rb) {
    const fp2 t = fp2_make(ta, tb);
    const fp2 q = fp2_mul(t, t);
    fp2 p = fp2_bcast(k_atan_coef(0));
#pragma unroll
    for (int i = 1; i < 9; ++i) p = fp2_fma(p, q, fp2_bcast(k_atan_coef(i)));
    const fp2 r = fp2_mul(t, p);
    ra = fp2_lo(r);
    rb = fp2_hi(r);
}

// Euler angles (Eq. (6.5)) of a rotation D = R1(phi1) R2(phi2) R3(phi3): phi2 = atan2(D13, c2)
// with c2 = |(D23, D33)| >= 0, phi1 = atan2(-D23, D33), and phi3 read from R1(phi1)^T D =
// R2(phi2) R3(phi3), whose second row is (sin phi3, cos phi3, 0). Near cos phi2 = 0 only
// phi1 + -phi3 is determined; this choice keeps R1 R2 R3(angles) = D there too. D must be
// finite (the caller substitutes NaN angles for a non-finite input).
template <typename T, bool FAST>
__device__ __forceinline__ void euler_from_D(const T D[9], T ang[3]) {
    const T c2sq = D[5] * D[5] + D[8] * D[8];
    const T c2 = k_sqrtT<FAST>(c2sq);
    // (x1, y1) = (cos phi1, sin phi1) scaled by r1 = c2. Gimbal lock (phi1 = 0) is taken where
    // c2^2 < norm_floor: cos phi2 < 2^-50 (FP32) makes phi2 = +-pi/2 to the working precision,
    // and below it the squares may have lost digits to underflow, so c2 would not be |(x1, y1)|.
    const bool lock = !(c2sq >= Lim<T>::norm_floor());
    const T x1 = lock ? T(1) : D[8], y1 = lock ? T(0) : -D[5], r1 = lock ? T(1) : c2;
    // (cos phi3, sin phi3) scaled by r1
    const T s3 = x1 * D[3] + y1 * D[6], c3 = x1 * D[4] + y1 * D[7];
    if constexpr (FAST && sizeof(T) == 4) {
        // k_angle of phi1 and phi3 with their two arctan polynomials evaluated as one pair
        float pa, pb;
        k_atan_unit_pair(__fdividef(y1, r1 + fabsf(x1)), __fdividef(s3, r1 + fabsf(c3)), pa, pb);
        const float psi1 = 2.f * pa, psi3 = 2.f * pb;
        ang[0] = x1 < 0.f ? copysignf(3.141592653589793f, y1) - psi1 : psi1;
        ang[2] = c3 < 0.f ? copysignf(3.141592653589793f, s3) - psi3 : psi3;
    } else {
        ang[0] = k_angle<FAST>(y1, x1, r1);
        ang[2] = k_angle<FAST>(s3, c3, r1);
    }
    ang[1] = k_angle<FAST, true>(D[2], c2, T(1));   // (c2, D13) is a unit vector
}

// The adjoint below for FP32 with its products in packed pairs (the same formulas): the needed
// entries of M = D^T D_bar as (M_j0, M_j1) = sum_r D_rj (Db_r0, Db_r1) and (M_02, M_12); the first
// two rows of T = D S as pairs across the rows, (T_0k, T_1k) = sum_j (D_0j, D_1j) S_jk; and
// G = T D^T as (G_0l, G_1l) = sum_k (T_0k, T_1k) D_lk (G is symmetric: G_01 is taken from l = 1).
__device__ __forceinline__ void eig3_adjoint_f32(const Eig3<float> &E, const float lb[3], const float Db[9],
                                                 bool has_ang, const float ab[3], float gap_mask, float out[6]) {
    const float *D = E.D;
    const fp2 b0 = fp2_make(Db[0], Db[1]), b1 = fp2_make(Db[3], Db[4]), b2 = fp2_make(Db[6], Db[7]);
    const fp2 d0 = fp2_make(D[0], D[1]), d1 = fp2_make(D[3], D[4]), d2 = fp2_make(D[6], D[7]);
    const fp2 M0 = fp2_fma(fp2_bcast(D[6]), b2, fp2_fma(fp2_bcast(D[3]), b1, fp2_mul(fp2_bcast(D[0]), b0)));
    const fp2 M1 = fp2_fma(fp2_bcast(D[7]), b2, fp2_fma(fp2_bcast(D[4]), b1, fp2_mul(fp2_bcast(D[1]), b0)));
    const fp2 M2 = fp2_fma(fp2_bcast(D[8]), b2, fp2_fma(fp2_bcast(D[5]), b1, fp2_mul(fp2_bcast(D[2]), b0)));
    const fp2 Mq = fp2_fma(d2, fp2_bcast(Db[8]), fp2_fma(d1, fp2_bcast(Db[5]), fp2_mul(d0, fp2_bcast(Db[2]))));
    const float M01 = fp2_hi(M0);
    float M10 = fp2_lo(M1), M20 = fp2_lo(M2), M21 = fp2_hi(M2), M02 = fp2_lo(Mq);
    const float M12 = fp2_hi(Mq);
    if (has_ang) {
        const float c2sq = D[5] * D[5] + D[8] * D[8];
        const float c2 = k_sqrt(c2sq), s2 = D[2];
        float c1 = 1.f, s1 = 0.f;
        if (c2sq >= Lim<float>::norm_floor()) {   // the gimbal-lock rule of euler_from_D
            const float ic = k_rcp(c2);
            c1 = D[8] * ic;
            s1 = -D[5] * ic;
        }
        const float s3 = c1 * D[3] + s1 * D[6], c3 = c1 * D[4] + s1 * D[7];
        const float rc = (c2 > gap_mask) ? (ab[0] - s2 * ab[2]) * k_rcp(c2) : 0.f;
        M21 += c3 * rc + s3 * ab[1];
        M02 += -s3 * rc + c3 * ab[1];
        M10 += ab[2];
    }
    const float thr = gap_mask * E.fro;
    const float g01 = E.lam[1] - E.lam[0], g02 = E.lam[2] - E.lam[0], g12 = E.lam[2] - E.lam[1];
    const float S01 = (M01 - M10) * ((fabsf(g01) > thr) ? E.s * k_rcp(g01) : 0.f);
    const float S02 = (M02 - M20) * ((fabsf(g02) > thr) ? E.s * k_rcp(g02) : 0.f);
    const float S12 = (M12 - M21) * ((fabsf(g12) > thr) ? E.s * k_rcp(g12) : 0.f);
    const float S00 = 2.f * lb[0], S11 = 2.f * lb[1], S22 = 2.f * lb[2];
    // rows 0 and 1 of T = D S, paired across the rows; row 2 scalar
    const fp2 c0 = fp2_make(D[0], D[3]), c1p = fp2_make(D[1], D[4]), c2p = fp2_make(D[2], D[5]);
    const fp2 T0 = fp2_fma(c2p, fp2_bcast(S02), fp2_fma(c1p, fp2_bcast(S01), fp2_mul(c0, fp2_bcast(S00))));
    const fp2 T1 = fp2_fma(c2p, fp2_bcast(S12), fp2_fma(c1p, fp2_bcast(S11), fp2_mul(c0, fp2_bcast(S01))));
    const fp2 T2 = fp2_fma(c2p, fp2_bcast(S22), fp2_fma(c1p, fp2_bcast(S12), fp2_mul(c0, fp2_bcast(S02))));
    const float R0 = D[6] * S00 + D[7] * S01 + D[8] * S02;
    const float R1 = D[6] * S01 + D[7] * S11 + D[8] * S12;
    const float R2 = D[6] * S02 + D[7] * S12 + D[8] * S22;
    // (G_0l, G_1l) = sum_k (T_0k, T_1k) D_lk
    const fp2 G0 = fp2_fma(T2, fp2_bcast(D[2]), fp2_fma(T1, fp2_bcast(D[1]), fp2_mul(T0, fp2_bcast(D[0]))));
    const fp2 G1 = fp2_fma(T2, fp2_bcast(D[5]), fp2_fma(T1, fp2_bcast(D[4]), fp2_mul(T0, fp2_bcast(D[3]))));
    const fp2 G2 = fp2_fma(T2, fp2_bcast(D[8]), fp2_fma(T1, fp2_bcast(D[7]), fp2_mul(T0, fp2_bcast(D[6]))));
    const float G22 = R0 * D[6] + R1 * D[7] + R2 * D[8];
    out[0] = 0.5f * fp2_lo(G0);
    out[1] = 0.5f * fp2_hi(G1);
    out[2] = 0.5f * G22;
    out[3] = fp2_lo(G1);
    out[4] = fp2_lo(G2);
    out[5] = fp2_hi(G2);
}

// Packed gradient of L(lam, D) (A_bar = D (diag(lam_bar) + F o (D^T D_bar)) D^T, F_jk =
// 1/(lam_k - lam_j)), from a decomposition in scaled units: lam_s = s * lam, so
// 1/(lam_k - lam_j) = s / (lam_s_k - lam_s_j).
//
// Euler-angle cotangents ab (used when has_ang): with D = R1 R2 R3 (Eq. (6.5)), D^T dD = [omega]x,
// omega = M_phi dphi, M_phi = [[c2 c3, s3, 0], [-c2 s3, c3, 0], [s2, 0, 1]], and omega =
// (Omega_21, Omega_02, Omega_10) of Omega_jk = v_j^T dA v_k / (lam_k - lam_j). So
// ab . dphi = mu . omega with M_phi^T mu = ab, and mu joins D^T D_bar at (2,1), (0,2), (1,0).
// The 1/cos(phi2) part is dropped where cos(phi2) <= gap_mask (gimbal lock, where phi1 and phi3
// are not separately differentiable). The cosines and sines are read from D exactly as the
// forward reads the angles (euler_from_D).
template <typename T>
__device__ __forceinline__ void eig3_adjoint(const Eig3<T> &E, const T lb[3], const T Db[9], bool has_ang,
                                             const T ab[3], T gap_mask, T out[6]) {
    if constexpr (sizeof(T) == 4) {
        eig3_adjoint_f32(E, lb, Db, has_ang, ab, gap_mask, out);
        return;
    }
    const T *D = E.D;
    T M[9];  // D^T D_bar
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[3 * j + k] = D[j] * Db[k] + D[3 + j] * Db[3 + k] + D[6 + j] * Db[6 + k];
    if (has_ang) {
        const T c2sq = D[5] * D[5] + D[8] * D[8];
        const T c2 = k_sqrt(c2sq), s2 = D[2];
        T c1 = T(1), s1 = T(0);
        if (c2sq >= Lim<T>::norm_floor()) {   // the gimbal-lock rule of euler_from_D
            const T ic = k_rcp(c2);
            c1 = D[8] * ic;
            s1 = -D[5] * ic;
        }
        const T s3 = c1 * D[3] + s1 * D[6], c3 = c1 * D[4] + s1 * D[7];
        const T rc = (c2 > gap_mask) ? (ab[0] - s2 * ab[2]) * k_rcp(c2) : T(0);
        M[7] += c3 * rc + s3 * ab[1];
        M[2] += -s3 * rc + c3 * ab[1];
        M[3] += ab[2];
    }
    // Only the symmetric part of A_bar enters the packed gradient (A_bar_ij + A_bar_ji), so form
    // S = K + K^T, K = diag(lam_bar) + F o M: S_jj = 2 lam_bar_j, S_jk = (M_jk - M_kj) / (lam_k - lam_j).
    const T thr = gap_mask * E.fro;
    T S[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) S[4 * j] = T(2) * lb[j];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = j + 1; k < 3; ++k) {
            const T gap = E.lam[k] - E.lam[j];
            const T ig = (k_abs(gap) > thr) ? E.s * k_rcp(gap) : T(0);
            S[3 * j + k] = S[3 * k + j] = (M[3 * j + k] - M[3 * k + j]) * ig;
        }
    T Tm[9];  // D S
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) Tm[3 * i + k] = D[3 * i] * S[k] + D[3 * i + 1] * S[3 + k] + D[3 * i + 2] * S[6 + k];
    // G = D S D^T is symmetric: packed diagonal G_ii / 2, packed off-diagonal G_il
    auto G = [&](int i, int l) { return Tm[3 * i] * D[3 * l] + Tm[3 * i + 1] * D[3 * l + 1] + Tm[3 * i + 2] * D[3 * l + 2]; };
    out[0] = T(0.5) * G(0, 0);
    out[1] = T(0.5) * G(1, 1);
    out[2] = T(0.5) * G(2, 2);
    out[3] = G(0, 1);
    out[4] = G(0, 2);
    out[5] = G(1, 2);
}

// --------------------------------------------------------------------------------------------
// 2x2: Section 3.
// --------------------------------------------------------------------------------------------
template <typename T> struct Eig2 {
    T lam[2];
    T phi, c, s;   // phi and cos phi, sin phi
    T s_scale, inv_s, fro;
    bool bad;
};

template <typename T, bool FAST_TRIG>
__device__ __forceinline__ void eig2_method(T a11, T a22, T a12, Eig2<T> &R) {
    const T BIG = Lim<T>::big();
    if (!(k_abs(a11) <= BIG && k_abs(a22) <= BIG && k_abs(a12) <= BIG)) {
        const T nan = T(0) / T(0);
        R.lam[0] = R.lam[1] = R.phi = R.c = R.s = R.fro = nan;
        R.s_scale = R.inv_s = T(1);
        R.bad = true;
        return;
    }
    R.bad = false;
    const T amax = k_max(k_max(k_abs(a11), k_abs(a22)), k_abs(a12));
    pow2_scale(amax, R.s_scale, R.inv_s);
    a11 *= R.s_scale; a22 *= R.s_scale; a12 *= R.s_scale;
    const T d = a11 - a22;
    const T sg = d < T(0) ? T(-1) : T(1);            // sign(0) = +1
    const T ad = k_abs(d), y = T(2) * a12 * sg;
    const T r = k_sqrtT<FAST_TRIG>(d * d + T(4) * a12 * a12);
    R.lam[0] = T(0.5) * (a11 + a22 + sg * r);       // Eq. (3.2)
    R.lam[1] = T(0.5) * (a11 + a22 - sg * r);       // Eq. (3.3)
    // Eq. (3.5): phi = arctan(2 A12 / (A11 - A22)) / 2, the half angle of the vector (|d|, y) of
    // length r, whose tangent is y / (r + |d|) (in [-1, 1]); A11 = A22, A12 = 0 gives phi = 0.
    // At the tie A11 = A22 the tangent is exactly +-1 and phi the rounded +-pi/4, whatever r is:
    // there 4 A12^2 may underflow (A12 below ~1e-19 of the largest entry in FP32, 1e-154 in FP64),
    // so the tie does not go through r. Off the tie, |d| is 0 or at least an ulp of the largest
    // entry (A11 and A22 are both within a factor 2 of it, or d is as large as it), so d^2 does not
    // underflow and r >= |d| is accurate.
    if constexpr (FAST_TRIG) {
        if (ad > T(0) || y != T(0)) {
            const T t = ad > T(0) ? __fdividef(y, r + ad) : copysignf(T(1), y);
            R.phi = ad > T(0) ? k_atan_unit(t) : copysignf(T(0.7853981633974483), y);
            R.c = k_rsqrt(T(1) + t * t);
            R.s = t * R.c;
        } else {
            R.phi = T(0);
            R.c = T(1);
            R.s = T(0);
        }
    } else {
        R.phi = T(0.5) * k_atan2(y, ad);
        // cos 2phi = |d| / r >= 0 and sin 2phi = y / r; half angles without cancellation
        if (ad > T(0)) {
            const T c = k_sqrt(T(0.5) * (T(1) + ad / r));
            R.c = c;
            R.s = y / r * T(0.5) / c;
        } else if (y != T(0)) {
            R.c = k_sqrt(T(0.5));
            R.s = y > T(0) ? R.c : -R.c;
        } else {
            R.c = T(1);
            R.s = T(0);
        }
    }
    R.fro = k_sqrtT<FAST_TRIG>(a11 * a11 + a22 * a22 + T(2) * a12 * a12);
}

}  // namespace kd
