// Structure-tensor loss over a field of 3x3 tensors, forward (two sums) and backward (packed
// gradient per tensor), each tensor decomposed by the FP32 precision form of the method.
//   L = sum (lam_max - lam_min)^2 + sum (v_max . w)^2
// The forward kernel keeps compensated FP32 sums per thread, reduces them per block in FP64 into
// a workspace of per-block partials, and a one-block kernel adds the partials in a fixed order,
// so the result does not depend on scheduling.
//
// Algorithmic operation count per tensor of the fused forward + backward (FP32 and MUFU
// operations, compares and selects the formulas' branches need, one slot each; loads and stores
// one each), by step of the method:
//   load, widen BF16, largest entry, power-of-two scale               25
//   invariants p', q', N and ||A||_F (Eqs. (4.5)-(4.8))               38
//   Delta and the three eigenvalues (Eqs. (4.9)-(4.12))               30
//   three-equal / two-equal tests                                      8
//   v, w with their clamps (Eqs. (5.1)-(5.2))                         28
//   cos/sin of phi2, phi3 (Eqs. (5.3)-(5.4))                           6
//   g1, g2, f1, f2, sign search (Eqs. (5.5)-(5.14))                   64
//   phi1 (Eq. (5.15))                                                  9
//   D = R1 R2 R3 (Eq. (2.6))                                          16
//   D^T A D, test, first-order correction (in every warp)             79
//   ordering, lam_max - lam_min, v_max . w, compensated sums          27
//   gradient (c_j, p, q, six packed entries), scale, BF16, stores     78
//   total                                                            408
// bench.py's algorithmic issue bound uses 410 per tensor.
#include <cuda_bf16.h>

#include "kd_internal.h"

namespace kd {

// Threads per block of the loss kernels: one block of 1024 per SM (up to 64 registers), measured
// 8% faster on the fused kernel than 256-thread blocks.
constexpr int kStThreads = 1024;

__device__ __forceinline__ float ld_f(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_f(const uint16_t *p) {
    return __uint_as_float(((uint32_t)__ldcs((const unsigned short *)p)) << 16);
}
__device__ __forceinline__ void st_f(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st_f(uint16_t *p, float v) {
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    __stcs((unsigned short *)p, *reinterpret_cast<unsigned short *>(&b));
}

// The eigenpairs of one tensor ordered by eigenvalue (largest, middle, smallest) by three
// compare-exchanges of (lam, column of D), strict comparisons so that ties keep the column order:
// selects only, no run-time label indexes an array (which would move it to local memory).
// an = lam_max - lam_min (unscaled) and vw = v_max . w are the roots of the two loss terms.
struct StTerms {
    float l[3];      // scaled eigenvalues: max, mid, min
    float v[3][3];   // v[j][r]: component r of the eigenvector of l[j]
    float an, vw;
};
__device__ __forceinline__ void st_cx(float &la, float va[3], float &lb, float vb[3]) {
    const bool sw = lb > la;
    const float l0 = la, l1 = lb;
    la = sw ? l1 : l0;
    lb = sw ? l0 : l1;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float x = va[r], y = vb[r];
        va[r] = sw ? y : x;
        vb[r] = sw ? x : y;
    }
}
__device__ __forceinline__ StTerms st_terms(const Eig3<float> &E, float w0, float w1, float w2) {
    StTerms t;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        t.l[j] = E.lam[j];
#pragma unroll
        for (int r = 0; r < 3; ++r) t.v[j][r] = E.D[3 * r + j];
    }
    st_cx(t.l[0], t.v[0], t.l[1], t.v[1]);
    st_cx(t.l[0], t.v[0], t.l[2], t.v[2]);
    st_cx(t.l[1], t.v[1], t.l[2], t.v[2]);
    t.an = (t.l[0] - t.l[2]) * E.inv_s;
    t.vw = t.v[0][0] * w0 + t.v[0][1] * w1 + t.v[0][2] * w2;
    return t;
}

// Packed gradient of one tensor's loss terms, written out for this loss (the general 3x3 adjoint
// with lam_bar = +-2 an at the two labels and D_bar = 2 vw w in the column of lam_max reduces to
// it). With v_j the unit eigenvectors, dlam_k = v_k^T dA v_k and, to first order,
// dv_max = sum_{j != max} v_j (v_j^T dA v_max) / (lam_max - lam_j), so with
//   c_j = 2 vw (v_j . w) / (lam_max - lam_j)   (0 where lam_max - lam_j <= gap_mask ||A||_F),
//   u = sum_{j != max} c_j v_j,  alpha = 2 an,  p = alpha v_max + u,  q = alpha v_min,
// the packed gradient is g_aa = v_max,a p_a - v_min,a q_a on the diagonal and
// g_ab = v_max,a p_b + v_max,b p_a - 2 v_min,a q_b off it (the packed entry stands for A_ab and
// A_ba). The 1/(lam_max - lam_j) are taken from the scaled eigenvalues: s / (lam_s_max - lam_s_j);
// the reciprocals are formed unconditionally and the masked terms selected away (no branch).
__device__ __forceinline__ void st_grad(const Eig3<float> &E, const StTerms &L, float w0, float w1, float w2,
                                        const Params<float> &P, float out[6]) {
    const float *vmax = L.v[0], *vmid = L.v[1], *vmin = L.v[2];
    const float gmid = L.l[0] - L.l[1], gmin = L.l[0] - L.l[2];
    const float thr = P.gap_mask * E.fro;
    const float g2s = 2.f * L.vw * E.s;
    const float rmid = __fdividef(1.f, gmid), rmin = __fdividef(1.f, gmin);
    const float tmid = g2s * (vmid[0] * w0 + vmid[1] * w1 + vmid[2] * w2) * rmid;
    const float tmin = g2s * (vmin[0] * w0 + vmin[1] * w1 + vmin[2] * w2) * rmin;
    const float cmid = gmid > thr ? tmid : 0.f, cmin = gmin > thr ? tmin : 0.f;
    const float alpha = 2.f * L.an;
    float p[3], q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        p[r] = alpha * vmax[r] + cmin * vmin[r] + cmid * vmid[r];
        q[r] = alpha * vmin[r];
    }
    out[0] = vmax[0] * p[0] - vmin[0] * q[0];
    out[1] = vmax[1] * p[1] - vmin[1] * q[1];
    out[2] = vmax[2] * p[2] - vmin[2] * q[2];
    out[3] = vmax[0] * p[1] + vmax[1] * p[0] - 2.f * vmin[0] * q[1];
    out[4] = vmax[0] * p[2] + vmax[2] * p[0] - 2.f * vmin[0] * q[2];
    out[5] = vmax[1] * p[2] + vmax[2] * p[1] - 2.f * vmin[1] * q[2];
}

// Kahan (compensated) running sum in FP32
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
}

// Per-block reduction of the two compensated sums into partials[2 blockIdx.x + {0, 1}] (FP64);
// every thread of the block takes part.
__device__ __forceinline__ void st_block_partials(float s0, float c0, float s1, float c1, double *partials) {
    double d0 = (double)s0 - (double)c0, d1 = (double)s1 - (double)c1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, off);
        d1 += __shfl_down_sync(0xffffffffu, d1, off);
    }
    __shared__ double sh[2][kStThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = d0; sh[1][warp] = d1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int k = 0; k < kStThreads / 32; ++k) { a += sh[0][k]; b += sh[1][k]; }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// One pass over the field, grid-stride, one tensor per thread and iteration. FWD accumulates the
// two loss terms into the block's partial sums, BWD writes scale * dL/dA. IT is the element-offset
// type (32-bit when every plane offset fits); plane addresses are one base per array plus
// loop-invariant plane offsets, and the next tensor of the sequence is loaded before the current
// one is decomposed, so that the load latency overlaps the arithmetic.
template <typename TI, typename IT, bool FWD, bool BWD>
__device__ __forceinline__ void st_pass(const TI *__restrict__ A, IT n, IT ld, float w0, float w1, float w2,
                                        float scale, const Params<float> &P, double *__restrict__ partials,
                                        TI *__restrict__ A_bar) {
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    const IT stride = (IT)gridDim.x * blockDim.x;
    IT i = (IT)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float a[6];
        const TI *Ai = A + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = ld_f(Ai + k * ld);
        for (;;) {
            const IT inext = i + stride;
            const bool more = inext < n;
            float b[6];
            if (more) {
                const TI *An = A + inext;
#pragma unroll
                for (int k = 0; k < 6; ++k) b[k] = ld_f(An + k * ld);
            }
            Eig3<float> E;
            eig3_method<float, true, INV_F32, true>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
            const StTerms L = st_terms(E, w0, w1, w2);
            if constexpr (FWD) {
                kahan_add(s0, c0, L.an * L.an);
                kahan_add(s1, c1, L.vw * L.vw);
            }
            if constexpr (BWD) {
                float out[6];
                st_grad(E, L, w0, w1, w2, P, out);
                TI *Gi = A_bar + i;
#pragma unroll
                for (int k = 0; k < 6; ++k) st_f(Gi + k * ld, scale * out[k]);
            }
            if (!more) break;
            i = inext;
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] = b[k];
        }
    }
    if constexpr (FWD) st_block_partials(s0, c0, s1, c1, partials);
}

template <typename TI, typename IT>
__global__ void __launch_bounds__(kStThreads, 1)
k_st_fwd(const TI *__restrict__ A, IT n, IT ld, float w0, float w1, float w2, Params<float> P,
         double *__restrict__ partials) {
    st_pass<TI, IT, true, false>(A, n, ld, w0, w1, w2, 1.f, P, partials, nullptr);
}

template <typename TI, typename IT>
__global__ void __launch_bounds__(kStThreads, 1)
k_st_bwd(const TI *__restrict__ A, IT n, IT ld, float w0, float w1, float w2, float scale, Params<float> P,
         TI *__restrict__ A_bar) {
    st_pass<TI, IT, false, true>(A, n, ld, w0, w1, w2, scale, P, nullptr, A_bar);
}

// Forward and backward in one pass: each tensor is decomposed once; the loss terms go to the
// per-block partial sums (as in k_st_fwd) and scale * dL/dA to A_bar.
template <typename TI, typename IT>
__global__ void __launch_bounds__(kStThreads, 1)
k_st_fwd_bwd(const TI *__restrict__ A, IT n, IT ld, float w0, float w1, float w2, float scale, Params<float> P,
             double *__restrict__ partials, TI *__restrict__ A_bar) {
    st_pass<TI, IT, true, true>(A, n, ld, w0, w1, w2, scale, P, partials, A_bar);
}

__global__ void __launch_bounds__(kThreads)
k_st_finalize(const double *__restrict__ partials, int blocks, double *__restrict__ loss) {
    double a = 0, b = 0;
    for (int k = threadIdx.x; k < blocks; k += blockDim.x) { a += partials[2 * k]; b += partials[2 * k + 1]; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ double sh[2][kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int k = 0; k < kThreads / 32; ++k) { x += sh[0][k]; y += sh[1][k]; }
        loss[0] = x;
        loss[1] = y;
    }
}

// 32-bit element offsets when every plane offset of the 6-plane arrays fits
inline bool st_small_index(int64_t ld) { return ld < (int64_t)600000000; }

int st_loss_blocks(int64_t n) {
    int a = grid_for(k_st_fwd<float, int64_t>, n, kStThreads), b = grid_for(k_st_fwd<uint16_t, int64_t>, n, kStThreads);
    int c = grid_for(k_st_fwd_bwd<float, int64_t>, n, kStThreads);
    int d = grid_for(k_st_fwd_bwd<uint16_t, int64_t>, n, kStThreads);
    int e = grid_for(k_st_fwd<float, uint32_t>, n, kStThreads), f = grid_for(k_st_fwd<uint16_t, uint32_t>, n, kStThreads);
    int g = grid_for(k_st_fwd_bwd<float, uint32_t>, n, kStThreads);
    int h = grid_for(k_st_fwd_bwd<uint16_t, uint32_t>, n, kStThreads);
    return max(max(max(a, b), max(c, d)), max(max(e, f), max(g, h)));
}

template <typename TI, typename IT>
static void run_st_fwd(const void *A, int64_t n, int64_t ld, const float w[3], double *partials, int blocks,
                       const Params<float> &P, cudaStream_t st) {
    k_st_fwd<TI, IT><<<blocks, kStThreads, 0, st>>>((const TI *)A, (IT)n, (IT)ld, w[0], w[1], w[2], P, partials);
}

template <typename TI, typename IT>
static void run_st_bwd(const void *A, int64_t n, int64_t ld, const float w[3], float scale, void *A_bar,
                       const Params<float> &P, cudaStream_t st) {
    auto k = k_st_bwd<TI, IT>;
    k<<<grid_for(k, n, kStThreads), kStThreads, 0, st>>>((const TI *)A, (IT)n, (IT)ld, w[0], w[1], w[2], scale, P,
                                                         (TI *)A_bar);
}

template <typename TI, typename IT>
static void run_st_fwd_bwd(const void *A, int64_t n, int64_t ld, const float w[3], float scale, double *partials,
                           int blocks, void *A_bar, const Params<float> &P, cudaStream_t st) {
    k_st_fwd_bwd<TI, IT><<<blocks, kStThreads, 0, st>>>((const TI *)A, (IT)n, (IT)ld, w[0], w[1], w[2], scale, P,
                                                        partials, (TI *)A_bar);
}

kd_status launch_st_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        double *partials, int blocks, double *loss, const kd_opts &o, cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    const bool small = st_small_index(ld);
    if (in_t == KD_BF16) {
        if (small) run_st_fwd<uint16_t, uint32_t>(A, n, ld, w, partials, blocks, P, st);
        else run_st_fwd<uint16_t, int64_t>(A, n, ld, w, partials, blocks, P, st);
    } else if (in_t == KD_F32) {
        if (small) run_st_fwd<float, uint32_t>(A, n, ld, w, partials, blocks, P, st);
        else run_st_fwd<float, int64_t>(A, n, ld, w, partials, blocks, P, st);
    } else {
        return KD_ERR_UNSUPPORTED;
    }
    kd_status s = launch_status();
    if (s != KD_OK) return s;
    k_st_finalize<<<1, kThreads, 0, st>>>(partials, blocks, loss);
    return launch_status();
}

kd_status launch_st_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        float scale, void *A_bar, const kd_opts &o, cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    const bool small = st_small_index(ld);
    if (in_t == KD_BF16) {
        if (small) run_st_bwd<uint16_t, uint32_t>(A, n, ld, w, scale, A_bar, P, st);
        else run_st_bwd<uint16_t, int64_t>(A, n, ld, w, scale, A_bar, P, st);
    } else if (in_t == KD_F32) {
        if (small) run_st_bwd<float, uint32_t>(A, n, ld, w, scale, A_bar, P, st);
        else run_st_bwd<float, int64_t>(A, n, ld, w, scale, A_bar, P, st);
    } else {
        return KD_ERR_UNSUPPORTED;
    }
    return launch_status();
}

kd_status launch_st_fwd_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                            double *partials, int blocks, double *loss, void *A_bar, const kd_opts &o,
                            cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    const bool small = st_small_index(ld);
    if (in_t == KD_BF16) {
        if (small) run_st_fwd_bwd<uint16_t, uint32_t>(A, n, ld, w, scale, partials, blocks, A_bar, P, st);
        else run_st_fwd_bwd<uint16_t, int64_t>(A, n, ld, w, scale, partials, blocks, A_bar, P, st);
    } else if (in_t == KD_F32) {
        if (small) run_st_fwd_bwd<float, uint32_t>(A, n, ld, w, scale, partials, blocks, A_bar, P, st);
        else run_st_fwd_bwd<float, int64_t>(A, n, ld, w, scale, partials, blocks, A_bar, P, st);
    } else {
        return KD_ERR_UNSUPPORTED;
    }
    kd_status s = launch_status();
    if (s != KD_OK) return s;
    k_st_finalize<<<1, kThreads, 0, st>>>(partials, blocks, loss);
    return launch_status();
}

}  // namespace kd
