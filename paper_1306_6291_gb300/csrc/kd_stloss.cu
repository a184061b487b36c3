// Structure-tensor loss over a field of 3x3 tensors, forward (two sums) and backward (packed
// gradient per tensor), each tensor decomposed by the FP32 precision form of the method.
//   L = sum (lam_max - lam_min)^2 + sum (v_max . w)^2
// The forward kernel keeps compensated FP32 sums per thread, reduces them per block in FP64 into
// a workspace of per-block partials, and a one-block kernel adds the partials in a fixed order,
// so the result does not depend on scheduling.
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

// Labels of the largest and smallest eigenvalue (on ties the first index wins; when all three
// are equal the smallest is taken as the next label after the largest), the eigenvalue term's
// root an = lam_max - lam_min (unscaled) and vw = v_max . w. Written with selects only, so that no
// array is indexed by a run-time label (which would move it to local memory).
struct StTerms {
    int imax, imin;
    float an, vw;
    float vmax[3];
};
__device__ __forceinline__ float sel3(int k, float a, float b, float c) { return k == 0 ? a : (k == 1 ? b : c); }
__device__ __forceinline__ StTerms st_terms(const Eig3<float> &E, float w0, float w1, float w2) {
    StTerms t;
    float vmax = E.lam[0], vmin = E.lam[0];
    t.imax = 0;
    t.imin = 0;
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        if (E.lam[k] > vmax) { vmax = E.lam[k]; t.imax = k; }
        if (E.lam[k] < vmin) { vmin = E.lam[k]; t.imin = k; }
    }
    if (t.imax == t.imin) t.imin = t.imax == 2 ? 0 : t.imax + 1;   // all equal: vmin = vmax
    t.an = (vmax - vmin) * E.inv_s;
#pragma unroll
    for (int r = 0; r < 3; ++r) t.vmax[r] = sel3(t.imax, E.D[3 * r], E.D[3 * r + 1], E.D[3 * r + 2]);
    t.vw = t.vmax[0] * w0 + t.vmax[1] * w1 + t.vmax[2] * w2;
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
// A_ba). The 1/(lam_max - lam_j) are taken from the scaled eigenvalues: s / (lam_s_max - lam_s_j).
__device__ __forceinline__ void st_grad(const Eig3<float> &E, const StTerms &L, float w0, float w1, float w2,
                                        const Params<float> &P, float out[6]) {
    const int imid = 3 - L.imax - L.imin;
    float vmin[3], vmid[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        vmin[r] = sel3(L.imin, E.D[3 * r], E.D[3 * r + 1], E.D[3 * r + 2]);
        vmid[r] = sel3(imid, E.D[3 * r], E.D[3 * r + 1], E.D[3 * r + 2]);
    }
    const float lmax = sel3(L.imax, E.lam[0], E.lam[1], E.lam[2]);
    const float gmin = lmax - sel3(L.imin, E.lam[0], E.lam[1], E.lam[2]);
    const float gmid = lmax - sel3(imid, E.lam[0], E.lam[1], E.lam[2]);
    const float thr = P.gap_mask * E.fro;
    const float g2 = 2.f * L.vw;
    const float cmin = gmin > thr ? g2 * (vmin[0] * w0 + vmin[1] * w1 + vmin[2] * w2) * E.s * k_rcp(gmin) : 0.f;
    const float cmid = gmid > thr ? g2 * (vmid[0] * w0 + vmid[1] * w1 + vmid[2] * w2) * E.s * k_rcp(gmid) : 0.f;
    const float alpha = 2.f * L.an;
    float p[3], q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        p[r] = alpha * L.vmax[r] + cmin * vmin[r] + cmid * vmid[r];
        q[r] = alpha * vmin[r];
    }
    out[0] = L.vmax[0] * p[0] - vmin[0] * q[0];
    out[1] = L.vmax[1] * p[1] - vmin[1] * q[1];
    out[2] = L.vmax[2] * p[2] - vmin[2] * q[2];
    out[3] = L.vmax[0] * p[1] + L.vmax[1] * p[0] - 2.f * vmin[0] * q[1];
    out[4] = L.vmax[0] * p[2] + L.vmax[2] * p[0] - 2.f * vmin[0] * q[2];
    out[5] = L.vmax[1] * p[2] + L.vmax[2] * p[1] - 2.f * vmin[1] * q[2];
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
