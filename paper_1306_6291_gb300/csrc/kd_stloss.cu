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
    t.vw = sel3(t.imax, E.D[0], E.D[1], E.D[2]) * w0 + sel3(t.imax, E.D[3], E.D[4], E.D[5]) * w1 +
           sel3(t.imax, E.D[6], E.D[7], E.D[8]) * w2;
    return t;
}

template <typename TI>
__device__ __forceinline__ void st_decompose(const TI *A, int64_t ld, int64_t i, const Params<float> &P,
                                             Eig3<float> &E) {
    eig3_method<float, true, false, true>(ld_f(A + i), ld_f(A + i + ld), ld_f(A + i + 2 * ld),
                                          ld_f(A + i + 3 * ld), ld_f(A + i + 4 * ld), ld_f(A + i + 5 * ld), P, E);
}

template <typename TI>
__global__ void __launch_bounds__(kStThreads)
k_st_fwd(const TI *__restrict__ A, int64_t n, int64_t ld, float w0, float w1, float w2,
         Params<float> P, double *__restrict__ partials) {
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;   // Kahan sums
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Eig3<float> E;
        st_decompose(A, ld, i, P, E);
        const StTerms L = st_terms(E, w0, w1, w2);
        float y = L.an * L.an - c0, t = s0 + y;
        c0 = (t - s0) - y; s0 = t;
        y = L.vw * L.vw - c1; t = s1 + y;
        c1 = (t - s1) - y; s1 = t;
    }
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

// Packed gradient of one tensor's loss terms: lam_bar = +-2 (lam_max - lam_min) at the two
// labels, D_bar = 2 (v_max . w) w in the column of lam_max, through the 3x3 adjoint.
__device__ __forceinline__ void st_grad(const Eig3<float> &E, const StTerms &L, float w0, float w1, float w2,
                                        const Params<float> &P, float out[6]) {
    float lb[3], Db[9];
    const float g = 2.f * L.vw;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lb[k] = (k == L.imax ? 2.f * L.an : 0.f) - (k == L.imin ? 2.f * L.an : 0.f);
        Db[k] = k == L.imax ? g * w0 : 0.f;
        Db[3 + k] = k == L.imax ? g * w1 : 0.f;
        Db[6 + k] = k == L.imax ? g * w2 : 0.f;
    }
    eig3_adjoint(E, lb, Db, false, lb, P.gap_mask, out);
}

template <typename TI>
__global__ void __launch_bounds__(kStThreads)
k_st_bwd(const TI *__restrict__ A, int64_t n, int64_t ld, float w0, float w1, float w2, float scale,
         Params<float> P, TI *__restrict__ A_bar) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Eig3<float> E;
        st_decompose(A, ld, i, P, E);
        const StTerms L = st_terms(E, w0, w1, w2);
        float out[6];
        st_grad(E, L, w0, w1, w2, P, out);
#pragma unroll
        for (int k = 0; k < 6; ++k) st_f(A_bar + i + k * ld, scale * out[k]);
    }
}

// Forward and backward in one pass: each tensor is decomposed once; the loss terms go to the
// per-block partial sums (as in k_st_fwd) and scale * dL/dA to A_bar.
template <typename TI>
__global__ void __launch_bounds__(kStThreads)
k_st_fwd_bwd(const TI *__restrict__ A, int64_t n, int64_t ld, float w0, float w1, float w2, float scale,
             Params<float> P, double *__restrict__ partials, TI *__restrict__ A_bar) {
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;   // Kahan sums
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Eig3<float> E;
        st_decompose(A, ld, i, P, E);
        const StTerms L = st_terms(E, w0, w1, w2);
        float y = L.an * L.an - c0, t = s0 + y;
        c0 = (t - s0) - y; s0 = t;
        y = L.vw * L.vw - c1; t = s1 + y;
        c1 = (t - s1) - y; s1 = t;
        float out[6];
        st_grad(E, L, w0, w1, w2, P, out);
#pragma unroll
        for (int k = 0; k < 6; ++k) st_f(A_bar + i + k * ld, scale * out[k]);
    }
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

int st_loss_blocks(int64_t n) {
    int a = grid_for(k_st_fwd<float>, n, kStThreads), b = grid_for(k_st_fwd<uint16_t>, n, kStThreads);
    int c = grid_for(k_st_fwd_bwd<float>, n, kStThreads), d = grid_for(k_st_fwd_bwd<uint16_t>, n, kStThreads);
    return max(max(a, b), max(c, d));
}

kd_status launch_st_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        double *partials, int blocks, double *loss, const kd_opts &o, cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    if (in_t == KD_BF16)
        k_st_fwd<uint16_t><<<blocks, kStThreads, 0, st>>>((const uint16_t *)A, n, ld, w[0], w[1], w[2], P, partials);
    else if (in_t == KD_F32)
        k_st_fwd<float><<<blocks, kStThreads, 0, st>>>((const float *)A, n, ld, w[0], w[1], w[2], P, partials);
    else
        return KD_ERR_UNSUPPORTED;
    kd_status s = launch_status();
    if (s != KD_OK) return s;
    k_st_finalize<<<1, kThreads, 0, st>>>(partials, blocks, loss);
    return launch_status();
}

kd_status launch_st_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        float scale, void *A_bar, const kd_opts &o, cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    if (in_t == KD_BF16) {
        auto k = k_st_bwd<uint16_t>;
        k<<<grid_for(k, n, kStThreads), kStThreads, 0, st>>>((const uint16_t *)A, n, ld, w[0], w[1], w[2], scale, P,
                                                (uint16_t *)A_bar);
    } else if (in_t == KD_F32) {
        auto k = k_st_bwd<float>;
        k<<<grid_for(k, n, kStThreads), kStThreads, 0, st>>>((const float *)A, n, ld, w[0], w[1], w[2], scale, P,
                                                (float *)A_bar);
    } else {
        return KD_ERR_UNSUPPORTED;
    }
    return launch_status();
}

kd_status launch_st_fwd_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                            double *partials, int blocks, double *loss, void *A_bar, const kd_opts &o,
                            cudaStream_t st) {
    const Params<float> P = resolve<float>(o);
    if (in_t == KD_BF16)
        k_st_fwd_bwd<uint16_t><<<blocks, kStThreads, 0, st>>>((const uint16_t *)A, n, ld, w[0], w[1], w[2], scale, P,
                                                             partials, (uint16_t *)A_bar);
    else if (in_t == KD_F32)
        k_st_fwd_bwd<float><<<blocks, kStThreads, 0, st>>>((const float *)A, n, ld, w[0], w[1], w[2], scale, P,
                                                          partials, (float *)A_bar);
    else
        return KD_ERR_UNSUPPORTED;
    kd_status s = launch_status();
    if (s != KD_OK) return s;
    k_st_finalize<<<1, kThreads, 0, st>>>(partials, blocks, loss);
    return launch_status();
}

}  // namespace kd
