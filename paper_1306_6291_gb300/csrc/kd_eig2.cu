// Batched 2x2 forward and adjoint (Section 3): eigenvalues, angle and D of each matrix; one
// thread handles four matrices of its grid-stride sequence.
#include "kd_soa.cuh"

namespace kd {

// Threads per block of the 2x2 kernels (measured: 512 slightly ahead of 256 and of 1024).
constexpr int kEig2Threads = 512;

// The 2x2 arithmetic is ~50 instructions, so the kernel is bound by memory latency and bandwidth:
// each thread loads U matrices of its grid-stride sequence at once (3U loads in flight) before
// computing them.
template <typename T, int U, typename IT>
__global__ void __launch_bounds__(kEig2Threads)
k_eig2_fwd(const T *__restrict__ A, IT n, IT ld, T *__restrict__ lam, T *__restrict__ phi,
           T *__restrict__ D, unsigned long long *stats) {
    const IT stride = (IT)gridDim.x * blockDim.x;
    for (IT i0 = (IT)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        T x[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const IT i = i0 + u * stride;
            if (i < n) {
#pragma unroll
                for (int k = 0; k < 3; ++k) x[u][k] = ld_as<T>(A + i + k * ld);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const IT i = i0 + u * stride;
            if (i >= n) break;
            Eig2<T> E;
            eig2_method<T, sizeof(T) == 4>(x[u][0], x[u][1], x[u][2], E);
            if (lam) {
                st(lam + i, E.lam[0] * E.inv_s);
                st(lam + i + ld, E.lam[1] * E.inv_s);
            }
            if (phi) st(phi + i, E.phi);
            if (D) {
                st(D + i, E.c);
                st(D + i + ld, -E.s);
                st(D + i + 2 * ld, E.s);
                st(D + i + 3 * ld, E.c);
            }
            if (stats) count_kase(stats, E.bad ? 255 : (E.lam[0] == E.lam[1] ? 1 : 0));
        }
    }
}

// The 2x2 adjoint, unrolled like the forward: A and the cotangents of U matrices are loaded
// together before any is computed.
template <typename T, int U, typename IT>
__global__ void __launch_bounds__(kEig2Threads)
k_eig2_adj(const T *__restrict__ A, IT n, IT ld, const T *__restrict__ lam_bar,
           const T *__restrict__ phi_bar, T *__restrict__ A_bar, T gap_mask) {
    const IT stride = (IT)gridDim.x * blockDim.x;
    for (IT i0 = (IT)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        T x[U][6];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const IT i = i0 + u * stride;
            if (i < n) {
#pragma unroll
                for (int k = 0; k < 3; ++k) x[u][k] = ld_as<T>(A + i + k * ld);
                x[u][3] = lam_bar ? ld_as<T>(lam_bar + i) : T(0);
                x[u][4] = lam_bar ? ld_as<T>(lam_bar + i + ld) : T(0);
                x[u][5] = phi_bar ? ld_as<T>(phi_bar + i) : T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const IT i = i0 + u * stride;
            if (i >= n) break;
            Eig2<T> E;
            eig2_method<T, sizeof(T) == 4>(x[u][0], x[u][1], x[u][2], E);
            const T lb1 = x[u][3], lb2 = x[u][4], pb = x[u][5];
            const T c = E.c, s = E.s, gap = E.lam[0] - E.lam[1];   // scaled units
            // 1/(lam1 - lam2) of the unscaled matrix = s_scale / gap
            const T t = (k_abs(gap) > gap_mask * E.fro) ? pb * E.s_scale * k_rcp(gap) : T(0);
            st(A_bar + i, c * c * lb1 + s * s * lb2 - c * s * t);
            st(A_bar + i + ld, s * s * lb1 + c * c * lb2 + c * s * t);
            st(A_bar + i + 2 * ld, T(2) * c * s * (lb1 - lb2) + (c * c - s * s) * t);
        }
    }
}

template <typename T, typename IT>
static void run_eig2_fwd(const void *A, int64_t n, int64_t ld, void *lam, void *phi, void *D,
                         unsigned long long *stats, cudaStream_t st) {
    constexpr int U = 4;
    auto k = k_eig2_fwd<T, U, IT>;
    const int64_t per = (n + U - 1) / U;   // each thread handles up to U matrices
    k<<<grid_for(k, per, kEig2Threads), kEig2Threads, 0, st>>>((const T *)A, (IT)n, (IT)ld, (T *)lam, (T *)phi, (T *)D, stats);
}

// 32-bit offsets when every plane offset and the unrolled indices fit (4 planes of D, and
// i0 + 4 * stride stays below 2^32).
kd_status launch_eig2_fwd(const void *A, kd_dtype t, int64_t n, int64_t ld, void *lam, void *phi,
                          void *D, const kd_opts &o, cudaStream_t st) {
    const bool small = ld < (int64_t)858993459;
    if (t == KD_F32) {
        if (small) run_eig2_fwd<float, uint32_t>(A, n, ld, lam, phi, D, o.stats, st);
        else run_eig2_fwd<float, int64_t>(A, n, ld, lam, phi, D, o.stats, st);
        return launch_status();
    }
    if (t == KD_F64) {
        if (small) run_eig2_fwd<double, uint32_t>(A, n, ld, lam, phi, D, o.stats, st);
        else run_eig2_fwd<double, int64_t>(A, n, ld, lam, phi, D, o.stats, st);
        return launch_status();
    }
    return KD_ERR_UNSUPPORTED;
}

template <typename T, typename IT>
static void run_eig2_adj(const void *A, int64_t n, int64_t ld, const void *lam_bar, const void *phi_bar,
                         void *A_bar, T gap_mask, cudaStream_t st) {
    constexpr int U = 4;
    auto k = k_eig2_adj<T, U, IT>;
    const int64_t per = (n + U - 1) / U;
    k<<<grid_for(k, per, kEig2Threads), kEig2Threads, 0, st>>>((const T *)A, (IT)n, (IT)ld, (const T *)lam_bar, (const T *)phi_bar,
                                              (T *)A_bar, gap_mask);
}

kd_status launch_eig2_adj(const void *A, kd_dtype t, int64_t n, int64_t ld, const void *lam_bar,
                          const void *phi_bar, void *A_bar, const kd_opts &o, cudaStream_t st) {
    const bool small = ld < (int64_t)858993459;
    if (t == KD_F32) {
        const float gm = resolve<float>(o).gap_mask;
        if (small) run_eig2_adj<float, uint32_t>(A, n, ld, lam_bar, phi_bar, A_bar, gm, st);
        else run_eig2_adj<float, int64_t>(A, n, ld, lam_bar, phi_bar, A_bar, gm, st);
        return launch_status();
    }
    if (t == KD_F64) {
        const double gm = resolve<double>(o).gap_mask;
        if (small) run_eig2_adj<double, uint32_t>(A, n, ld, lam_bar, phi_bar, A_bar, gm, st);
        else run_eig2_adj<double, int64_t>(A, n, ld, lam_bar, phi_bar, A_bar, gm, st);
        return launch_status();
    }
    return KD_ERR_UNSUPPORTED;
}

}  // namespace kd
