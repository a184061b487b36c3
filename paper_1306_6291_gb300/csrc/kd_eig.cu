// Batched 3x3 and 2x2 kernels: forward (eigenvalues, D, angles) and adjoints. One thread per
// matrix, grid-stride over the batch; SoA planes read and written once with streaming
// (evict-first) cache hints, since every byte is touched exactly once.
#include <cuda_bf16.h>

#include "kd_internal.h"

// Minimum resident blocks per SM requested from the compiler for the 3x3 kernels (register cap).
#ifndef KD_FWD_MINB
#define KD_FWD_MINB 6
#endif
#ifndef KD_ADJ_MINB
#define KD_ADJ_MINB 5
#endif
// Threads per block of the 3x3 kernels.
#ifndef KD_EIG3_THREADS
#define KD_EIG3_THREADS 256
#endif

namespace kd {

// ---- loads / stores --------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T ld_as(const float *p) { return (T)__ldcs(p); }
template <typename T> __device__ __forceinline__ T ld_as(const double *p) { return (T)__ldcs(p); }
template <typename T> __device__ __forceinline__ T ld_as(const uint16_t *p) {
    return (T)__uint_as_float(((uint32_t)__ldcs((const unsigned short *)p)) << 16);
}
__device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st(double *p, double v) { __stcs(p, v); }

// Per-category counters, one atomic per warp and category.
__device__ __forceinline__ void count_kase(unsigned long long *stats, int kase) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const unsigned b = __ballot_sync(mask, kase == (c < 3 ? c : 255));
        if (b && lane == leader) atomicAdd(stats + c, (unsigned long long)__popc(b));
    }
}

// ---- 3x3 forward ---------------------------------------------------------------------------
// The six input planes of matrix i.
template <typename T, typename TI, typename IT>
__device__ __forceinline__ void load6(const TI *__restrict__ A, IT ld, IT i, T a[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = ld_as<T>(A + i + k * ld);
}

// IT is the element-offset type: 32-bit when every plane offset fits, else 64-bit. Each thread
// loads the next matrix of its grid-stride sequence before working on the current one, so the
// load latency overlaps the arithmetic. ALL: lam, D and angles requested, no kase or counters (a
// separate instantiation without the run-time output checks).
template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT, bool ALL>
__global__ void __launch_bounds__(KD_EIG3_THREADS, sizeof(T) == 4 ? KD_FWD_MINB : 1)
k_eig3_fwd(const TI *__restrict__ A, IT n, IT ld, T *__restrict__ lam, T *__restrict__ D,
           T *__restrict__ ang, uint8_t *__restrict__ kase, Params<T> P, unsigned long long *stats) {
    if constexpr (ALL) {
        kase = nullptr;
        stats = nullptr;
    }
    const IT stride = (IT)gridDim.x * blockDim.x;
    IT i = (IT)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a[6];
    load6(A, ld, i, a);
    for (;;) {
        const IT inext = i + stride;
        const bool more = inext < n;
        T b[6];
        if (more) load6(A, ld, inext, b);
        Eig3<T> E;
        eig3_method<T, MIXED, INV64, FAST>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
        if (ALL || lam) {
#pragma unroll
            for (int k = 0; k < 3; ++k) st(lam + i + k * ld, E.lam[k] * E.inv_s);
        }
        if (ALL || D) {
#pragma unroll
            for (int k = 0; k < 9; ++k) st(D + i + k * ld, E.D[k]);
        }
        if (ALL || ang) {
            T g[3];
            euler_from_D<T, FAST>(E.D, g);
            if (E.kase == 255) g[0] = g[1] = g[2] = E.lam[0];   // NaN
#pragma unroll
            for (int k = 0; k < 3; ++k) st(ang + i + k * ld, g[k]);
        }
        if (!ALL && kase) kase[i] = (uint8_t)E.kase;
        if (!ALL && stats) count_kase(stats, E.kase);
        if (!more) break;
        i = inext;
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = b[k];
    }
}

// ---- 3x3 adjoint ---------------------------------------------------------------------------
// Cotangents lam_bar (3), D_bar (9), ang_bar (3) of matrix i into c[0..14] (0 for a null plane).
template <typename T, typename IT>
__device__ __forceinline__ void load_cot(const T *__restrict__ lam_bar, const T *__restrict__ D_bar,
                                         const T *__restrict__ ang_bar, IT ld, IT i, T c[15]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = lam_bar ? ld_as<T>(lam_bar + i + k * ld) : T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) c[3 + k] = D_bar ? ld_as<T>(D_bar + i + k * ld) : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[12 + k] = ang_bar ? ld_as<T>(ang_bar + i + k * ld) : T(0);
}

// The inputs and cotangents of a matrix are loaded at the top of its iteration; with 5 blocks
// of 256 threads per SM (48 registers) the other warps cover their latency. (Prefetching the next
// matrix, in registers or staged in shared memory by cp.async, measured slower: more registers
// or more instructions per matrix.) Separate instantiations for calls with Euler-angle
// cotangents (ANG) and for calls with both lam_bar and D_bar given (FULL, loaded without null
// checks), so that the common calls carry no code for the absent ones.
template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT, bool ANG, bool FULL>
__global__ void __launch_bounds__(KD_EIG3_THREADS, sizeof(T) == 4 ? KD_ADJ_MINB : 1)
k_eig3_adj(const TI *__restrict__ A, IT n, IT ld, const T *__restrict__ lam_bar,
           const T *__restrict__ D_bar, const T *__restrict__ ang_bar, T *__restrict__ A_bar, Params<T> P) {
    const IT stride = (IT)gridDim.x * blockDim.x;
    for (IT i = (IT)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T c[15], a[6], out[6];
        if constexpr (FULL) {
#pragma unroll
            for (int k = 0; k < 3; ++k) c[k] = ld_as<T>(lam_bar + i + k * ld);
#pragma unroll
            for (int k = 0; k < 9; ++k) c[3 + k] = ld_as<T>(D_bar + i + k * ld);
#pragma unroll
            for (int k = 0; k < 3; ++k) c[12 + k] = ANG ? ld_as<T>(ang_bar + i + k * ld) : T(0);
        } else {
            load_cot(lam_bar, D_bar, ANG ? ang_bar : nullptr, ld, i, c);
        }
        load6(A, ld, i, a);
        Eig3<T> E;
        eig3_method<T, MIXED, INV64, FAST>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
        eig3_adjoint(E, c, c + 3, ANG, c + 12, P.gap_mask, out);
#pragma unroll
        for (int k = 0; k < 6; ++k) st(A_bar + i + k * ld, out[k]);
    }
}

// 32-bit offsets cover every plane (at most 9 per array) when 10 * ld < 2^32.
inline bool small_index(int64_t ld) { return ld < (int64_t)429496729; }

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT, bool ALL>
static void run_eig3_fwd_k(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang, uint8_t *kase,
                           const kd_opts &o, cudaStream_t st) {
    auto k = k_eig3_fwd<TI, T, MIXED, INV64, FAST, IT, ALL>;
    k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, (IT)n, (IT)ld, (T *)lam, (T *)D,
                                                                    (T *)ang, kase, resolve<T>(o), o.stats);
}

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST>
static kd_status run_eig3_fwd(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang,
                              uint8_t *kase, const kd_opts &o, cudaStream_t st) {
    const bool all = lam && D && ang && !kase && !o.stats;
    if (small_index(ld)) {
        if (all) run_eig3_fwd_k<TI, T, MIXED, INV64, FAST, uint32_t, true>(A, n, ld, lam, D, ang, kase, o, st);
        else run_eig3_fwd_k<TI, T, MIXED, INV64, FAST, uint32_t, false>(A, n, ld, lam, D, ang, kase, o, st);
    } else {
        if (all) run_eig3_fwd_k<TI, T, MIXED, INV64, FAST, int64_t, true>(A, n, ld, lam, D, ang, kase, o, st);
        else run_eig3_fwd_k<TI, T, MIXED, INV64, FAST, int64_t, false>(A, n, ld, lam, D, ang, kase, o, st);
    }
    return launch_status();
}

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT, bool ANG, bool FULL>
static void run_eig3_adj_k(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db, const void *ab,
                           void *Ab, const kd_opts &o, cudaStream_t st) {
    auto k = k_eig3_adj<TI, T, MIXED, INV64, FAST, IT, ANG, FULL>;
    k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, (IT)n, (IT)ld, (const T *)lb,
                                                                    (const T *)Db, (const T *)ab, (T *)Ab,
                                                                    resolve<T>(o));
}

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT>
static void run_eig3_adj_it(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db, const void *ab,
                            void *Ab, const kd_opts &o, cudaStream_t st) {
    const bool full = lb && Db;
    if (ab) {
        if (full) run_eig3_adj_k<TI, T, MIXED, INV64, FAST, IT, true, true>(A, n, ld, lb, Db, ab, Ab, o, st);
        else run_eig3_adj_k<TI, T, MIXED, INV64, FAST, IT, true, false>(A, n, ld, lb, Db, ab, Ab, o, st);
    } else {
        if (full) run_eig3_adj_k<TI, T, MIXED, INV64, FAST, IT, false, true>(A, n, ld, lb, Db, ab, Ab, o, st);
        else run_eig3_adj_k<TI, T, MIXED, INV64, FAST, IT, false, false>(A, n, ld, lb, Db, ab, Ab, o, st);
    }
}

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST>
static kd_status run_eig3_adj(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db,
                              const void *ab, void *Ab, const kd_opts &o, cudaStream_t st) {
    if (small_index(ld)) run_eig3_adj_it<TI, T, MIXED, INV64, FAST, uint32_t>(A, n, ld, lb, Db, ab, Ab, o, st);
    else run_eig3_adj_it<TI, T, MIXED, INV64, FAST, int64_t>(A, n, ld, lb, Db, ab, Ab, o, st);
    return launch_status();
}

kd_status launch_eig3_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, void *lam, void *D,
                          void *ang, uint8_t *kase, bool mixed, bool inv64, const kd_opts &o,
                          cudaStream_t st) {
    if (in_t == KD_F64) return run_eig3_fwd<double, double, false, false, false>(A, n, ld, lam, D, ang, kase, o, st);
    if (in_t == KD_F32) {
        if (!mixed) return run_eig3_fwd<float, float, false, false, false>(A, n, ld, lam, D, ang, kase, o, st);
        if (inv64) return run_eig3_fwd<float, float, true, true, true>(A, n, ld, lam, D, ang, kase, o, st);
        return run_eig3_fwd<float, float, true, false, true>(A, n, ld, lam, D, ang, kase, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv64) return run_eig3_fwd<uint16_t, float, true, true, true>(A, n, ld, lam, D, ang, kase, o, st);
        return run_eig3_fwd<uint16_t, float, true, false, true>(A, n, ld, lam, D, ang, kase, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

kd_status launch_eig3_adj(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const void *lam_bar,
                          const void *D_bar, const void *ang_bar, void *A_bar, bool mixed, bool inv64,
                          const kd_opts &o, cudaStream_t st) {
    if (in_t == KD_F64) return run_eig3_adj<double, double, false, false, false>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    if (in_t == KD_F32) {
        if (!mixed) return run_eig3_adj<float, float, false, false, false>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        if (inv64) return run_eig3_adj<float, float, true, true, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_eig3_adj<float, float, true, false, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv64) return run_eig3_adj<uint16_t, float, true, true, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_eig3_adj<uint16_t, float, true, false, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

// ---- 2x2 -----------------------------------------------------------------------------------
// The 2x2 arithmetic is ~50 instructions, so the kernel is bound by memory latency and bandwidth:
// each thread loads U matrices of its grid-stride sequence at once (3U loads in flight) before
// computing them.
template <typename T, int U, typename IT>
__global__ void __launch_bounds__(kThreads)
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
__global__ void __launch_bounds__(kThreads)
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
    k<<<grid_for(k, per), kThreads, 0, st>>>((const T *)A, (IT)n, (IT)ld, (T *)lam, (T *)phi, (T *)D, stats);
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
    k<<<grid_for(k, per), kThreads, 0, st>>>((const T *)A, (IT)n, (IT)ld, (const T *)lam_bar, (const T *)phi_bar,
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
