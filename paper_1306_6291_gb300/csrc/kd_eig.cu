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
#define KD_ADJ_MINB 1
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
    for (int k = 0; k < 6; ++k) a[k] = ld_as<T>(A + k * ld + i);
}

// Asynchronous element copies global -> shared (cp.async, 4 or 8 bytes): a thread stages the
// next matrix's inputs without holding them in registers. Each thread reads back only what it
// copied itself, after waiting for its own copies, so no block barrier is needed.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async element size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The six input planes of matrix i staged into s[k][threadIdx.x].
template <typename TI, typename IT>
__device__ __forceinline__ void stage6(TI (*s)[KD_EIG3_THREADS], const TI *__restrict__ A, IT ld, IT i) {
#pragma unroll
    for (int k = 0; k < 6; ++k) cp_async<sizeof(TI)>(&s[k][threadIdx.x], A + k * ld + i);
}

// IT is the element-offset type: 32-bit when every plane offset fits, else 64-bit. Each thread
// loads the next matrix of its grid-stride sequence before working on the current one, so the
// load latency overlaps the arithmetic.
template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT>
__global__ void __launch_bounds__(KD_EIG3_THREADS, KD_FWD_MINB)
k_eig3_fwd(const TI *__restrict__ A, IT n, IT ld, T *__restrict__ lam, T *__restrict__ D,
           T *__restrict__ ang, uint8_t *__restrict__ kase, Params<T> P, unsigned long long *stats) {
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
        if (lam) {
#pragma unroll
            for (int k = 0; k < 3; ++k) st(lam + k * ld + i, E.lam[k] * E.inv_s);
        }
        if (D) {
#pragma unroll
            for (int k = 0; k < 9; ++k) st(D + k * ld + i, E.D[k]);
        }
        if (ang) {
            T g[3];
            euler_from_D<T, FAST>(E.D, g);
            if (E.kase == 255) g[0] = g[1] = g[2] = E.lam[0];   // NaN
#pragma unroll
            for (int k = 0; k < 3; ++k) st(ang + k * ld + i, g[k]);
        }
        if (kase) kase[i] = (uint8_t)E.kase;
        if (stats) count_kase(stats, E.kase);
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
    for (int k = 0; k < 3; ++k) c[k] = lam_bar ? ld_as<T>(lam_bar + k * ld + i) : T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) c[3 + k] = D_bar ? ld_as<T>(D_bar + k * ld + i) : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[12 + k] = ang_bar ? ld_as<T>(ang_bar + k * ld + i) : T(0);
}

// The same staged into s[k][threadIdx.x] (planes that are null are not copied).
template <typename T, typename IT>
__device__ __forceinline__ void stage_cot(T (*s)[KD_EIG3_THREADS], const T *__restrict__ lam_bar,
                                          const T *__restrict__ D_bar, const T *__restrict__ ang_bar, IT ld, IT i) {
    if (lam_bar) {
#pragma unroll
        for (int k = 0; k < 3; ++k) cp_async<sizeof(T)>(&s[k][threadIdx.x], lam_bar + k * ld + i);
    }
    if (D_bar) {
#pragma unroll
        for (int k = 0; k < 9; ++k) cp_async<sizeof(T)>(&s[3 + k][threadIdx.x], D_bar + k * ld + i);
    }
    if (ang_bar) {
#pragma unroll
        for (int k = 0; k < 3; ++k) cp_async<sizeof(T)>(&s[12 + k][threadIdx.x], ang_bar + k * ld + i);
    }
}

// FP32 / FP64: the inputs and cotangents of matrix i + stride are staged (cp.async, double
// buffer) while matrix i is decomposed, and the cotangents of matrix i are read from shared
// memory only when the adjoint needs them. BF16: the cotangents of matrix i are loaded before its
// decomposition, the next matrix's input into registers.
template <typename TI, typename T, bool MIXED, bool INV64, bool FAST, typename IT>
__global__ void __launch_bounds__(KD_EIG3_THREADS, KD_ADJ_MINB)
k_eig3_adj(const TI *__restrict__ A, IT n, IT ld, const T *__restrict__ lam_bar,
           const T *__restrict__ D_bar, const T *__restrict__ ang_bar, T *__restrict__ A_bar, Params<T> P) {
    constexpr bool ASYNC = sizeof(TI) >= 4;
    __shared__ TI s_in[ASYNC ? 2 : 1][ASYNC ? 6 : 1][KD_EIG3_THREADS];
    __shared__ T s_cot[ASYNC ? 2 : 1][ASYNC ? 15 : 1][KD_EIG3_THREADS];
    const IT stride = (IT)gridDim.x * blockDim.x;
    IT i = (IT)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a[6];
    if constexpr (ASYNC) {
        stage6<TI>(s_in[0], A, ld, i);
        stage_cot<T>(s_cot[0], lam_bar, D_bar, ang_bar, ld, i);
        cp_async_commit();
    } else {
        load6(A, ld, i, a);
    }
    for (int it = 0;; ++it) {
        const int cur = it & 1;
        const IT inext = i + stride;
        const bool more = inext < n;
        T c[15], b[6], out[6];
        if constexpr (ASYNC) {
            cp_async_wait_all();
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] = (T)s_in[cur][k][threadIdx.x];
            if (more) {
                stage6<TI>(s_in[cur ^ 1], A, ld, inext);
                stage_cot<T>(s_cot[cur ^ 1], lam_bar, D_bar, ang_bar, ld, inext);
            }
            cp_async_commit();
        } else {
            load_cot(lam_bar, D_bar, ang_bar, ld, i, c);
            if (more) load6(A, ld, inext, b);
        }
        Eig3<T> E;
        eig3_method<T, MIXED, INV64, FAST>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
        if constexpr (ASYNC) {
#pragma unroll
            for (int k = 0; k < 3; ++k) c[k] = lam_bar ? s_cot[cur][k][threadIdx.x] : T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) c[3 + k] = D_bar ? s_cot[cur][3 + k][threadIdx.x] : T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) c[12 + k] = ang_bar ? s_cot[cur][12 + k][threadIdx.x] : T(0);
        }
        eig3_adjoint(E, c, c + 3, ang_bar != nullptr, c + 12, P.gap_mask, out);
#pragma unroll
        for (int k = 0; k < 6; ++k) st(A_bar + k * ld + i, out[k]);
        if (!more) break;
        i = inext;
        if constexpr (!ASYNC) {
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] = b[k];
        }
    }
}

// 32-bit offsets cover every plane (at most 9 per array) when 10 * ld < 2^32.
inline bool small_index(int64_t ld) { return ld < (int64_t)429496729; }

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST>
static kd_status run_eig3_fwd(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang,
                              uint8_t *kase, const kd_opts &o, cudaStream_t st) {
    if (small_index(ld)) {
        auto k = k_eig3_fwd<TI, T, MIXED, INV64, FAST, uint32_t>;
        k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, (uint32_t)n, (uint32_t)ld, (T *)lam, (T *)D,
                                                (T *)ang, kase, resolve<T>(o), o.stats);
    } else {
        auto k = k_eig3_fwd<TI, T, MIXED, INV64, FAST, int64_t>;
        k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, n, ld, (T *)lam, (T *)D, (T *)ang, kase,
                                                resolve<T>(o), o.stats);
    }
    return launch_status();
}

template <typename TI, typename T, bool MIXED, bool INV64, bool FAST>
static kd_status run_eig3_adj(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db,
                              const void *ab, void *Ab, const kd_opts &o, cudaStream_t st) {
    if (small_index(ld)) {
        auto k = k_eig3_adj<TI, T, MIXED, INV64, FAST, uint32_t>;
        k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, (uint32_t)n, (uint32_t)ld, (const T *)lb,
                                                (const T *)Db, (const T *)ab, (T *)Ab, resolve<T>(o));
    } else {
        auto k = k_eig3_adj<TI, T, MIXED, INV64, FAST, int64_t>;
        k<<<grid_for(k, n, KD_EIG3_THREADS), KD_EIG3_THREADS, 0, st>>>((const TI *)A, n, ld, (const T *)lb, (const T *)Db, (const T *)ab,
                                                (T *)Ab, resolve<T>(o));
    }
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
                for (int k = 0; k < 3; ++k) x[u][k] = ld_as<T>(A + k * ld + i);
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
                st(lam + ld + i, E.lam[1] * E.inv_s);
            }
            if (phi) st(phi + i, E.phi);
            if (D) {
                st(D + i, E.c);
                st(D + ld + i, -E.s);
                st(D + 2 * ld + i, E.s);
                st(D + 3 * ld + i, E.c);
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
                for (int k = 0; k < 3; ++k) x[u][k] = ld_as<T>(A + k * ld + i);
                x[u][3] = lam_bar ? ld_as<T>(lam_bar + i) : T(0);
                x[u][4] = lam_bar ? ld_as<T>(lam_bar + ld + i) : T(0);
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
            st(A_bar + ld + i, s * s * lb1 + c * c * lb2 + c * s * t);
            st(A_bar + 2 * ld + i, T(2) * c * s * (lb1 - lb2) + (c * c - s * s) * t);
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
