// Array-of-structures batches: matrix i is the record (A11, A22, A33, A12, A13, A23) at element
// 6 i; outputs are records too (lam 3, D 9, angles 3, A_bar 6 per matrix).
//
// FP32 forward with 16-byte aligned arrays: tiles of 256 matrices move through shared memory
// with 1-D TMA bulk copies (cp.async.bulk): the next tile's 6 KiB input is in flight while the
// current tile is decomposed, the outputs are written to shared memory and stored back as three
// contiguous bulk copies. Each thread reads its record as three 8-byte words (conflict-free) and
// writes its outputs at record strides 3 and 9 (conflict-free, strides odd). Tiles that are not
// whole (the tail) and every other dtype or alignment use plain per-thread loads and stores.
//
// Every wait on a TMA transaction is bounded (2 s): on expiry the block stops, sets bit 0 of the
// library's fault word (kd_device_fault) and returns; no wait is unbounded.
#include "kd_soa.cuh"

namespace kd {

__device__ unsigned int g_fault = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true when the phase completed; false once limit_ns have passed without it
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, phase))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void tma_load_1d(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(smem_dst)),
                 "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_store_1d(void *gmem_dst, const void *smem_src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem_dst), "r"(smem_u32(smem_src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

constexpr int kTile = 256;                    // matrices per tile = threads per block
constexpr uint64_t kWaitLimitNs = 2000000000ull;

template <typename T> __device__ __forceinline__ T ld_aos(const float *p) { return (T)*p; }
template <typename T> __device__ __forceinline__ T ld_aos(const double *p) { return (T)*p; }
template <typename T> __device__ __forceinline__ T ld_aos(const uint16_t *p) {
    return (T)__uint_as_float(((uint32_t)*p) << 16);
}

// ---- FP32 forward through TMA-staged tiles ---------------------------------------------------
// ALL: lam, D and angles requested and no kase (an instantiation without run-time output checks).
template <bool MIXED, int INV, bool FAST, bool ALL>
__global__ void __launch_bounds__(kTile)
k_eig3_fwd_aos_tma(const float *__restrict__ A, uint32_t ntiles, float *__restrict__ lam, float *__restrict__ D,
                   float *__restrict__ ang, uint8_t *__restrict__ kase, Params<float> P,
                   unsigned long long *stats) {
    __shared__ __align__(128) float s_in[2][kTile * 6];
    __shared__ __align__(128) float s_lam[kTile * 3];
    __shared__ __align__(128) float s_D[kTile * 9];
    __shared__ __align__(128) float s_ang[kTile * 3];
    __shared__ __align__(8) uint64_t s_bar[2];
    const int tid = threadIdx.x;
    const uint32_t in_bytes = kTile * 6 * sizeof(float);
    // tiles in order, block b taking b, b + G, ...: the scrambled order of the SoA kernels
    // (TileWalk) measured 2% slower here (0.273 against 0.268 ms on the precision workload)
    uint32_t t = blockIdx.x;
    if (t >= ntiles) return;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&s_bar[0], in_bytes);
        tma_load_1d(s_in[0], A + (size_t)t * kTile * 6, in_bytes, &s_bar[0]);
    }
    uint32_t ph0 = 0u, ph1 = 0u;
    for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
        const int buf = it & 1;
        const uint32_t tn = t + gridDim.x;
        const bool more = tn < ntiles;
        if (tid == 0 && more) {
            // every thread finished reading s_in[buf ^ 1] before the last __syncthreads
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[buf ^ 1], in_bytes);
            tma_load_1d(s_in[buf ^ 1], A + (size_t)tn * kTile * 6, in_bytes, &s_bar[buf ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&s_bar[buf], buf ? ph1 : ph0, kWaitLimitNs);
        if (buf) ph1 ^= 1u; else ph0 ^= 1u;
        if (__syncthreads_or(!ok)) {
            // give up on this block: record the fault, let the copies already issued finish
            // (each wait bounded again) and return
            if (tid == 0) {
                atomicOr(&g_fault, 1u);
                if (more) (void)mbar_wait_bounded(&s_bar[buf ^ 1], buf ? ph0 : ph1, kWaitLimitNs);
                bulk_wait0();
            }
            return;
        }
        const float2 *in2 = reinterpret_cast<const float2 *>(s_in[buf]) + tid * 3;
        const float2 x0 = in2[0], x1 = in2[1], x2 = in2[2];
        Eig3<float> E;
        eig3_method<float, MIXED, INV, FAST>(x0.x, x0.y, x1.x, x1.y, x2.x, x2.y, P, E);
        float g[3] = {0.f, 0.f, 0.f};
        if (ALL || ang) {
            euler_from_D<float, FAST>(E.D, g);
            if (E.kase == 255) g[0] = g[1] = g[2] = E.lam[0];
        }
        if (!ALL && kase) kase[(size_t)t * kTile + tid] = (uint8_t)kase_code(E);
        if (!ALL && stats) count_kase(stats, kase_code(E));
        // the previous tile's bulk stores must have finished reading the staging buffers
        if (tid == 0) bulk_wait_read0();
        __syncthreads();
        if (ALL || lam) {
#pragma unroll
            for (int k = 0; k < 3; ++k) s_lam[tid * 3 + k] = E.lam[k] * E.inv_s;
        }
        if (ALL || D) {
#pragma unroll
            for (int k = 0; k < 9; ++k) s_D[tid * 9 + k] = E.D[k];
        }
        if (ALL || ang) {
#pragma unroll
            for (int k = 0; k < 3; ++k) s_ang[tid * 3 + k] = g[k];
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const size_t base = (size_t)t * kTile;
            if (lam) tma_store_1d(lam + base * 3, s_lam, kTile * 3 * sizeof(float));
            if (D) tma_store_1d(D + base * 9, s_D, kTile * 9 * sizeof(float));
            if (ang) tma_store_1d(ang + base * 3, s_ang, kTile * 3 * sizeof(float));
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();
}

// ---- any dtype / alignment: plain per-thread records ------------------------------------------
template <typename TI, typename T, bool MIXED, int INV, bool FAST>
__global__ void __launch_bounds__(kTile)
k_eig3_fwd_aos(const TI *__restrict__ A, int64_t first, int64_t n, T *__restrict__ lam, T *__restrict__ D,
               T *__restrict__ ang, uint8_t *__restrict__ kase, Params<T> P, unsigned long long *stats) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const TI *a = A + 6 * i;
        Eig3<T> E;
        eig3_method<T, MIXED, INV, FAST>(ld_aos<T>(a), ld_aos<T>(a + 1), ld_aos<T>(a + 2), ld_aos<T>(a + 3),
                                           ld_aos<T>(a + 4), ld_aos<T>(a + 5), P, E);
        if (lam) {
#pragma unroll
            for (int k = 0; k < 3; ++k) lam[3 * i + k] = E.lam[k] * E.inv_s;
        }
        if (D) {
#pragma unroll
            for (int k = 0; k < 9; ++k) D[9 * i + k] = E.D[k];
        }
        if (ang) {
            T g[3];
            euler_from_D<T, FAST>(E.D, g);
            if (E.kase == 255) g[0] = g[1] = g[2] = E.lam[0];
#pragma unroll
            for (int k = 0; k < 3; ++k) ang[3 * i + k] = g[k];
        }
        if (kase) kase[i] = (uint8_t)kase_code(E);
        if (stats) count_kase(stats, kase_code(E));
    }
}

// ANG: angle cotangents given; FULL: lam_bar and D_bar both given (instantiations without the
// checks of absent cotangents).
template <typename TI, typename T, bool MIXED, int INV, bool FAST, bool ANG, bool FULL>
__global__ void __launch_bounds__(kTile)
k_eig3_adj_aos(const TI *__restrict__ A, int64_t n, const T *__restrict__ lam_bar, const T *__restrict__ D_bar,
               const T *__restrict__ ang_bar, T *__restrict__ A_bar, Params<T> P, TileWalk W) {
    // tiles of kTile matrices in the scrambled order of TileWalk; past the end of a partial last
    // tile the loads are clamped to the last matrix and nothing is stored
    if (blockIdx.x >= W.T) return;
    const int64_t last = n - 1;
    uint32_t t = tile_first(W);
    for (uint32_t j = blockIdx.x; j < W.T; j += gridDim.x, t = tile_next(W, t)) {
        const int64_t i = (int64_t)t * blockDim.x + threadIdx.x;
        const int64_t ic = i < last ? i : last;
        const TI *a = A + 6 * ic;
        T lb[3], Db[9], ab[3], out[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) lb[k] = (FULL || lam_bar) ? lam_bar[3 * ic + k] : T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) Db[k] = (FULL || D_bar) ? D_bar[9 * ic + k] : T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) ab[k] = ANG ? ang_bar[3 * ic + k] : T(0);
        Eig3<T> E;
        eig3_method<T, MIXED, INV, FAST>(ld_aos<T>(a), ld_aos<T>(a + 1), ld_aos<T>(a + 2), ld_aos<T>(a + 3),
                                           ld_aos<T>(a + 4), ld_aos<T>(a + 5), P, E);
        eig3_adjoint(E, lb, Db, ANG, ab, P.gap_mask, out);
        if (i < n) {
#pragma unroll
            for (int k = 0; k < 6; ++k) A_bar[6 * i + k] = out[k];
        }
    }
}

// ---- self-test of the bounded wait ------------------------------------------------------------
// One thread arms an mbarrier for a transaction that is never issued and waits with a short
// limit; it must give up and report through *flag (1 = gave up as designed).
__global__ void k_selftest_wait_timeout(unsigned int *flag, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16);
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    *flag = ok ? 2u : 1u;
}

// ---- launchers ----------------------------------------------------------------------------
template <typename TI, typename T, bool MIXED, int INV, bool FAST>
static kd_status run_fwd_aos(const void *A, int64_t first, int64_t n, void *lam, void *D, void *ang, uint8_t *kase,
                             const kd_opts &o, cudaStream_t st) {
    if (first >= n) return KD_OK;
    auto k = k_eig3_fwd_aos<TI, T, MIXED, INV, FAST>;
    k<<<grid_for(k, n - first, kTile), kTile, 0, st>>>((const TI *)A, first, n, (T *)lam, (T *)D, (T *)ang, kase,
                                                       resolve<T>(o), o.stats);
    return launch_status();
}

template <bool MIXED, int INV>
static kd_status run_fwd_aos_f32(const void *A, int64_t n, void *lam, void *D, void *ang, uint8_t *kase,
                                 const kd_opts &o, cudaStream_t st) {
    const bool tma = aligned(A, 16) && aligned(lam, 16) && aligned(D, 16) && aligned(ang, 16);
    const int64_t ntiles = tma ? n / kTile : 0;
    if (ntiles > 0) {
        const bool all = lam && D && ang && !kase && !o.stats;
        auto k = all ? k_eig3_fwd_aos_tma<MIXED, INV, MIXED, true> : k_eig3_fwd_aos_tma<MIXED, INV, MIXED, false>;
        int grid = grid_for(k, ntiles * kTile, kTile);
        k<<<grid, kTile, 0, st>>>((const float *)A, (uint32_t)ntiles, (float *)lam, (float *)D, (float *)ang, kase,
                                  resolve<float>(o), o.stats);
        kd_status s = launch_status();
        if (s != KD_OK) return s;
    }
    return run_fwd_aos<float, float, MIXED, INV, MIXED>(A, ntiles * kTile, n, lam, D, ang, kase, o, st);
}

kd_status launch_eig3_fwd_aos(const void *A, kd_dtype in_t, int64_t n, void *lam, void *D, void *ang,
                              uint8_t *kase, bool mixed, int inv, const kd_opts &o, cudaStream_t st) {
    if (in_t == KD_F64) return run_fwd_aos<double, double, false, INV_F32, false>(A, 0, n, lam, D, ang, kase, o, st);
    if (in_t == KD_F32) {
        if (!mixed) {
            if (inv == INV_F64) return run_fwd_aos<float, float, false, INV_F64, false>(A, 0, n, lam, D, ang, kase, o, st);
            if (inv == INV_FF) return run_fwd_aos<float, float, false, INV_FF, false>(A, 0, n, lam, D, ang, kase, o, st);
            return run_fwd_aos_f32<false, INV_F32>(A, n, lam, D, ang, kase, o, st);
        }
        if (inv == INV_F64) return run_fwd_aos_f32<true, INV_F64>(A, n, lam, D, ang, kase, o, st);
        if (inv == INV_FF) return run_fwd_aos_f32<true, INV_FF>(A, n, lam, D, ang, kase, o, st);
        return run_fwd_aos_f32<true, INV_F32>(A, n, lam, D, ang, kase, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv == INV_F64) return run_fwd_aos<uint16_t, float, true, INV_F64, true>(A, 0, n, lam, D, ang, kase, o, st);
        if (inv == INV_FF) return run_fwd_aos<uint16_t, float, true, INV_FF, true>(A, 0, n, lam, D, ang, kase, o, st);
        return run_fwd_aos<uint16_t, float, true, INV_F32, true>(A, 0, n, lam, D, ang, kase, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, bool ANG, bool FULL>
static void run_adj_aos_k(const void *A, int64_t n, const void *lb, const void *Db, const void *ab, void *Ab,
                          const kd_opts &o, cudaStream_t st) {
    auto k = k_eig3_adj_aos<TI, T, MIXED, INV, FAST, ANG, FULL>;
    const int grid = grid_for(k, n, kTile);
    k<<<grid, kTile, 0, st>>>((const TI *)A, n, (const T *)lb, (const T *)Db, (const T *)ab, (T *)Ab, resolve<T>(o),
                              tile_walk(n, kTile, grid));
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST>
static kd_status run_adj_aos(const void *A, int64_t n, const void *lb, const void *Db, const void *ab, void *Ab,
                             const kd_opts &o, cudaStream_t st) {
    const bool full = lb && Db;
    if (ab) {
        if (full) run_adj_aos_k<TI, T, MIXED, INV, FAST, true, true>(A, n, lb, Db, ab, Ab, o, st);
        else run_adj_aos_k<TI, T, MIXED, INV, FAST, true, false>(A, n, lb, Db, ab, Ab, o, st);
    } else {
        if (full) run_adj_aos_k<TI, T, MIXED, INV, FAST, false, true>(A, n, lb, Db, ab, Ab, o, st);
        else run_adj_aos_k<TI, T, MIXED, INV, FAST, false, false>(A, n, lb, Db, ab, Ab, o, st);
    }
    return launch_status();
}

kd_status launch_eig3_adj_aos(const void *A, kd_dtype in_t, int64_t n, const void *lam_bar, const void *D_bar,
                              const void *ang_bar, void *A_bar, bool mixed, int inv, const kd_opts &o,
                              cudaStream_t st) {
    if (in_t == KD_F64)
        return run_adj_aos<double, double, false, INV_F32, false>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
    if (in_t == KD_F32) {
        if (!mixed) {
            if (inv == INV_F64)
                return run_adj_aos<float, float, false, INV_F64, false>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
            if (inv == INV_FF)
                return run_adj_aos<float, float, false, INV_FF, false>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
            return run_adj_aos<float, float, false, INV_F32, false>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
        }
        if (inv == INV_F64)
            return run_adj_aos<float, float, true, INV_F64, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
        if (inv == INV_FF)
            return run_adj_aos<float, float, true, INV_FF, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_adj_aos<float, float, true, INV_F32, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv == INV_F64)
            return run_adj_aos<uint16_t, float, true, INV_F64, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
        if (inv == INV_FF)
            return run_adj_aos<uint16_t, float, true, INV_FF, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_adj_aos<uint16_t, float, true, INV_F32, true>(A, n, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

kd_status read_device_fault(unsigned int *code, bool clear) {
    unsigned int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return KD_ERR_LAUNCH;
    if (cudaMemcpyFromSymbol(&v, g_fault, sizeof(v)) != cudaSuccess) return KD_ERR_LAUNCH;
    if (clear) {
        const unsigned int zero = 0;
        if (cudaMemcpyToSymbol(g_fault, &zero, sizeof(zero)) != cudaSuccess) return KD_ERR_LAUNCH;
    }
    *code = v;
    return KD_OK;
}

kd_status launch_selftest_wait_timeout(unsigned int *flag, cudaStream_t st) {
    k_selftest_wait_timeout<<<1, 1, 0, st>>>(flag, 1000000ull);   // 1 ms
    return launch_status();
}

}  // namespace kd
