// Batched 3x3 forward (Sections 4-6 and Eq. (6.5)): eigenvalues, D and Euler angles of each
// matrix, one thread per matrix, over the SoA planes in tiles (TileWalk).
#include "kd_soa.cuh"

namespace kd {

// IT is the element-offset type: 32-bit when every plane offset fits, else 64-bit. The batch is
// visited tile by tile in the scrambled order of TileWalk (one matrix per thread and tile); each
// thread loads its matrix of the next tile before working on the current one, so the load
// latency overlaps the arithmetic. OUT: 0 checks every output pointer at run time; otherwise it
// is the set of outputs requested (OUT_LAM | OUT_D | OUT_ANG) of a call without kase or counters,
// an instantiation without run-time output checks (for the common requests).
constexpr int OUT_LAM = 1, OUT_D = 2, OUT_ANG = 4;

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, int OUT>
__global__ void __launch_bounds__(eig3_threads<T>(), 1)
k_eig3_fwd(const TI *__restrict__ A, IT n, IT ld, T *__restrict__ lam, T *__restrict__ D,
           T *__restrict__ ang, uint8_t *__restrict__ kase, Params<T> P, unsigned long long *stats,
           TileWalk W) {
    constexpr bool FIXED = OUT != 0;
    uint32_t j = blockIdx.x;
    if (j >= W.T) return;
    const IT last = n - 1;
    uint32_t t = tile_first(W);
    IT i = (IT)t * blockDim.x + threadIdx.x;
    T a[6];
    load6(A, ld, i < last ? i : last, a);
    for (;;) {
        const uint32_t jn = j + gridDim.x;
        const bool more = jn < W.T;
        const uint32_t tn = tile_next(W, t);
        const IT inext = (IT)tn * blockDim.x + threadIdx.x;
        T b[6];
        if (more) load6(A, ld, inext < last ? inext : last, b);
        Eig3<T> E;
        eig3_method<T, MIXED, INV, FAST>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
        if (i < n) {
            if (FIXED ? (OUT & OUT_LAM) != 0 : lam != nullptr) {
#pragma unroll
                for (int k = 0; k < 3; ++k) st(pl(lam, ld, k, i), E.lam[k] * E.inv_s);
            }
            if (FIXED ? (OUT & OUT_D) != 0 : D != nullptr) {
#pragma unroll
                for (int k = 0; k < 9; ++k) st(pl(D, ld, k, i), E.D[k]);
            }
            if (FIXED ? (OUT & OUT_ANG) != 0 : ang != nullptr) {
                T g[3];
                euler_from_D<T, FAST>(E.D, g);
                if (E.kase == 255) g[0] = g[1] = g[2] = E.lam[0];   // NaN
#pragma unroll
                for (int k = 0; k < 3; ++k) st(pl(ang, ld, k, i), g[k]);
            }
            if (!FIXED && kase) kase[i] = (uint8_t)kase_code(E);
            if (!FIXED && stats) count_kase(stats, kase_code(E));
        }
        if (!more) break;
        j = jn;
        t = tn;
        i = inext;
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = b[k];
    }
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, int OUT>
static void run_eig3_fwd_k(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang, uint8_t *kase,
                           const kd_opts &o, cudaStream_t st) {
    auto k = k_eig3_fwd<TI, T, MIXED, INV, FAST, IT, OUT>;
    const int grid = grid_for(k, n, eig3_threads<T>());
    k<<<grid, eig3_threads<T>(), 0, st>>>((const TI *)A, (IT)n, (IT)ld, (T *)lam, (T *)D, (T *)ang, kase, resolve<T>(o),
                                          o.stats, tile_walk(n, eig3_threads<T>(), grid));
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, bool LEAN>
static void run_eig3_fwd_it(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang, uint8_t *kase,
                            const kd_opts &o, cudaStream_t st) {
    const int set = (lam ? OUT_LAM : 0) | (D ? OUT_D : 0) | (ang ? OUT_ANG : 0);
    const bool plain = !kase && !o.stats;
    if (!LEAN && plain && set == (OUT_LAM | OUT_D | OUT_ANG))
        run_eig3_fwd_k<TI, T, MIXED, INV, FAST, IT, OUT_LAM | OUT_D | OUT_ANG>(A, n, ld, lam, D, ang, kase, o, st);
    else if (!LEAN && plain && set == (OUT_LAM | OUT_ANG))
        run_eig3_fwd_k<TI, T, MIXED, INV, FAST, IT, OUT_LAM | OUT_ANG>(A, n, ld, lam, D, ang, kase, o, st);
    else if (!LEAN && plain && set == (OUT_LAM | OUT_D))
        run_eig3_fwd_k<TI, T, MIXED, INV, FAST, IT, OUT_LAM | OUT_D>(A, n, ld, lam, D, ang, kase, o, st);
    else
        run_eig3_fwd_k<TI, T, MIXED, INV, FAST, IT, 0>(A, n, ld, lam, D, ang, kase, o, st);
}

// LEAN: only the instantiation with run-time output checks (for the less common forms and modes,
// to bound the build time)
template <typename TI, typename T, bool MIXED, int INV, bool FAST, bool LEAN = false>
static kd_status run_eig3_fwd(const void *A, int64_t n, int64_t ld, void *lam, void *D, void *ang,
                              uint8_t *kase, const kd_opts &o, cudaStream_t st) {
    if (small_index(ld)) run_eig3_fwd_it<TI, T, MIXED, INV, FAST, uint32_t, LEAN>(A, n, ld, lam, D, ang, kase, o, st);
    else run_eig3_fwd_it<TI, T, MIXED, INV, FAST, int64_t, LEAN>(A, n, ld, lam, D, ang, kase, o, st);
    return launch_status();
}

kd_status launch_eig3_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, void *lam, void *D,
                          void *ang, uint8_t *kase, bool mixed, int inv, const kd_opts &o,
                          cudaStream_t st) {
    if (in_t == KD_F64) return run_eig3_fwd<double, double, false, INV_F32, false>(A, n, ld, lam, D, ang, kase, o, st);
    if (in_t == KD_F32) {
        if (!mixed) {
            if (inv == INV_F64) return run_eig3_fwd<float, float, false, INV_F64, false, true>(A, n, ld, lam, D, ang, kase, o, st);
            if (inv == INV_FF) return run_eig3_fwd<float, float, false, INV_FF, false, true>(A, n, ld, lam, D, ang, kase, o, st);
            return run_eig3_fwd<float, float, false, INV_F32, false>(A, n, ld, lam, D, ang, kase, o, st);
        }
        if (inv == INV_F64) return run_eig3_fwd<float, float, true, INV_F64, true>(A, n, ld, lam, D, ang, kase, o, st);
        if (inv == INV_FF) return run_eig3_fwd<float, float, true, INV_FF, true>(A, n, ld, lam, D, ang, kase, o, st);
        return run_eig3_fwd<float, float, true, INV_F32, true>(A, n, ld, lam, D, ang, kase, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv == INV_F64) return run_eig3_fwd<uint16_t, float, true, INV_F64, true>(A, n, ld, lam, D, ang, kase, o, st);
        if (inv == INV_FF) return run_eig3_fwd<uint16_t, float, true, INV_FF, true, true>(A, n, ld, lam, D, ang, kase, o, st);
        return run_eig3_fwd<uint16_t, float, true, INV_F32, true>(A, n, ld, lam, D, ang, kase, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

}  // namespace kd
