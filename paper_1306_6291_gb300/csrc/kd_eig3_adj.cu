// Batched 3x3 adjoint: packed gradient from eigenvalue, eigenvector and Euler-angle cotangents,
// recomputing each decomposition from A; one thread per matrix, over the SoA planes in tiles
// (TileWalk).
#include "kd_soa.cuh"

namespace kd {

// Cotangents lam_bar (3), D_bar (9), ang_bar (3) of matrix i into c[0..14] (0 for a null plane).
template <typename T, typename IT>
__device__ __forceinline__ void load_cot(const T *__restrict__ lam_bar, const T *__restrict__ D_bar,
                                         const T *__restrict__ ang_bar, IT ld, IT i, T c[15]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = lam_bar ? ld_as<T>(pl(lam_bar, ld, k, i)) : T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) c[3 + k] = D_bar ? ld_as<T>(pl(D_bar, ld, k, i)) : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[12 + k] = ang_bar ? ld_as<T>(pl(ang_bar, ld, k, i)) : T(0);
}

// The cotangents of a matrix are loaded at the top of its iteration and the next matrix's A
// before the decomposition, so that its latency overlaps the arithmetic. Staging everything in
// shared memory with cp.async, or prefetching the cotangents as well, measured slower (more
// instructions or more registers per matrix). Separate instantiations for calls with Euler-angle
// cotangents (ANG) and for calls with both lam_bar and D_bar given (FULL, loaded without null
// checks), so that the common calls carry no code for the absent ones.
template <typename T, typename IT, bool ANG, bool FULL>
__device__ __forceinline__ void adj_load_cot(const T *__restrict__ lam_bar, const T *__restrict__ D_bar,
                                             const T *__restrict__ ang_bar, IT ld, IT i, T c[15]) {
    if constexpr (FULL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) c[k] = ld_as<T>(pl(lam_bar, ld, k, i));
#pragma unroll
        for (int k = 0; k < 9; ++k) c[3 + k] = ld_as<T>(pl(D_bar, ld, k, i));
#pragma unroll
        for (int k = 0; k < 3; ++k) c[12 + k] = ANG ? ld_as<T>(pl(ang_bar, ld, k, i)) : T(0);
    } else {
        load_cot(lam_bar, D_bar, ANG ? ang_bar : nullptr, ld, i, c);
    }
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, bool ANG, bool FULL>
__global__ void __launch_bounds__(eig3_threads<T>(), 1)
k_eig3_adj(const TI *__restrict__ A, IT n, IT ld, const T *__restrict__ lam_bar,
           const T *__restrict__ D_bar, const T *__restrict__ ang_bar, T *__restrict__ A_bar, Params<T> P,
           TileWalk W) {
    uint32_t j = blockIdx.x;
    if (j >= W.T) return;
    const IT last = n - 1;
    uint32_t t = tile_first(W);
    IT i = (IT)t * blockDim.x + threadIdx.x;
    T a[6];
    load6(A, ld, i < last ? i : last, a);
    for (;;) {
        T c[15], out[6], b[6];
        adj_load_cot<T, IT, ANG, FULL>(lam_bar, D_bar, ang_bar, ld, i < last ? i : last, c);
        const uint32_t jn = j + gridDim.x;
        const bool more = jn < W.T;
        const uint32_t tn = tile_next(W, t);
        const IT inext = (IT)tn * blockDim.x + threadIdx.x;
        if (more) load6(A, ld, inext < last ? inext : last, b);
        Eig3<T> E;
        eig3_method<T, MIXED, INV, FAST>(a[0], a[1], a[2], a[3], a[4], a[5], P, E);
        eig3_adjoint(E, c, c + 3, ANG, c + 12, P.gap_mask, out);
        if (i < n) {
#pragma unroll
            for (int k = 0; k < 6; ++k) st(pl(A_bar, ld, k, i), out[k]);
        }
        if (!more) break;
        j = jn;
        t = tn;
        i = inext;
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = b[k];
    }
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, bool ANG, bool FULL>
static void run_eig3_adj_k(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db, const void *ab,
                           void *Ab, const kd_opts &o, cudaStream_t st) {
    auto k = k_eig3_adj<TI, T, MIXED, INV, FAST, IT, ANG, FULL>;
    const int grid = grid_for(k, n, eig3_threads<T>());
    k<<<grid, eig3_threads<T>(), 0, st>>>((const TI *)A, (IT)n, (IT)ld, (const T *)lb, (const T *)Db, (const T *)ab,
                                          (T *)Ab, resolve<T>(o), tile_walk(n, eig3_threads<T>(), grid));
}

template <typename TI, typename T, bool MIXED, int INV, bool FAST, typename IT, bool LEAN>
static void run_eig3_adj_it(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db, const void *ab,
                            void *Ab, const kd_opts &o, cudaStream_t st) {
    const bool full = lb && Db;
    if (ab) {
        if (full && !LEAN) run_eig3_adj_k<TI, T, MIXED, INV, FAST, IT, true, true>(A, n, ld, lb, Db, ab, Ab, o, st);
        else run_eig3_adj_k<TI, T, MIXED, INV, FAST, IT, true, false>(A, n, ld, lb, Db, ab, Ab, o, st);
    } else {
        if (full && !LEAN) run_eig3_adj_k<TI, T, MIXED, INV, FAST, IT, false, true>(A, n, ld, lb, Db, ab, Ab, o, st);
        else run_eig3_adj_k<TI, T, MIXED, INV, FAST, IT, false, false>(A, n, ld, lb, Db, ab, Ab, o, st);
    }
}

// LEAN: only the instantiations with run-time cotangent checks (the less common forms and modes)
template <typename TI, typename T, bool MIXED, int INV, bool FAST, bool LEAN = false>
static kd_status run_eig3_adj(const void *A, int64_t n, int64_t ld, const void *lb, const void *Db,
                              const void *ab, void *Ab, const kd_opts &o, cudaStream_t st) {
    if (small_index(ld)) run_eig3_adj_it<TI, T, MIXED, INV, FAST, uint32_t, LEAN>(A, n, ld, lb, Db, ab, Ab, o, st);
    else run_eig3_adj_it<TI, T, MIXED, INV, FAST, int64_t, LEAN>(A, n, ld, lb, Db, ab, Ab, o, st);
    return launch_status();
}

kd_status launch_eig3_adj(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const void *lam_bar,
                          const void *D_bar, const void *ang_bar, void *A_bar, bool mixed, int inv,
                          const kd_opts &o, cudaStream_t st) {
    if (in_t == KD_F64)
        return run_eig3_adj<double, double, false, INV_F32, false>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    if (in_t == KD_F32) {
        if (!mixed) {
            if (inv == INV_F64)
                return run_eig3_adj<float, float, false, INV_F64, false, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
            if (inv == INV_FF)
                return run_eig3_adj<float, float, false, INV_FF, false, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
            return run_eig3_adj<float, float, false, INV_F32, false>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        }
        if (inv == INV_F64)
            return run_eig3_adj<float, float, true, INV_F64, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        if (inv == INV_FF)
            return run_eig3_adj<float, float, true, INV_FF, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_eig3_adj<float, float, true, INV_F32, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    if (in_t == KD_BF16 && mixed) {
        if (inv == INV_F64)
            return run_eig3_adj<uint16_t, float, true, INV_F64, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        if (inv == INV_FF)
            return run_eig3_adj<uint16_t, float, true, INV_FF, true, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
        return run_eig3_adj<uint16_t, float, true, INV_F32, true>(A, n, ld, lam_bar, D_bar, ang_bar, A_bar, o, st);
    }
    return KD_ERR_UNSUPPORTED;
}

}  // namespace kd
