// Shared pieces of the SoA (structure-of-arrays) kernels: streaming loads and stores, the
// per-category counters, plane access of the 3x3 inputs, launch-shape constants. Planes are read
// and written once with evict-first cache hints, since every byte is touched exactly once.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "kd_internal.h"


namespace kd {

// Threads per block of the 3x3 kernels: the FP32 ones run one block of 1024 threads per SM (up to
// 64 registers per thread, 32 warps), so that each SM works through 1024 consecutive matrices of
// every plane at a time; measured faster than 4-6 resident blocks of 256 at the same or higher
// occupancy (forward 76% -> 77%, adjoint 78% -> 79% of the HBM roofline on the precision
// workload, 68% -> 73% and 71% -> 76% on N(0,1) matrices). The FP64 ones (more than 64 registers
// per thread, bound by the FP64 pipe) use blocks of 64: on 65,536 matrices 256-thread blocks left
// 104 SMs with two blocks and 48 with one; 64-thread blocks spread the batch evenly (forward
// 0.070 ms against 0.077 ms, adjoint 0.064 against 0.071; no change at 2^24).
template <typename T> constexpr int eig3_threads() { return sizeof(T) == 4 ? 1024 : 64; }

// ---- loads / stores --------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T ld_as(const float *p) { return (T)__ldcs(p); }
template <typename T> __device__ __forceinline__ T ld_as(const double *p) { return (T)__ldcs(p); }
template <typename T> __device__ __forceinline__ T ld_as(const uint16_t *p) {
    return (T)__uint_as_float(((uint32_t)__ldcs((const unsigned short *)p)) << 16);
}
__device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st(double *p, double v) { __stcs(p, v); }

// Per-category counters, one atomic per warp and category: stats[0..3] count the matrices of
// each case (general, two equal, three equal, non-finite) from a kase code, stats[4] those whose
// refinement did not converge (code bit 16; those are also counted under their case).
__device__ __forceinline__ void count_kase(unsigned long long *stats, int code) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    const int base = code == 255 ? 255 : (code & 15);
    const bool unconv = code != 255 && (code & 16) != 0;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const unsigned b = __ballot_sync(mask, c < 4 ? base == (c < 3 ? c : 255) : unconv);
        if (b && lane == leader) atomicAdd(stats + c, (unsigned long long)__popc(b));
    }
}

// Element i of plane k of a SoA array A (plane stride ld elements): the plane's base, the same
// for every thread, plus the element's byte offset. The 3x3 kernels take 32-bit element offsets
// only where i < 429,496,729 (small_index), so that the byte offset i * sizeof(P) fits 32 bits
// as well for elements of up to 8 bytes, and the access can use the uniform-base +
// 32-bit-offset address form: no 64-bit address arithmetic per access. Measured against
// (A + i) + k * ld: 1-2% faster 3x3 kernels (adjoint 502 instead of 508 slots per matrix); the
// loss kernels measured 1% slower with it and keep their per-array base.
template <typename P, typename IT>
__device__ __forceinline__ P *pl(P *A, IT ld, int k, IT i) {
    P *base = A + (size_t)k * (size_t)ld;
    if constexpr (sizeof(IT) == 4) {
        using B = typename std::conditional<std::is_const<P>::value, const char, char>::type;
        return reinterpret_cast<P *>(reinterpret_cast<B *>(base) + (uint32_t)i * (uint32_t)sizeof(P));
    } else {
        return base + i;
    }
}

// The six input planes of matrix i.
template <typename T, typename TI, typename IT>
__device__ __forceinline__ void load6(const TI *__restrict__ A, IT ld, IT i, T a[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = ld_as<T>(pl(A, ld, k, i));
}

// 32-bit offsets cover every plane (at most 9 per array) when 10 * ld < 2^32.
inline bool small_index(int64_t ld) { return ld < (int64_t)429496729; }

// Order in which the 3x3 kernels visit a batch. The batch is cut into T tiles of blockDim
// consecutive matrices (one per thread; the last tile may be partial); block b takes the tiles
// perm(b), perm(b + G), perm(b + 2G), ... (G blocks) with perm(j) = j M mod T, gcd(M, T) = 1 and M
// near 0.618 T, so that at any time the SMs work on tiles spread over the whole batch rather than
// on one window of G tiles. Where the cost per matrix varies along the batch (runs of easy and of
// hard matrices, as in the four groups of the precision workload) the memory-bound and the
// issue-bound stretches overlap across the SMs instead of following one another. t0 = M mod T is
// block 0's step to block 1's first tile and step = G M mod T the step from one tile of a block to
// its next. In the partial tile the threads past the end compute on the last matrix (their loads
// are clamped to it) and store nothing, so every matrix goes through the same instructions
// whatever its position in the batch. Measured on the precision workload (2^24): forward 0.259 ms
// against 0.269 ms in the plain grid-stride order, adjoint 0.290 ms against 0.294 ms; on a batch
// of uniformly hard matrices the walk's bookkeeping costs about 10 instruction slots per matrix
// (1-2%).
struct TileWalk {
    uint32_t T, t0, step;
};

inline TileWalk tile_walk(int64_t n, int threads, int grid) {
    TileWalk w;
    const int64_t T = (n + threads - 1) / threads;
    w.T = (uint32_t)(T > 0 ? T : 1);
    auto gcd = [](uint64_t a, uint64_t b) {
        while (b) { const uint64_t t = a % b; a = b; b = t; }
        return a;
    };
    uint64_t M = ((uint64_t)(0.6180339887498949 * (double)w.T)) | 1u;
    while (gcd(M, w.T) != 1) M += 2;
    w.t0 = (uint32_t)(M % w.T);
    w.step = (uint32_t)(((uint64_t)grid * M) % w.T);
    return w;
}

// First tile of this block and the advance to the next one (device side of TileWalk).
__device__ __forceinline__ uint32_t tile_first(const TileWalk &w) {
    return (uint32_t)(((uint64_t)blockIdx.x * w.t0) % w.T);
}
__device__ __forceinline__ uint32_t tile_next(const TileWalk &w, uint32_t t) {
    const uint32_t u = t + w.step;
    return u >= w.T ? u - w.T : u;
}

}  // namespace kd
