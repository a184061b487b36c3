// Shared pieces of the SoA (structure-of-arrays) kernels: streaming loads and stores, the
// per-category counters, plane access of the 3x3 inputs, launch-shape constants. Planes are read
// and written once with evict-first cache hints, since every byte is touched exactly once.
#pragma once

#include <cuda_bf16.h>

#include "kd_internal.h"


namespace kd {

// Threads per block of the 3x3 kernels: the FP32 ones run one block of 1024 threads per SM (up to
// 64 registers per thread, 32 warps), so that each SM works through 1024 consecutive matrices of
// every plane at a time; measured faster than 4-6 resident blocks of 256 at the same or higher
// occupancy (forward 76% -> 77%, adjoint 78% -> 79% of the HBM roofline on the precision
// workload, 68% -> 73% and 71% -> 76% on N(0,1) matrices). The FP64 ones use 256 (they need more
// registers per thread than 64).
template <typename T> constexpr int eig3_threads() { return sizeof(T) == 4 ? 1024 : 256; }

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

// The six input planes of matrix i.
template <typename T, typename TI, typename IT>
__device__ __forceinline__ void load6(const TI *__restrict__ A, IT ld, IT i, T a[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = ld_as<T>(A + i + k * ld);
}

// 32-bit offsets cover every plane (at most 9 per array) when 10 * ld < 2^32.
inline bool small_index(int64_t ld) { return ld < (int64_t)429496729; }

}  // namespace kd
