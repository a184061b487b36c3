// Host-side helpers shared by the kdiag translation units (argument checks, launch shape,
// option resolution). Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "kdiag.h"
#include "kd_method.cuh"

namespace kd {

constexpr int kThreads = 256;

// Grid for a grid-stride kernel over n items: enough resident blocks to fill every SM (as the
// occupancy calculator reports for this kernel), never more blocks than items need.
template <typename K>
inline int grid_for(K kernel, int64_t n, int threads = kThreads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (sms <= 0) sms = 1;
    if (per_sm <= 0) per_sm = 1;
    int64_t need = (n + threads - 1) / threads;
    int64_t full = (int64_t)sms * per_sm;
    int64_t g = need < full ? need : full;
    return (int)(g < 1 ? 1 : g);
}

inline bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline size_t dtype_size(kd_dtype t) {
    switch (t) {
        case KD_F32: return 4;
        case KD_F64: return 8;
        case KD_BF16: return 2;
    }
    return 0;
}

// Argument checks shared by every entry point: n >= 0, ld >= n, a non-null A when n > 0.
inline kd_status check_common(const void *A, int64_t n, int64_t ld) {
    if (n < 0 || ld < n) return KD_ERR_INVALID_ARG;
    if (n > 0 && !A) return KD_ERR_INVALID_ARG;
    return KD_OK;
}

// Option checks shared by every entry point (value ranges of kdiag.h, finite thresholds, an
// 8-byte aligned stats pointer).
inline kd_status check_opts(const kd_opts &o) {
    if (o.form < -1 || o.form > 1) return KD_ERR_INVALID_ARG;
    if (o.max_sweeps < 0 || o.max_sweeps > 8) return KD_ERR_INVALID_ARG;
    if (o.invariants < KD_INV_F32 || o.invariants > KD_INV_FLOAT_FLOAT) return KD_ERR_INVALID_ARG;
    if (o.layout != KD_LAYOUT_SOA && o.layout != KD_LAYOUT_AOS) return KD_ERR_INVALID_ARG;
    if (!std::isfinite(o.degen_tau) || !std::isfinite(o.triple_tau) || !std::isfinite(o.conv_kappa) ||
        !std::isfinite(o.gap_mask))
        return KD_ERR_INVALID_ARG;
    if (!aligned(o.stats, 8)) return KD_ERR_MISALIGNED;
    return KD_OK;
}

inline kd_status launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KD_OK : KD_ERR_LAUNCH;
}

// Resolve the options for an arithmetic type (defaults documented in kdiag.h).
template <typename T>
inline Params<T> resolve(const kd_opts &o) {
    const bool f32 = sizeof(T) == 4;
    Params<T> P;
    P.tau2 = (T)(o.degen_tau > 0 ? o.degen_tau : (f32 ? 3e-3 : 5e-6));
    P.tau3 = (T)(o.triple_tau > 0 ? o.triple_tau : (f32 ? 1e-6 : 1e-12));
    P.kappa = (T)(o.conv_kappa > 0 ? o.conv_kappa : 3e-7);
    P.gap_mask = (T)(o.gap_mask >= 0 ? o.gap_mask : (f32 ? 1e-6 : 1e-12));
    P.max_sweeps = o.max_sweeps;
    return P;
}

}  // namespace kd

namespace kd {

// Launchers, one per entry point; arguments already validated by the C-ABI layer.
kd_status launch_eig3_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, void *lam, void *D,
                          void *ang, uint8_t *kase, bool mixed, int inv, const kd_opts &o,
                          cudaStream_t st);
kd_status launch_eig3_adj(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const void *lam_bar,
                          const void *D_bar, const void *ang_bar, void *A_bar, bool mixed, int inv,
                          const kd_opts &o, cudaStream_t st);
kd_status launch_eig2_fwd(const void *A, kd_dtype t, int64_t n, int64_t ld, void *lam, void *phi,
                          void *D, const kd_opts &o, cudaStream_t st);
kd_status launch_eig2_adj(const void *A, kd_dtype t, int64_t n, int64_t ld, const void *lam_bar,
                          const void *phi_bar, void *A_bar, const kd_opts &o, cudaStream_t st);
kd_status launch_eig3_fwd_aos(const void *A, kd_dtype in_t, int64_t n, void *lam, void *D, void *ang,
                              uint8_t *kase, bool mixed, int inv, const kd_opts &o, cudaStream_t st);
kd_status launch_eig3_adj_aos(const void *A, kd_dtype in_t, int64_t n, const void *lam_bar, const void *D_bar,
                              const void *ang_bar, void *A_bar, bool mixed, int inv, const kd_opts &o,
                              cudaStream_t st);
kd_status read_device_fault(unsigned int *code, bool clear);
kd_status launch_selftest_wait_timeout(unsigned int *flag, cudaStream_t st);
int st_loss_blocks(int64_t n);
kd_status launch_st_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        double *partials, int blocks, double *loss, const kd_opts &o, cudaStream_t st);
kd_status launch_st_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                        float scale, void *A_bar, const kd_opts &o, cudaStream_t st);
kd_status launch_st_fwd_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                            double *partials, int blocks, double *loss, void *A_bar, const kd_opts &o,
                            cudaStream_t st);

}  // namespace kd
