// kd_st_loss_fwd_noalloc: the structure-tensor loss forward without a caller-supplied workspace.
//
// Some callers cannot call cudaMalloc at all: plugins living inside a host application that owns
// every byte of device memory, and latency-critical loops in which cudaMalloc's implicit device
// synchronisation is not allowed. This entry point serves them: its per-block partial sums live
// in a fixed file-scope device array, so the call allocates nothing.
//
// The array is shared by every call on a device and keeps the contents of the last call. The
// forward kernel overwrites every partial it later reads, so nothing has to be cleared, but two
// calls that overlap on the GPU (different streams, no ordering between them) race on it.
#include <cmath>
#include <mutex>

#include "kd_internal.h"

namespace {

// Capacity: one pair of partial sums per block, one block per KD_ST_NOALLOC_CHUNK tensors.
constexpr int kMaxBlocks = 8192;
constexpr int64_t kChunk = 16384;   // tensors per block (16 per thread of a 1024-thread block)

// Every GPU that loads the library holds these 128 KiB until the process exits.
static __device__ __align__(256) double g_st_partials[2 * kMaxBlocks];

// Device address of g_st_partials per device ordinal, found once per device. In host code the
// symbol's name is only a host-side stand-in, so the address must come from the runtime.
std::mutex g_mu;
double *g_addr[64] = {nullptr};

kd_status scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KD_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_st_partials) != cudaSuccess || !p) return KD_ERR_LAUNCH;
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return KD_OK;
}

}  // namespace

extern "C" kd_status kd_st_loss_fwd_noalloc(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                                            const float w[3], double *loss, const kd_opts *opts,
                                            void *stream) {
    kd_opts o;
    if (opts) o = *opts;
    else kd_opts_default(&o);
    if (n < 0 || ld < n || (n > 0 && !A) || !w || !loss) return KD_ERR_INVALID_ARG;
    // the option checks of the other entry points
    if (o.form < -1 || o.form > 1 || o.max_sweeps < 0 || o.max_sweeps > 8 ||
        (o.invariants_f64 != 0 && o.invariants_f64 != 1) ||
        (o.layout != KD_LAYOUT_SOA && o.layout != KD_LAYOUT_AOS) || !std::isfinite(o.degen_tau) ||
        !std::isfinite(o.triple_tau) || !std::isfinite(o.conv_kappa) || !std::isfinite(o.gap_mask))
        return KD_ERR_INVALID_ARG;
    if (!kd::aligned(o.stats, 8)) return KD_ERR_MISALIGNED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (in_t != KD_F32 && in_t != KD_BF16) return KD_ERR_UNSUPPORTED;
    if (!kd::aligned(A, kd::dtype_size(in_t)) || !kd::aligned(loss, 8)) return KD_ERR_MISALIGNED;
    if (n > (int64_t)kMaxBlocks * kChunk) return KD_ERR_TOO_LARGE;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) return KD_ERR_NO_DEVICE;
    double *partials = nullptr;
    kd_status s = scratch_for_current_device(&partials);
    if (s != KD_OK) return s;
    if (n == 0) {
        if (cudaMemsetAsync(loss, 0, 2 * sizeof(double), (cudaStream_t)stream) != cudaSuccess) return KD_ERR_LAUNCH;
        return KD_OK;
    }
    const int blocks = (int)((n + kChunk - 1) / kChunk);
    return kd::launch_st_fwd(A, in_t, n, ld, w, partials, blocks, loss, o, (cudaStream_t)stream);
}
