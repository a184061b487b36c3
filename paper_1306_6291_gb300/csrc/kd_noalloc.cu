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
#include "kd_internal.h"

namespace {

// Capacity: one pair of partial sums per block of the forward kernel. The kernel is grid-stride
// and runs the resident grid of the other loss entry points (one 1024-thread block per SM), far
// below this; the limit on n is the documented KD_ERR_TOO_LARGE bound of the entry point.
constexpr int kMaxBlocks = 8192;
constexpr int64_t kMaxN = (int64_t)kMaxBlocks * 16384;

// Every GPU that loads the library holds these 128 KiB until the process exits.
static __device__ __align__(256) double g_st_partials[2 * kMaxBlocks];

// Device address of g_st_partials in the context current on the calling thread. In host code the
// symbol's name is only a host-side stand-in, so the address must come from the runtime. It is
// looked up on every call and never cached: the address belongs to one context, and a cached
// value would go stale after cudaDeviceReset (which unloads the module) or be wrong for another
// context of the same device (a caller-created context made current with cuCtxSetCurrent). The
// lookup is a table search in the runtime, cheap next to a launch; the first lookup in a context
// loads the library's module there, which is why the first call should come before any capture.
kd_status scratch_for_current_context(double **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_st_partials) != cudaSuccess || !p) {
        cudaGetLastError();   // clear the (non-sticky) error, so that a later launch check does not see it
        return KD_ERR_LAUNCH;
    }
    *out = (double *)p;
    return KD_OK;
}

}  // namespace

extern "C" kd_status kd_st_loss_fwd_noalloc(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                                            const float w[3], double *loss, const kd_opts *opts,
                                            void *stream) {
    kd_opts o;
    if (opts) o = *opts;
    else kd_opts_default(&o);
    kd_status s = kd::check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = kd::check_opts(o)) != KD_OK) return s;
    if (!w || !loss) return KD_ERR_INVALID_ARG;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (in_t != KD_F32 && in_t != KD_BF16) return KD_ERR_UNSUPPORTED;
    if (!kd::aligned(A, kd::dtype_size(in_t)) || !kd::aligned(loss, 8)) return KD_ERR_MISALIGNED;
    if (n > kMaxN) return KD_ERR_TOO_LARGE;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) return KD_ERR_NO_DEVICE;
    double *partials = nullptr;
    if ((s = scratch_for_current_context(&partials)) != KD_OK) return s;
    if (n == 0) {
        if (cudaMemsetAsync(loss, 0, 2 * sizeof(double), (cudaStream_t)stream) != cudaSuccess) return KD_ERR_LAUNCH;
        return KD_OK;
    }
    // the resident grid of kd_st_loss_fwd (grid-stride kernel); never more blocks than the array holds
    const int blocks = kd::st_loss_blocks(n);
    if (blocks > kMaxBlocks) return KD_ERR_TOO_LARGE;
    return kd::launch_st_fwd(A, in_t, n, ld, w, partials, blocks, loss, o, (cudaStream_t)stream);
}
