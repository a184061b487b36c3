// C-ABI of kdiag (declared in include/kdiag.h): argument validation, option defaults and
// dispatch to the kernels. Every check happens before any launch, so a rejected call has no
// effect on the device.
#include <cmath>

#include "kd_internal.h"

using namespace kd;

namespace {

inline kd_opts get_opts(const kd_opts *o) {
    kd_opts r;
    if (o) r = *o;
    else kd_opts_default(&r);
    return r;
}

inline bool all_aligned(size_t a, std::initializer_list<const void *> ps) {
    for (const void *p : ps)
        if (!aligned(p, a)) return false;
    return true;
}

inline bool have_device() {
    int c = 0;
    return cudaGetDeviceCount(&c) == cudaSuccess && c > 0;
}

// form for a 3x3 call: auto = mixed for FP32/BF16, plain for FP64; FP64 has only the plain form,
// BF16 only the mixed one
inline kd_status form_for(kd_dtype in_t, kd_dtype out_t, int form, bool &mixed) {
    if (in_t == KD_F64) {
        if (out_t != KD_F64 || form == KD_FORM_MIXED) return KD_ERR_UNSUPPORTED;
        mixed = false;
        return KD_OK;
    }
    if ((in_t == KD_F32 || in_t == KD_BF16) && out_t == KD_F32) {
        mixed = form != KD_FORM_PLAIN;
        if (in_t == KD_BF16 && !mixed) return KD_ERR_UNSUPPORTED;
        return KD_OK;
    }
    return KD_ERR_UNSUPPORTED;
}

}  // namespace

extern "C" {

void kd_opts_default(kd_opts *o) {
    if (!o) return;
    o->form = -1;
    o->invariants = KD_INV_F32;
    o->max_sweeps = 4;
    o->layout = KD_LAYOUT_SOA;
    o->degen_tau = 0.0;
    o->triple_tau = 0.0;
    o->conv_kappa = 0.0;
    o->gap_mask = -1.0;
    o->stats = nullptr;
}

const char *kd_status_string(kd_status s) {
    switch (s) {
        case KD_OK: return "ok";
        case KD_ERR_INVALID_ARG: return "invalid argument";
        case KD_ERR_MISALIGNED: return "misaligned pointer";
        case KD_ERR_UNSUPPORTED: return "unsupported dtype/form combination";
        case KD_ERR_LAUNCH: return "CUDA launch failed";
        case KD_ERR_NO_DEVICE: return "no CUDA device";
        case KD_ERR_TOO_LARGE: return "n exceeds the fixed scratch capacity of this entry point";
    }
    return "unknown status";
}

int kd_version(void) { return 200; }

kd_status kd_eig3_sym(const void *A, kd_dtype in_t, int64_t n, int64_t ld, void *lam, void *D,
                      void *ang, kd_dtype out_t, uint8_t *kase, const kd_opts *opts, void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    bool mixed = false;
    if ((s = form_for(in_t, out_t, o.form, mixed)) != KD_OK) return s;
    if (!aligned(A, dtype_size(in_t)) || !all_aligned(dtype_size(out_t), {lam, D, ang}))
        return KD_ERR_MISALIGNED;
    if (n == 0) return KD_OK;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    if (o.layout == KD_LAYOUT_AOS)
        return launch_eig3_fwd_aos(A, in_t, n, lam, D, ang, kase, mixed, o.invariants, o,
                                   (cudaStream_t)stream);
    return launch_eig3_fwd(A, in_t, n, ld, lam, D, ang, kase, mixed, o.invariants, o,
                           (cudaStream_t)stream);
}

kd_status kd_eig2_sym(const void *A, kd_dtype in_t, int64_t n, int64_t ld, void *lam, void *phi,
                      void *D, kd_dtype out_t, const kd_opts *opts, void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (in_t != out_t || (in_t != KD_F32 && in_t != KD_F64)) return KD_ERR_UNSUPPORTED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (!all_aligned(dtype_size(in_t), {A, lam, phi, D})) return KD_ERR_MISALIGNED;
    if (n == 0) return KD_OK;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    return launch_eig2_fwd(A, in_t, n, ld, lam, phi, D, o, (cudaStream_t)stream);
}

kd_status kd_eig3_sym_adjoint(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const void *lam_bar,
                              const void *D_bar, const void *ang_bar, void *A_bar, const kd_opts *opts,
                              void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (n > 0 && !A_bar) return KD_ERR_INVALID_ARG;
    const kd_dtype out_t = in_t == KD_F64 ? KD_F64 : KD_F32;
    bool mixed = false;
    if ((s = form_for(in_t, out_t, o.form, mixed)) != KD_OK) return s;
    if (!aligned(A, dtype_size(in_t)) || !all_aligned(dtype_size(out_t), {lam_bar, D_bar, ang_bar, A_bar}))
        return KD_ERR_MISALIGNED;
    if (n == 0) return KD_OK;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    if (o.layout == KD_LAYOUT_AOS)
        return launch_eig3_adj_aos(A, in_t, n, lam_bar, D_bar, ang_bar, A_bar, mixed, o.invariants, o,
                                   (cudaStream_t)stream);
    return launch_eig3_adj(A, in_t, n, ld, lam_bar, D_bar, ang_bar, A_bar, mixed, o.invariants, o,
                           (cudaStream_t)stream);
}

kd_status kd_eig2_sym_adjoint(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const void *lam_bar,
                              const void *phi_bar, void *A_bar, const kd_opts *opts, void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (n > 0 && !A_bar) return KD_ERR_INVALID_ARG;
    if (in_t != KD_F32 && in_t != KD_F64) return KD_ERR_UNSUPPORTED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (!all_aligned(dtype_size(in_t), {A, lam_bar, phi_bar, A_bar})) return KD_ERR_MISALIGNED;
    if (n == 0) return KD_OK;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    return launch_eig2_adj(A, in_t, n, ld, lam_bar, phi_bar, A_bar, o, (cudaStream_t)stream);
}

size_t kd_st_loss_workspace_bytes(int64_t n) {
    if (n <= 0 || !have_device()) return 0;
    return (size_t)st_loss_blocks(n) * 2 * sizeof(double);
}

kd_status kd_st_loss_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                         void *workspace, size_t workspace_bytes, double *loss, const kd_opts *opts,
                         void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (!w || !loss) return KD_ERR_INVALID_ARG;
    if (in_t != KD_F32 && in_t != KD_BF16) return KD_ERR_UNSUPPORTED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (!aligned(A, dtype_size(in_t)) || !aligned(loss, 8) || !aligned(workspace, 8)) return KD_ERR_MISALIGNED;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    if (n == 0) {
        // empty field: the sums are zero (written on the stream, no kernel over the data)
        if (cudaMemsetAsync(loss, 0, 2 * sizeof(double), (cudaStream_t)stream) != cudaSuccess) return KD_ERR_LAUNCH;
        return KD_OK;
    }
    const int blocks = st_loss_blocks(n);
    if (!workspace || workspace_bytes < (size_t)blocks * 2 * sizeof(double)) return KD_ERR_INVALID_ARG;
    return launch_st_fwd(A, in_t, n, ld, w, (double *)workspace, blocks, loss, o, (cudaStream_t)stream);
}

kd_status kd_st_loss_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                         void *A_bar, const kd_opts *opts, void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (!w || (n > 0 && !A_bar)) return KD_ERR_INVALID_ARG;
    if (in_t != KD_F32 && in_t != KD_BF16) return KD_ERR_UNSUPPORTED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (!all_aligned(dtype_size(in_t), {A, A_bar})) return KD_ERR_MISALIGNED;
    if (n == 0) return KD_OK;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    return launch_st_bwd(A, in_t, n, ld, w, scale, A_bar, o, (cudaStream_t)stream);
}

kd_status kd_st_loss_fwd_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                             void *workspace, size_t workspace_bytes, double *loss, void *A_bar,
                             const kd_opts *opts, void *stream) {
    const kd_opts o = get_opts(opts);
    kd_status s = check_common(A, n, ld);
    if (s != KD_OK) return s;
    if ((s = check_opts(o)) != KD_OK) return s;
    if (!w || !loss || (n > 0 && !A_bar)) return KD_ERR_INVALID_ARG;
    if (in_t != KD_F32 && in_t != KD_BF16) return KD_ERR_UNSUPPORTED;
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    if (!all_aligned(dtype_size(in_t), {A, A_bar}) || !aligned(loss, 8) || !aligned(workspace, 8))
        return KD_ERR_MISALIGNED;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    if (n == 0) {
        if (cudaMemsetAsync(loss, 0, 2 * sizeof(double), (cudaStream_t)stream) != cudaSuccess) return KD_ERR_LAUNCH;
        return KD_OK;
    }
    const int blocks = st_loss_blocks(n);
    if (!workspace || workspace_bytes < (size_t)blocks * 2 * sizeof(double)) return KD_ERR_INVALID_ARG;
    return launch_st_fwd_bwd(A, in_t, n, ld, w, scale, (double *)workspace, blocks, loss, A_bar, o,
                             (cudaStream_t)stream);
}

kd_status kd_device_fault(unsigned int *code, int clear) {
    if (!code) return KD_ERR_INVALID_ARG;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    return read_device_fault(code, clear != 0);
}

kd_status kd_selftest_wait_timeout(unsigned int *flag, void *stream) {
    if (!flag) return KD_ERR_INVALID_ARG;
    if (!aligned(flag, 4)) return KD_ERR_MISALIGNED;
    if (!have_device()) return KD_ERR_NO_DEVICE;
    return launch_selftest_wait_timeout(flag, (cudaStream_t)stream);
}

}  // extern "C"
