// Host-buffer pipeline of the 3x3 calls (kd_eig3_sym_host): the batch lives in host memory and
// is moved through the device chunk by chunk. Chunk c uses stream c mod nstreams and that
// stream's slice of the caller's workspace, so the host-to-device copies of one chunk, the
// kernels of another and the device-to-host copies of a third run at the same time on the copy
// engines and the SMs. Each plane group of a chunk moves with one strided 2-D copy (rows are the
// planes: host pitch n, device pitch chunk). Stream order alone makes a slice safe to reuse: the
// chunk that reuses it is queued behind the copies of the chunk that used it last.
#include "kd_internal.h"

using namespace kd;

namespace {

constexpr size_t kAlign = 256;

inline size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte sizes of one stream's slice: A (6 planes of the input type), then lam, D, ang, A_bar,
// lam_bar, D_bar, ang_bar (3 + 9 + 3 + 6 + 3 + 9 + 3 planes of the output type).
struct Slice {
    size_t a, out[7], total;
};
constexpr int kRows[7] = {3, 9, 3, 6, 3, 9, 3};

inline Slice slice_for(size_t in_sz, size_t out_sz, int64_t chunk) {
    Slice s;
    s.a = round_up(6 * in_sz * (size_t)chunk);
    s.total = s.a;
    for (int k = 0; k < 7; ++k) {
        s.out[k] = round_up(kRows[k] * out_sz * (size_t)chunk);
        s.total += s.out[k];
    }
    return s;
}

inline kd_dtype out_type_for(kd_dtype in_t) { return in_t == KD_F64 ? KD_F64 : KD_F32; }

inline bool valid_in_type(kd_dtype t) { return t == KD_F32 || t == KD_F64 || t == KD_BF16; }

// `rows` rows of `width` bytes between pitched buffers: one 2-D copy while both pitches are
// below 2^31 bytes (the copy engines' pitch limit), one copy per row beyond.
inline bool copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, int rows,
                      cudaMemcpyKind kind, cudaStream_t st) {
    const size_t lim = (size_t)1 << 31;
    if (dpitch < lim && spitch < lim)
        return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, st) == cudaSuccess;
    for (int r = 0; r < rows; ++r)
        if (cudaMemcpyAsync((char *)dst + r * dpitch, (const char *)src + r * spitch, width, kind, st) != cudaSuccess)
            return false;
    return true;
}

}  // namespace

extern "C" {

size_t kd_eig3_host_workspace_bytes(kd_dtype in_t, int64_t chunk, int nstreams) {
    if (!valid_in_type(in_t) || chunk <= 0 || nstreams <= 0 || nstreams > 16) return 0;
    return slice_for(dtype_size(in_t), dtype_size(out_type_for(in_t)), chunk).total * (size_t)nstreams;
}

kd_status kd_eig3_sym_host(const void *A_h, kd_dtype in_t, int64_t n, const void *lam_bar_h,
                           const void *D_bar_h, const void *ang_bar_h, void *lam_h, void *D_h, void *ang_h,
                           void *A_bar_h, int64_t chunk, void *workspace, size_t workspace_bytes,
                           const kd_opts *opts, void *const *streams, int nstreams) {
    if (n < 0 || chunk <= 0 || nstreams <= 0 || nstreams > 16 || !streams) return KD_ERR_INVALID_ARG;
    if (!valid_in_type(in_t)) return KD_ERR_UNSUPPORTED;
    const bool adj = lam_bar_h || D_bar_h || ang_bar_h;
    const bool fwd = lam_h || D_h || ang_h;
    if (n > 0 && !A_h) return KD_ERR_INVALID_ARG;
    if (adj != (A_bar_h != nullptr)) return KD_ERR_INVALID_ARG;
    const kd_dtype out_t = out_type_for(in_t);
    const size_t isz = dtype_size(in_t), osz = dtype_size(out_t);
    // Every dtype, form and option check of the two device calls, on an empty batch (returns
    // before any launch), so that nothing is queued for a call that would be rejected midway.
    kd_status s = kd_eig3_sym(A_h, in_t, 0, 0, nullptr, nullptr, nullptr, out_t, nullptr, opts, nullptr);
    if (s != KD_OK) return s;
    if (adj && (s = kd_eig3_sym_adjoint(A_h, in_t, 0, 0, nullptr, nullptr, nullptr, nullptr, opts, nullptr)) != KD_OK)
        return s;
    kd_opts o;
    if (opts) o = *opts;
    else kd_opts_default(&o);
    if (o.layout != KD_LAYOUT_SOA) return KD_ERR_UNSUPPORTED;
    const void *hin[4] = {A_h, lam_bar_h, D_bar_h, ang_bar_h};
    void *hout[4] = {lam_h, D_h, ang_h, A_bar_h};
    if (!aligned(A_h, isz)) return KD_ERR_MISALIGNED;
    for (int k = 1; k < 4; ++k)
        if (!aligned(hin[k], osz)) return KD_ERR_MISALIGNED;
    for (int k = 0; k < 4; ++k)
        if (!aligned(hout[k], osz)) return KD_ERR_MISALIGNED;
    if (n == 0 || !(fwd || adj)) return KD_OK;   // nothing requested: no copies
    if (!aligned(workspace, kAlign)) return KD_ERR_MISALIGNED;
    const int64_t m = chunk < n ? chunk : n;
    const Slice sl = slice_for(isz, osz, m);
    if (!workspace || workspace_bytes < sl.total * (size_t)nstreams) return KD_ERR_INVALID_ARG;
    int c = 0;
    if (cudaGetDeviceCount(&c) != cudaSuccess || c <= 0) return KD_ERR_NO_DEVICE;

    const size_t hp_in = (size_t)n * isz, hp_out = (size_t)n * osz;   // host pitches
    const size_t dp_in = (size_t)m * isz, dp_out = (size_t)m * osz;   // device pitches
    for (int64_t s0 = 0, ci = 0; s0 < n; s0 += m, ++ci) {
        const int64_t w = (n - s0) < m ? (n - s0) : m;
        const int si = (int)(ci % nstreams);
        cudaStream_t st = (cudaStream_t)streams[si];
        char *base = (char *)workspace + sl.total * (size_t)si;
        char *dA = base;
        char *dout[7];
        {
            char *p = base + sl.a;
            for (int k = 0; k < 7; ++k) { dout[k] = p; p += sl.out[k]; }
        }
        // inputs: A, then the cotangents that were given
        if (!copy_rows(dA, dp_in, (const char *)A_h + s0 * isz, hp_in, (size_t)w * isz, 6, cudaMemcpyHostToDevice,
                       st))
            return KD_ERR_LAUNCH;
        for (int k = 1; k < 4; ++k) {
            if (!hin[k]) continue;
            if (!copy_rows(dout[3 + k], dp_out, (const char *)hin[k] + s0 * osz, hp_out, (size_t)w * osz,
                           kRows[3 + k], cudaMemcpyHostToDevice, st))
                return KD_ERR_LAUNCH;
        }
        if (fwd) {
            s = kd_eig3_sym(dA, in_t, w, m, lam_h ? dout[0] : nullptr, D_h ? dout[1] : nullptr,
                            ang_h ? dout[2] : nullptr, out_t, nullptr, &o, st);
            if (s != KD_OK) return s;
        }
        if (adj) {
            s = kd_eig3_sym_adjoint(dA, in_t, w, m, lam_bar_h ? dout[4] : nullptr, D_bar_h ? dout[5] : nullptr,
                                    ang_bar_h ? dout[6] : nullptr, dout[3], &o, st);
            if (s != KD_OK) return s;
        }
        for (int k = 0; k < 4; ++k) {
            if (!hout[k]) continue;
            if (!copy_rows((char *)hout[k] + s0 * osz, hp_out, dout[k], dp_out, (size_t)w * osz, kRows[k],
                           cudaMemcpyDeviceToHost, st))
                return KD_ERR_LAUNCH;
        }
    }
    return KD_OK;
}

}  // extern "C"
