/*
 * kdiag — batched closed-form diagonalization of real symmetric 2x2 and 3x3 matrices on NVIDIA
 * GB300 (sm_103a), after M.J. Kronenburg, "A Method for Fast Diagonalization of a 2x2 or 3x3 Real
 * Symmetric Matrix" (arXiv:1306.6291).
 *
 * The method (paper, Sections 2-6): A = D . Lambda . D^T (Eq. (2.1)) with D a rotation. For 2x2,
 * D = R(phi) (Eq. (2.5)); lam1, lam2 and phi come from Eqs. (3.2), (3.3), (3.5). For 3x3,
 * D = R1(phi1) R2(phi2) R3(phi3) (Eqs. (2.6)-(2.9)); the eigenvalues are the trigonometric roots of
 * the characteristic cubic (Eqs. (4.2)-(4.12)); the angles are solved from A = D Lambda D^T
 * (Eqs. (5.1)-(5.15), special cases Eqs. (5.20)-(5.25)); (phi1, phi2, phi3) are also the Euler
 * angles of the intrinsic X-Y'-Z'' sequence (Eq. (6.5)).
 *
 * CONVENTIONS (every entry point)
 *  - All array pointers are DEVICE pointers owned by the caller (except the host arrays of
 *    kd_eig3_sym_host). The library never allocates or frees memory and never synchronises
 *    (except kd_device_fault, which reads the fault word); every call is asynchronous on `stream`
 *    (a cudaStream_t passed as void*, NULL = the legacy default stream).
 *  - Layout (kd_opts.layout). Structure of arrays (KD_LAYOUT_SOA, the default): an array with k
 *    components is k planes of n elements, plane j starting at element j*ld of the pointer
 *    (ld >= n, counted in elements of that array's dtype); one `ld` serves every array of a call.
 *    Array of structures (KD_LAYOUT_AOS, 3x3 forward and adjoint): matrix i's k components are
 *    elements k*i .. k*i+k-1 (records of 6 for A and A_bar, 3 for lam and angles, 9 for D); `ld`
 *    must be >= n and is otherwise unused. FP32 AoS batches with 16-byte aligned arrays move
 *    through shared memory by TMA bulk copies.
 *      3x3 input A      6 planes (A11, A22, A33, A12, A13, A23)      (packed upper triangle)
 *      2x2 input A      3 planes (A11, A22, A12)
 *      lam              3 planes (3x3) / 2 planes (2x2), the paper's labels:
 *                       3x3 general case lam1 >= lam3 >= lam2 (Eqs. (4.10)-(4.12));
 *                       two equal eigenvalues: lam1, lam2 the pair, lam3 the distinct one (Eq. (5.20));
 *                       2x2: lam1 the eigenvalue of (cos phi, sin phi) (Section 3 sign rule)
 *      D                9 planes, row-major D_ij at plane 3i+j (3x3); 4 planes D11,D12,D21,D22 (2x2);
 *                       column k is the unit eigenvector of lam_k, det D = +1
 *      ang              3 planes (phi1, phi2, phi3); phi (2x2) 1 plane
 *      kase (optional)  n bytes (not planar): 0 general, 1 two equal eigenvalues, 2 three equal,
 *                       255 non-finite input; 16 is added (16, 17, 18) when the precision form's
 *                       refinement stopped with an off-diagonal of D^T A D still above
 *                       conv_kappa * ||A||_F (max_sweeps sweeps ran out, or max_sweeps = 0)
 *  - A NULL output pointer means "do not compute/write that output".
 *  - Packed gradients: the packed off-diagonal A12 stands for both A12 and A21, so its gradient is
 *    dL/dA12 + dL/dA21 of the full matrix; diagonal entries get dL/dAii.
 *  - n == 0 returns KD_OK without launching. Arguments are validated before any launch; a bad
 *    argument returns an error code and launches nothing. The kernels never trap: a non-finite
 *    input matrix gives NaN outputs and kase 255.
 *  - Memory and stream ordering are the caller's: inputs must be ready on `stream`.
 */
#ifndef KDIAG_H
#define KDIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kd_status {
    KD_OK = 0,
    KD_ERR_INVALID_ARG = 1,   /* null required pointer, n < 0, ld < n, bad option value */
    KD_ERR_MISALIGNED = 2,    /* a pointer not aligned to its element size */
    KD_ERR_UNSUPPORTED = 3,   /* dtype / form combination not provided */
    KD_ERR_LAUNCH = 4,        /* the CUDA launch failed (cudaGetLastError() was non-zero) */
    KD_ERR_NO_DEVICE = 5,     /* no CUDA device visible */
    KD_ERR_TOO_LARGE = 6      /* n beyond the fixed scratch capacity of kd_st_loss_fwd_noalloc */
} kd_status;

typedef enum kd_dtype { KD_F32 = 0, KD_F64 = 1, KD_BF16 = 2 } kd_dtype;

typedef enum kd_layout { KD_LAYOUT_SOA = 0, KD_LAYOUT_AOS = 1 } kd_layout;

typedef enum kd_form {
    /* The paper's formulas, arithmetic in the output dtype, no refinement. */
    KD_FORM_PLAIN = 0,
    /* FP32 precision form: the paper's formulas in FP32 with an exact power-of-two prescale and
       the shift by tr(A)/3 formed from exact differences, followed by Jacobi refinement of
       B = D^T A D (eigenvalues = Rayleigh quotients B_kk). Invariants: kd_opts.invariants. */
    KD_FORM_MIXED = 1
} kd_form;

/* Where the FP32 and BF16 3x3 forms (plain and mixed) evaluate the invariants p', q' of the
   shifted matrix B = A - (tr A / 3) I and the discriminant N = p'^3 - q'^2 of the cubic
   (Eqs. (4.5)-(4.9)), whose cancellation on nearly degenerate spectra costs accuracy:
   KD_INV_F32 in FP32 from the exact diagonal differences (the default); KD_INV_F64 in FP64
   arithmetic; KD_INV_FLOAT_FLOAT in compensated float-float arithmetic (each value a pair of
   FP32 numbers, products and sums through error-free transformations; p', q' and N of the
   exact-difference matrix 3B), FP32 instructions only. The FP64 form ignores the field. */
typedef enum kd_invariants { KD_INV_F32 = 0, KD_INV_F64 = 1, KD_INV_FLOAT_FLOAT = 2 } kd_invariants;

/* Options. Initialise with kd_opts_default(); a NULL kd_opts* means the defaults. A NaN or
   infinite threshold (degen_tau, triple_tau, conv_kappa, gap_mask) is KD_ERR_INVALID_ARG. */
typedef struct kd_opts {
    int32_t form;            /* kd_form, or -1 (the default) = KD_FORM_MIXED for FP32/BF16 input
                                and KD_FORM_PLAIN for FP64 input */
    int32_t invariants;      /* kd_invariants (default KD_INV_F32); other values are
                                KD_ERR_INVALID_ARG */
    int32_t max_sweeps;      /* mixed form: maximum refinement sweeps, 0..8 (default 4) */
    int32_t layout;          /* kd_layout (default KD_LAYOUT_SOA) */
    double degen_tau;        /* two eigenvalues are equal when their difference is <= degen_tau *
                                (lam_max - lam_min); <= 0 selects the default (3e-3 FP32, 5e-6 FP64) */
    double triple_tau;       /* three are equal when lam_max - lam_min <= triple_tau * ||A||_F;
                                <= 0 selects the default (1e-6 FP32, 1e-12 FP64) */
    double conv_kappa;       /* refinement stops when every off-diagonal of D^T A D is
                                <= conv_kappa * ||A||_F; <= 0 selects 3e-7 */
    double gap_mask;         /* adjoints: 1/(lam_k - lam_j) terms are dropped where
                                |lam_k - lam_j| <= gap_mask * ||A||_F; < 0 selects 1e-6 (FP32) /
                                1e-12 (FP64) */
    unsigned long long *stats; /* optional DEVICE counters [5], incremented per matrix by the
                                  forward calls: [0] general, [1] two equal, [2] three equal,
                                  [3] non-finite input, [4] refinement not converged (the
                                  matrix is also counted in [0]-[2]); NULL = off */
} kd_opts;

/* Fill *o with the defaults. */
void kd_opts_default(kd_opts *o);

/*
 * 3x3 forward. Computes, per matrix, the eigenvalues (Section 4), the rotation D = R1 R2 R3
 * (Eq. (2.6), angles from Section 5) and the Euler angles (Eq. (6.5)).
 * Supported: in_t = out_t = KD_F64 (plain form); in_t = KD_F32 or KD_BF16 with out_t = KD_F32
 * (plain or mixed form). Angles: phi2 in [-pi/2, pi/2], phi1 and phi3 in (-pi, pi]. At gimbal
 * lock (cos(phi2)^2 below 2^-100 in FP32, 2^-900 in FP64, where phi2 = +-pi/2 to working precision)
 * only phi1 +- phi3 is determined: phi1 = 0 is returned and phi3 carries the rotation, so
 * R1 R2 R3(angles) = D still holds.
 */
kd_status kd_eig3_sym(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                      void *lam, void *D, void *ang, kd_dtype out_t, uint8_t *kase,
                      const kd_opts *opts, void *stream);

/*
 * 2x2 forward, Section 3: lam1, lam2 (Eqs. (3.2)-(3.3), sign(0) = +1), phi = (1/2) arctan(2 A12 /
 * (A11 - A22)) (Eq. (3.5)) in [-pi/4, pi/4], phi = 0 for A11 = A22, A12 = 0; optional D = R(phi).
 * Supported: in_t = out_t = KD_F32 or KD_F64. `opts` is accepted for symmetry (stats only).
 */
kd_status kd_eig2_sym(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                      void *lam, void *phi, void *D, kd_dtype out_t,
                      const kd_opts *opts, void *stream);

/*
 * 3x3 adjoint: given cotangents lam_bar (3 planes), D_bar (9 planes) and ang_bar (3 planes) of
 * the outputs of kd_eig3_sym with the same options, writes the packed gradient A_bar (6 planes,
 * same dtype as the forward outputs: F32 for F32/BF16 input, F64 for F64 input). The
 * decomposition is recomputed from A (D is not read). A_bar = D (diag(lam_bar) + F o M) D^T,
 * F_jk = 1/(lam_k - lam_j) masked where |lam_k - lam_j| <= gap_mask ||A||_F, M = D^T D_bar plus the
 * angle terms: with D = R1 R2 R3 (Eq. (6.5)), D^T dD = [omega]x, omega = M_phi dphi,
 * M_phi = [[c2 c3, s3, 0], [-c2 s3, c3, 0], [s2, 0, 1]]; mu = M_phi^-T ang_bar is added to M at
 * (2,1), (0,2), (1,0) (0-based). The 1/cos(phi2) part is dropped where cos(phi2) <= gap_mask
 * (gimbal lock). Any cotangent may be NULL (treated as zero).
 */
kd_status kd_eig3_sym_adjoint(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                              const void *lam_bar, const void *D_bar, const void *ang_bar,
                              void *A_bar, const kd_opts *opts, void *stream);

/*
 * 2x2 adjoint of (lam1, lam2, phi) of kd_eig2_sym: packed gradient (3 planes, dtype of A) from
 * d lam1 = c^2 dA11 + s^2 dA22 + 2cs dA12, d lam2 = s^2 dA11 + c^2 dA22 - 2cs dA12,
 * d phi = (cos 2phi dA12 - cs (dA11 - dA22)) / (lam1 - lam2) (the phi term masked by gap_mask).
 * lam_bar (2 planes) or phi_bar (1 plane) may be NULL.
 */
kd_status kd_eig2_sym_adjoint(const void *A, kd_dtype in_t, int64_t n, int64_t ld,
                              const void *lam_bar, const void *phi_bar, void *A_bar,
                              const kd_opts *opts, void *stream);

/*
 * Structure-tensor loss over a field of n 3x3 tensors (in_t KD_BF16 or KD_F32, compute FP32):
 *     L = sum_i (lam_max - lam_min)^2 + sum_i (v_max . w)^2,
 * v_max the unit eigenvector of the largest eigenvalue, w a fixed 3-vector (host array).
 * kd_st_loss_fwd writes the two sums to loss[0], loss[1] (DEVICE doubles). It needs a DEVICE
 * workspace of kd_st_loss_workspace_bytes(n) bytes (per-block partial sums, fully overwritten by
 * each call; no clearing needed). Deterministic: the same input gives bit-identical sums.
 * kd_st_loss_bwd writes A_bar = scale * dL/dA (packed, dtype of A): the eigenvalue term gives
 * 2(lam_max - lam_min)(v_max v_max^T - v_min v_min^T), the alignment term
 * 2(v_max . w) sum_{j != max} (v_j . w) / (lam_max - lam_j) sym(v_j v_max^T) (masked by gap_mask).
 */
size_t kd_st_loss_workspace_bytes(int64_t n);
/* Forward and backward in one pass (each tensor decomposed once): the two sums to loss[0..1] and
 * A_bar = scale * dL/dA, with the workspace of kd_st_loss_fwd. */
kd_status kd_st_loss_fwd_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3], float scale,
                             void *workspace, size_t workspace_bytes, double *loss, void *A_bar,
                             const kd_opts *opts, void *stream);
kd_status kd_st_loss_fwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                         void *workspace, size_t workspace_bytes, double *loss,
                         const kd_opts *opts, void *stream);
kd_status kd_st_loss_bwd(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                         float scale, void *A_bar, const kd_opts *opts, void *stream);

/*
 * kd_st_loss_fwd_noalloc: kd_st_loss_fwd for callers that cannot call cudaMalloc, such as
 * plugins inside a host application that owns all device memory, or latency-critical loops where
 * cudaMalloc's implicit device synchronisation is not allowed. It takes no workspace and
 * allocates nothing: the per-block partial sums live in a fixed 128 KiB device array inside the
 * library (held on every GPU that loads the library until the process exits). The paper has no
 * counterpart of this entry point; it only changes where the forward's scratch lives.
 *  - n may be at most 134,217,728 (8192 blocks x 16384 tensors); larger n returns
 *    KD_ERR_TOO_LARGE and launches nothing.
 *  - Every call looks up the array's device address in the context current on the calling
 *    thread (cudaGetSymbolAddress; nothing is cached, so a call after cudaDeviceReset, or from
 *    another context of the same device, finds the address valid there). The first call in a
 *    context loads the library's device code into it: make that first call before any stream
 *    capture.
 *  - Every call on a device shares the array. The kernel overwrites each partial it reads, so
 *    nothing needs clearing between calls, but calls that overlap on the GPU race on it: order
 *    them on one stream (or with events).
 * Same arguments, checks and results (up to summation order) as kd_st_loss_fwd otherwise.
 */
kd_status kd_st_loss_fwd_noalloc(const void *A, kd_dtype in_t, int64_t n, int64_t ld, const float w[3],
                                 double *loss, const kd_opts *opts, void *stream);

/*
 * kd_eig3_sym_host: kd_eig3_sym and kd_eig3_sym_adjoint over a batch that lives in HOST memory.
 * Moving the batch between host and device is not part of the paper's method; this entry point
 * only streams it through the device. The batch is cut into chunks of `chunk` matrices; chunk c
 * goes to streams[c % nstreams] and that stream's slice of `workspace`: one strided copy per
 * plane group to the device, the forward (when any of lam_h, D_h, ang_h is given), the adjoint
 * (when any cotangent is given), one strided copy per output back. Chunks on different streams
 * overlap (copies in both directions and kernels at once).
 *  - A_h: (6, n) planes in host memory, plane k at A_h + k*n elements, dtype in_t (F32, BF16, F64).
 *  - lam_bar_h (3, n), D_bar_h (9, n), ang_bar_h (3, n): host cotangents or NULL; A_bar_h (6, n)
 *    receives the packed gradient and must be given exactly when some cotangent is.
 *  - lam_h (3, n), D_h (9, n), ang_h (3, n): host outputs or NULL. With no output and no
 *    cotangent at all (or n = 0) the call returns KD_OK after its checks, copying nothing.
 *    Cotangents and outputs are F64 for F64 input, else F32, all with row pitch n.
 *  - workspace: DEVICE memory of at least kd_eig3_host_workspace_bytes(in_t, min(chunk, n),
 *    nstreams) bytes, 256-byte aligned, owned by the caller.
 *  - streams: nstreams (1..16) CUDA streams owned by the caller (a NULL entry is the legacy
 *    default stream).
 * Host memory should be page-locked (cudaHostAlloc / cudaHostRegister): with pageable memory the
 * copies are staged by the driver and lose their overlap. The call only enqueues work and returns;
 * the outputs are ready once every stream has been synchronized. Option, dtype and alignment
 * checks are those of kd_eig3_sym / kd_eig3_sym_adjoint (SoA layout only) and all happen before
 * anything is enqueued; KD_ERR_LAUNCH means a copy or launch failed midway (earlier chunks may
 * have been enqueued).
 */
size_t kd_eig3_host_workspace_bytes(kd_dtype in_t, int64_t chunk, int nstreams);
kd_status kd_eig3_sym_host(const void *A_h, kd_dtype in_t, int64_t n, const void *lam_bar_h,
                           const void *D_bar_h, const void *ang_bar_h, void *lam_h, void *D_h, void *ang_h,
                           void *A_bar_h, int64_t chunk, void *workspace, size_t workspace_bytes,
                           const kd_opts *opts, void *const *streams, int nstreams);

/*
 * Device fault word of the library on the current device: bit 0 is set when a kernel gave up on a
 * bounded wait for a TMA transfer (after 2 s) and returned early, leaving that call's outputs
 * incomplete. Synchronises the device, writes the word to *code and clears it if `clear` != 0.
 */
kd_status kd_device_fault(unsigned int *code, int clear);

/*
 * Self-test of the bounded waits: one thread arms a shared-memory barrier for a transfer that
 * is never issued and waits with a 1 ms limit. Writes 1 to the DEVICE word *flag when the wait
 * gave up as designed (2 if it completed, which would be a bug). Asynchronous on `stream`.
 */
kd_status kd_selftest_wait_timeout(unsigned int *flag, void *stream);

/* Human-readable text for a status code (static storage). */
const char *kd_status_string(kd_status s);

/* Library version, major*10000 + minor*100 + patch. */
int kd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KDIAG_H */
