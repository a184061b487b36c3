"""Python binding of the kdiag C-ABI (include/kdiag.h).

The ``kd_*`` functions have the C names and arguments (integers for pointers, ``kd_opts`` for
options) and only marshal them; every step of the computation runs in the CUDA library. The
tensor-level helpers (``eig3``, ``eig3_aos``, ``eig2``, ``eig3_adjoint``, ``eig3_adjoint_aos``,
``eig2_adjoint``, ``st_loss_fwd``, ``st_loss_bwd``, ``st_loss_fwd_bwd``, ``eig3_host``) and the
``torch.autograd.Function`` wrappers (``Eig3Fn``, ``Eig2Fn``, ``StLossFn``) allocate outputs with
PyTorch, pass device pointers and PyTorch's current stream (``eig3_host``: its own streams), and
raise ``KdError`` on any non-zero status. There is no CPU path: without the library (or without a
CUDA device) the calls raise.

Tensor layout: structure-of-arrays, a ``(k, n)`` tensor whose row j is plane j (see kdiag.h).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

KD_OK, KD_ERR_INVALID_ARG, KD_ERR_MISALIGNED, KD_ERR_UNSUPPORTED, KD_ERR_LAUNCH, KD_ERR_NO_DEVICE, KD_ERR_TOO_LARGE = range(7)
KD_F32, KD_F64, KD_BF16 = 0, 1, 2
KD_FORM_AUTO, KD_FORM_PLAIN, KD_FORM_MIXED = -1, 0, 1
KD_LAYOUT_SOA, KD_LAYOUT_AOS = 0, 1
KD_INV_F32, KD_INV_F64, KD_INV_FLOAT_FLOAT = 0, 1, 2
KASE_GENERAL, KASE_TWO_EQUAL, KASE_TRIPLE, KASE_NONFINITE = 0, 1, 2, 255
KASE_UNCONVERGED = 16   # added to the case when the refinement did not converge

EXPORTS = ("kd_opts_default", "kd_eig3_sym", "kd_eig2_sym", "kd_eig3_sym_adjoint", "kd_eig2_sym_adjoint",
           "kd_st_loss_workspace_bytes", "kd_st_loss_fwd", "kd_st_loss_bwd", "kd_st_loss_fwd_bwd",
           "kd_st_loss_fwd_noalloc", "kd_eig3_host_workspace_bytes", "kd_eig3_sym_host",
           "kd_device_fault", "kd_selftest_wait_timeout", "kd_status_string", "kd_version")


class KdError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: kdiag status {status} ({status_string(status)})")
        self.status = status


class kd_opts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("invariants", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("degen_tau", ctypes.c_double), ("triple_tau", ctypes.c_double),
                ("conv_kappa", ctypes.c_double), ("gap_mask", ctypes.c_double),
                ("stats", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libkdiag.so, building it first if it is missing or stale (nvcc required)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    O = ctypes.POINTER(kd_opts)
    lib.kd_opts_default.argtypes = [O]
    lib.kd_opts_default.restype = None
    lib.kd_eig3_sym.argtypes = [P, i32, i64, i64, P, P, P, i32, P, O, P]
    lib.kd_eig2_sym.argtypes = [P, i32, i64, i64, P, P, P, i32, O, P]
    lib.kd_eig3_sym_adjoint.argtypes = [P, i32, i64, i64, P, P, P, P, O, P]
    lib.kd_eig2_sym_adjoint.argtypes = [P, i32, i64, i64, P, P, P, O, P]
    lib.kd_st_loss_workspace_bytes.argtypes = [i64]
    lib.kd_st_loss_workspace_bytes.restype = ctypes.c_size_t
    lib.kd_st_loss_fwd.argtypes = [P, i32, i64, i64, ctypes.POINTER(ctypes.c_float), P, ctypes.c_size_t, P, O, P]
    lib.kd_st_loss_bwd.argtypes = [P, i32, i64, i64, ctypes.POINTER(ctypes.c_float), ctypes.c_float, P, O, P]
    lib.kd_st_loss_fwd_bwd.argtypes = [P, i32, i64, i64, ctypes.POINTER(ctypes.c_float), ctypes.c_float, P,
                                       ctypes.c_size_t, P, P, O, P]
    lib.kd_st_loss_fwd_bwd.restype = ctypes.c_int
    lib.kd_st_loss_fwd_noalloc.argtypes = [P, i32, i64, i64, ctypes.POINTER(ctypes.c_float), P, O, P]
    lib.kd_st_loss_fwd_noalloc.restype = ctypes.c_int
    lib.kd_eig3_host_workspace_bytes.argtypes = [i32, i64, ctypes.c_int]
    lib.kd_eig3_host_workspace_bytes.restype = ctypes.c_size_t
    lib.kd_eig3_sym_host.argtypes = [P, i32, i64, P, P, P, P, P, P, P, i64, P, ctypes.c_size_t, O,
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    lib.kd_eig3_sym_host.restype = ctypes.c_int
    lib.kd_device_fault.argtypes = [ctypes.POINTER(ctypes.c_uint), ctypes.c_int]
    lib.kd_device_fault.restype = ctypes.c_int
    lib.kd_selftest_wait_timeout.argtypes = [P, P]
    lib.kd_selftest_wait_timeout.restype = ctypes.c_int
    lib.kd_status_string.argtypes = [i32]
    lib.kd_status_string.restype = ctypes.c_char_p
    lib.kd_version.restype = ctypes.c_int
    for f in ("kd_eig3_sym", "kd_eig2_sym", "kd_eig3_sym_adjoint", "kd_eig2_sym_adjoint", "kd_st_loss_fwd",
              "kd_st_loss_bwd"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


# ---- C-named entry points (argument marshalling only) --------------------------------------

def kd_opts_default() -> kd_opts:
    o = kd_opts()
    load().kd_opts_default(ctypes.byref(o))
    return o


def kd_eig3_sym(A, in_t, n, ld, lam, D, ang, out_t, kase, opts, stream) -> int:
    return load().kd_eig3_sym(A, in_t, n, ld, lam, D, ang, out_t, kase, _optp(opts), stream)


def kd_eig2_sym(A, in_t, n, ld, lam, phi, D, out_t, opts, stream) -> int:
    return load().kd_eig2_sym(A, in_t, n, ld, lam, phi, D, out_t, _optp(opts), stream)


def kd_eig3_sym_adjoint(A, in_t, n, ld, lam_bar, D_bar, ang_bar, A_bar, opts, stream) -> int:
    return load().kd_eig3_sym_adjoint(A, in_t, n, ld, lam_bar, D_bar, ang_bar, A_bar, _optp(opts), stream)


def kd_eig2_sym_adjoint(A, in_t, n, ld, lam_bar, phi_bar, A_bar, opts, stream) -> int:
    return load().kd_eig2_sym_adjoint(A, in_t, n, ld, lam_bar, phi_bar, A_bar, _optp(opts), stream)


def kd_st_loss_workspace_bytes(n) -> int:
    return int(load().kd_st_loss_workspace_bytes(n))


def kd_st_loss_fwd(A, in_t, n, ld, w, workspace, workspace_bytes, loss, opts, stream) -> int:
    return load().kd_st_loss_fwd(A, in_t, n, ld, _w3(w), workspace, workspace_bytes, loss, _optp(opts), stream)


def kd_st_loss_bwd(A, in_t, n, ld, w, scale, A_bar, opts, stream) -> int:
    return load().kd_st_loss_bwd(A, in_t, n, ld, _w3(w), float(scale), A_bar, _optp(opts), stream)


def kd_st_loss_fwd_bwd(A, in_t, n, ld, w, scale, workspace, workspace_bytes, loss, A_bar, opts, stream) -> int:
    return load().kd_st_loss_fwd_bwd(A, in_t, n, ld, _w3(w), float(scale), workspace, workspace_bytes, loss, A_bar,
                                     _optp(opts), stream)


def kd_eig3_host_workspace_bytes(in_t, chunk, nstreams) -> int:
    return int(load().kd_eig3_host_workspace_bytes(in_t, chunk, nstreams))


def kd_eig3_sym_host(A_h, in_t, n, lam_bar_h, D_bar_h, ang_bar_h, lam_h, D_h, ang_h, A_bar_h, chunk, workspace,
                     workspace_bytes, opts, streams, nstreams) -> int:
    """streams: a sequence of stream handles (ints, None for the default stream) or None."""
    arr = None
    if streams is not None:
        arr = (ctypes.c_void_p * max(1, len(streams)))(*[s or None for s in streams])
    return load().kd_eig3_sym_host(A_h, in_t, n, lam_bar_h, D_bar_h, ang_bar_h, lam_h, D_h, ang_h, A_bar_h, chunk,
                                   workspace, workspace_bytes, _optp(opts), arr, nstreams)


def kd_st_loss_fwd_noalloc(A, in_t, n, ld, w, loss, opts, stream) -> int:
    """The structure-tensor loss forward with its scratch in the library's fixed device array
    (for callers that cannot allocate device memory; see kdiag.h)."""
    return load().kd_st_loss_fwd_noalloc(A, in_t, n, ld, _w3(w), loss, _optp(opts), stream)


def kd_device_fault(clear: bool = True):
    """(status, fault word) of the current device; bit 0 = a bounded TMA wait gave up."""
    v = ctypes.c_uint(0)
    st = load().kd_device_fault(ctypes.byref(v), int(bool(clear)))
    return st, int(v.value)


def kd_selftest_wait_timeout(flag, stream) -> int:
    return load().kd_selftest_wait_timeout(flag, stream)


def status_string(s: int) -> str:
    return load().kd_status_string(int(s)).decode()


def kd_version() -> int:
    return int(load().kd_version())


def _optp(o):
    return None if o is None else ctypes.byref(o)


def _w3(w):
    return (ctypes.c_float * 3)(*[float(x) for x in w])


# ---- tensor helpers ----------------------------------------------------------------------

_DT = {torch.float32: KD_F32, torch.float64: KD_F64, torch.bfloat16: KD_BF16}


def make_opts(form=KD_FORM_AUTO, invariants_f64=False, max_sweeps=None, degen_tau=None, triple_tau=None,
              conv_kappa=None, gap_mask=None, stats=None, layout=KD_LAYOUT_SOA, invariants=None) -> kd_opts:
    """kd_opts from keyword arguments; `invariants` is a KD_INV_* mode (invariants_f64=True is
    short for KD_INV_F64)."""
    o = kd_opts_default()
    o.form = int(form)
    o.layout = int(layout)
    if invariants is not None:
        o.invariants = int(invariants)
    elif invariants_f64:
        o.invariants = KD_INV_F64
    if max_sweeps is not None:
        o.max_sweeps = int(max_sweeps)
    if degen_tau is not None:
        o.degen_tau = float(degen_tau)
    if triple_tau is not None:
        o.triple_tau = float(triple_tau)
    if conv_kappa is not None:
        o.conv_kappa = float(conv_kappa)
    if gap_mask is not None:
        o.gap_mask = float(gap_mask)
    if stats is not None:
        if stats.dtype != torch.int64 or not stats.is_cuda or stats.numel() < 5:
            raise ValueError("stats must be a CUDA int64 tensor with 5 elements")
        o.stats = stats.data_ptr()
    return o


def _planes(A: torch.Tensor, k: int, name: str = "A") -> torch.Tensor:
    if A.dim() != 2 or A.shape[0] != k:
        raise ValueError(f"{name} must be a ({k}, n) tensor of planes, got {tuple(A.shape)}")
    if not A.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if A.dtype not in _DT:
        raise ValueError(f"{name}: unsupported dtype {A.dtype}")
    return A.contiguous()


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(dev):
    return torch.cuda.current_stream(dev).cuda_stream


def _check(status, where):
    if status != KD_OK:
        raise KdError(status, where)


def _out_dtype(t):
    return torch.float64 if t == torch.float64 else torch.float32


def eig3(A: torch.Tensor, opts: kd_opts | None = None, lam=True, D=True, ang=True, kase=False):
    """Diagonalize n packed 3x3 matrices A (6, n). Returns (lam (3, n), D (9, n), ang (3, n),
    kase (n,) uint8), with None for outputs not requested."""
    A = _planes(A, 6)
    n = A.shape[1]
    odt = _out_dtype(A.dtype)
    outs = [torch.empty(k, n, device=A.device, dtype=odt) if want else None
            for k, want in ((3, lam), (9, D), (3, ang))]
    ks = torch.empty(n, device=A.device, dtype=torch.uint8) if kase else None
    with torch.cuda.device(A.device):
        st = kd_eig3_sym(A.data_ptr(), _DT[A.dtype], n, n, _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2]),
                         _DT[odt], _ptr(ks), opts, _stream(A.device))
    _check(st, "kd_eig3_sym")
    return outs[0], outs[1], outs[2], ks


def _aos_opts(opts):
    o = kd_opts_default() if opts is None else kd_opts.from_buffer_copy(opts)
    o.layout = KD_LAYOUT_AOS
    return o


def eig3_aos(A: torch.Tensor, opts: kd_opts | None = None, lam=True, D=True, ang=True, kase=False):
    """Array-of-structures variant of eig3: A is (n, 6) (rows A11, A22, A33, A12, A13, A23); returns
    lam (n, 3), D (n, 9) (row-major 3x3 per row), ang (n, 3), kase (n,)."""
    if A.dim() != 2 or A.shape[1] != 6:
        raise ValueError(f"A must be (n, 6) rows, got {tuple(A.shape)}")
    if not A.is_cuda or A.dtype not in _DT:
        raise ValueError("A must be a CUDA float32, float64 or bfloat16 tensor")
    A = A.contiguous()
    n = A.shape[0]
    odt = _out_dtype(A.dtype)
    outs = [torch.empty(n, k, device=A.device, dtype=odt) if want else None for k, want in ((3, lam), (9, D), (3, ang))]
    ks = torch.empty(n, device=A.device, dtype=torch.uint8) if kase else None
    with torch.cuda.device(A.device):
        st = kd_eig3_sym(A.data_ptr(), _DT[A.dtype], n, n, _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2]), _DT[odt],
                         _ptr(ks), _aos_opts(opts), _stream(A.device))
    _check(st, "kd_eig3_sym (AoS)")
    return outs[0], outs[1], outs[2], ks


def eig3_adjoint_aos(A: torch.Tensor, lam_bar=None, D_bar=None, ang_bar=None, opts: kd_opts | None = None):
    """Array-of-structures variant of eig3_adjoint: A (n, 6), lam_bar (n, 3), D_bar (n, 9),
    ang_bar (n, 3) -> A_bar (n, 6)."""
    A = A.contiguous()
    n = A.shape[0]
    odt = _out_dtype(A.dtype)
    cts = [None if t is None else t.to(odt).contiguous() for t in (lam_bar, D_bar, ang_bar)]
    out = torch.empty(n, 6, device=A.device, dtype=odt)
    with torch.cuda.device(A.device):
        st = kd_eig3_sym_adjoint(A.data_ptr(), _DT[A.dtype], n, n, _ptr(cts[0]), _ptr(cts[1]), _ptr(cts[2]),
                                 out.data_ptr(), _aos_opts(opts), _stream(A.device))
    _check(st, "kd_eig3_sym_adjoint (AoS)")
    return out


def eig2(A: torch.Tensor, opts: kd_opts | None = None, lam=True, phi=True, D=False):
    """Diagonalize n packed 2x2 matrices A (3, n). Returns (lam (2, n), phi (n,), D (4, n))."""
    A = _planes(A, 3)
    if A.dtype == torch.bfloat16:
        raise ValueError("eig2 takes float32 or float64")
    n = A.shape[1]
    l = torch.empty(2, n, device=A.device, dtype=A.dtype) if lam else None
    p = torch.empty(n, device=A.device, dtype=A.dtype) if phi else None
    d = torch.empty(4, n, device=A.device, dtype=A.dtype) if D else None
    with torch.cuda.device(A.device):
        st = kd_eig2_sym(A.data_ptr(), _DT[A.dtype], n, n, _ptr(l), _ptr(p), _ptr(d), _DT[A.dtype], opts,
                         _stream(A.device))
    _check(st, "kd_eig2_sym")
    return l, p, d


def eig3_adjoint(A: torch.Tensor, lam_bar=None, D_bar=None, opts: kd_opts | None = None,
                 ang_bar=None) -> torch.Tensor:
    """Packed gradient (6, n) for cotangents lam_bar (3, n), D_bar (9, n) and ang_bar (3, n) of
    eig3's outputs (any may be None)."""
    A = _planes(A, 6)
    n = A.shape[1]
    odt = _out_dtype(A.dtype)
    lb = None if lam_bar is None else lam_bar.to(odt).contiguous()
    Db = None if D_bar is None else D_bar.to(odt).contiguous()
    ab = None if ang_bar is None else ang_bar.to(odt).contiguous()
    for t, k, nm in ((lb, 3, "lam_bar"), (Db, 9, "D_bar"), (ab, 3, "ang_bar")):
        if t is not None and tuple(t.shape) != (k, n):
            raise ValueError(f"{nm} must be ({k}, {n})")
    out = torch.empty(6, n, device=A.device, dtype=odt)
    with torch.cuda.device(A.device):
        st = kd_eig3_sym_adjoint(A.data_ptr(), _DT[A.dtype], n, n, _ptr(lb), _ptr(Db), _ptr(ab), out.data_ptr(),
                                 opts, _stream(A.device))
    _check(st, "kd_eig3_sym_adjoint")
    return out


def eig2_adjoint(A: torch.Tensor, lam_bar=None, phi_bar=None, opts: kd_opts | None = None) -> torch.Tensor:
    A = _planes(A, 3)
    n = A.shape[1]
    lb = None if lam_bar is None else lam_bar.to(A.dtype).contiguous()
    pb = None if phi_bar is None else phi_bar.to(A.dtype).contiguous()
    out = torch.empty(3, n, device=A.device, dtype=A.dtype)
    with torch.cuda.device(A.device):
        st = kd_eig2_sym_adjoint(A.data_ptr(), _DT[A.dtype], n, n, _ptr(lb), _ptr(pb), out.data_ptr(), opts,
                                 _stream(A.device))
    _check(st, "kd_eig2_sym_adjoint")
    return out


def st_loss_workspace(n: int, device) -> torch.Tensor:
    with torch.cuda.device(device):
        nb = kd_st_loss_workspace_bytes(n)
    return torch.empty(max(nb, 16) // 8, device=device, dtype=torch.float64)


def st_loss_fwd(A: torch.Tensor, w, workspace: torch.Tensor | None = None, opts: kd_opts | None = None,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """The two sums (2,) float64 of the structure-tensor loss of A (6, n) (BF16 or FP32)."""
    A = _planes(A, 6)
    n = A.shape[1]
    ws = workspace if workspace is not None else st_loss_workspace(n, A.device)
    loss = out if out is not None else torch.empty(2, device=A.device, dtype=torch.float64)
    with torch.cuda.device(A.device):
        st = kd_st_loss_fwd(A.data_ptr(), _DT[A.dtype], n, n, w, ws.data_ptr(), ws.numel() * 8, loss.data_ptr(),
                            opts, _stream(A.device))
    _check(st, "kd_st_loss_fwd")
    return loss


def st_loss_bwd(A: torch.Tensor, w, scale: float = 1.0, opts: kd_opts | None = None,
                out: torch.Tensor | None = None) -> torch.Tensor:
    A = _planes(A, 6)
    n = A.shape[1]
    g = out if out is not None else torch.empty_like(A)
    with torch.cuda.device(A.device):
        st = kd_st_loss_bwd(A.data_ptr(), _DT[A.dtype], n, n, w, scale, g.data_ptr(), opts, _stream(A.device))
    _check(st, "kd_st_loss_bwd")
    return g


def st_loss_fwd_bwd(A: torch.Tensor, w, scale: float = 1.0, workspace: torch.Tensor | None = None,
                    opts: kd_opts | None = None):
    """Loss sums (2,) float64 and scale * dL/dA (dtype of A) in one pass."""
    A = _planes(A, 6)
    n = A.shape[1]
    ws = workspace if workspace is not None else st_loss_workspace(n, A.device)
    loss = torch.empty(2, device=A.device, dtype=torch.float64)
    g = torch.empty_like(A)
    with torch.cuda.device(A.device):
        st = kd_st_loss_fwd_bwd(A.data_ptr(), _DT[A.dtype], n, n, w, scale, ws.data_ptr(), ws.numel() * 8,
                                loss.data_ptr(), g.data_ptr(), opts, _stream(A.device))
    _check(st, "kd_st_loss_fwd_bwd")
    return loss, g


# ---- host buffers, pipelined ------------------------------------------------------------------

def eig3_host(A: torch.Tensor, lam_bar=None, D_bar=None, ang_bar=None, opts: kd_opts | None = None,
              outputs=("lam", "D", "ang"), chunk: int = 1 << 20, streams: int = 3, device="cuda",
              workspace: torch.Tensor | None = None, out: dict | None = None):
    """3x3 forward (and the adjoint when cotangents are given) for HOST (6, n) planes, ideally in
    pinned memory, through kd_eig3_sym_host: chunks rotate over `streams` CUDA streams so that
    host-to-device copies, kernels and device-to-host copies of different chunks overlap. Returns
    a dict of host tensors: 'lam' (3, n), 'D' (9, n), 'ang' (3, n) as requested, and 'A_bar'
    (6, n) when any cotangent is given. `workspace` (device, from eig3_host_workspace) and `out`
    (host tensors of those shapes) may be passed in to reuse them across calls."""
    if A.is_cuda or A.dim() != 2 or A.shape[0] != 6:
        raise ValueError("A must be a host (6, n) tensor")
    A = A.contiguous()
    dev = torch.device(device)
    n = A.shape[1]
    odt = _out_dtype(A.dtype)
    pin = A.is_pinned()
    rows = {"lam": 3, "D": 9, "ang": 3, "A_bar": 6}
    cts = {k: v for k, v in (("lam_bar", lam_bar), ("D_bar", D_bar), ("ang_bar", ang_bar)) if v is not None}
    for k, v in cts.items():
        if v.is_cuda or v.dtype != odt or not v.is_contiguous() or v.shape[1] != n:
            raise ValueError(f"{k} must be a contiguous host tensor of dtype {odt} with n columns")
    names = list(outputs) + (["A_bar"] if cts else [])
    outs = dict(out) if out is not None else {}
    for k in names:
        if k not in outs:
            outs[k] = torch.empty(rows[k], n, dtype=odt, pin_memory=pin)
    m = max(1, min(chunk, n))
    nst = max(1, streams)
    with torch.cuda.device(dev):
        ws = workspace if workspace is not None else eig3_host_workspace(A.dtype, m, nst, dev)
        sts = [torch.cuda.Stream(dev) for _ in range(nst)]
        cur = torch.cuda.current_stream(dev)
        for st in sts:
            st.wait_stream(cur)
        st = kd_eig3_sym_host(A.data_ptr(), _DT[A.dtype], n, _ptr(cts.get("lam_bar")), _ptr(cts.get("D_bar")),
                              _ptr(cts.get("ang_bar")), _ptr(outs.get("lam")), _ptr(outs.get("D")),
                              _ptr(outs.get("ang")), _ptr(outs.get("A_bar")), m, ws.data_ptr(), ws.numel(), opts,
                              [x.cuda_stream for x in sts], nst)
        _check(st, "kd_eig3_sym_host")
        for x in sts:
            cur.wait_stream(x)
        cur.synchronize()
    return {k: outs[k] for k in names}


def eig3_host_workspace(dtype: torch.dtype, chunk: int, streams: int = 3, device="cuda") -> torch.Tensor:
    """Device workspace (uint8) for eig3_host / kd_eig3_sym_host with this chunk and stream count."""
    nb = kd_eig3_host_workspace_bytes(_DT[dtype], chunk, streams)
    if nb == 0:
        raise ValueError("invalid dtype, chunk or stream count")
    return torch.empty(nb, dtype=torch.uint8, device=device)


# ---- autograd ----------------------------------------------------------------------------

class Eig3Fn(torch.autograd.Function):
    """(lam, D, ang) = Eig3Fn.apply(A, opts): A (6, n) packed; backward through
    kd_eig3_sym_adjoint, which recomputes the decomposition from A."""

    @staticmethod
    def forward(ctx, A, opts=None):
        lam, D, ang, _ = eig3(A, opts)
        ctx.save_for_backward(A)
        ctx.opts = opts
        return lam, D, ang

    @staticmethod
    def backward(ctx, lam_bar, D_bar, ang_bar):
        (A,) = ctx.saved_tensors
        g = eig3_adjoint(A, lam_bar, D_bar, ctx.opts, ang_bar=ang_bar)
        return g.to(A.dtype), None


class Eig2Fn(torch.autograd.Function):
    """(lam, phi) = Eig2Fn.apply(A, opts) for A (3, n); backward through kd_eig2_sym_adjoint."""

    @staticmethod
    def forward(ctx, A, opts=None):
        lam, phi, _ = eig2(A, opts)
        ctx.save_for_backward(A)
        ctx.opts = opts
        return lam, phi

    @staticmethod
    def backward(ctx, lam_bar, phi_bar):
        (A,) = ctx.saved_tensors
        return eig2_adjoint(A, lam_bar, phi_bar, ctx.opts), None


class StLossFn(torch.autograd.Function):
    """loss = StLossFn.apply(A, w, opts): the scalar sum of both terms of the structure-tensor
    loss (float64). When A needs a gradient the forward runs the fused kernel (each tensor
    decomposed once) and keeps dL/dA for the backward, which only scales it."""

    @staticmethod
    def forward(ctx, A, w, opts=None):
        if A.requires_grad:
            parts, g = st_loss_fwd_bwd(A, w, 1.0, opts=opts)
            ctx.save_for_backward(g)
        else:
            parts = st_loss_fwd(A, w, opts=opts)
        return parts.sum()

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return g * gout.to(g.dtype), None, None
