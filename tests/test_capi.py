"""Host-side checks of the C-ABI: the library builds for sm_103a, loads, exports every function
include/kdiag.h declares, and rejects bad arguments before touching a device. No kernel runs."""
import ctypes
import os
import re

import pytest

from paper_1306_6291_gb300 import kdiag as K

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kdiag.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kd_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = K.load()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(K.EXPORTS)


def test_header_documents_the_counters_and_the_kase_codes():
    """The stats array has five counters (the fifth: refinement not converged) and the kase
    output adds 16 for a refinement that did not converge; the binding agrees."""
    text = open(HEADER).read()
    assert "DEVICE counters [5]" in text and "[4] refinement not converged" in text
    assert "16 is added (16, 17, 18)" in text
    assert K.KASE_UNCONVERGED == 16


def test_version_status_strings_and_defaults():
    assert K.kd_version() == 200
    assert K.status_string(0) == "ok"
    assert "misaligned" in K.status_string(2)
    o = K.kd_opts_default()
    assert (o.form, o.invariants, o.max_sweeps, o.layout, o.gap_mask, o.stats) == (-1, 0, 4, 0, -1.0, None)


# pointers below are never dereferenced: every call is rejected (or is empty) before a launch
@pytest.mark.parametrize("args,expect", [
    ((None, K.KD_F32, -1, 0, None, None, None, K.KD_F32, None, None, None), K.KD_ERR_INVALID_ARG),
    ((None, K.KD_F32, 0, 0, None, None, None, K.KD_F32, None, None, None), K.KD_OK),
    ((None, K.KD_F32, 5, 5, None, None, None, K.KD_F32, None, None, None), K.KD_ERR_INVALID_ARG),
    ((64, K.KD_F32, 10, 9, None, None, None, K.KD_F32, None, None, None), K.KD_ERR_INVALID_ARG),
    ((64, K.KD_F64, 10, 10, None, None, None, K.KD_F32, None, None, None), K.KD_ERR_UNSUPPORTED),
    ((64, K.KD_F32, 10, 10, None, None, None, K.KD_F64, None, None, None), K.KD_ERR_UNSUPPORTED),
    ((66, K.KD_F32, 10, 10, None, None, None, K.KD_F32, None, None, None), K.KD_ERR_MISALIGNED),
])
def test_eig3_argument_checks(args, expect):
    assert K.kd_eig3_sym(*args) == expect


def test_valid_call_without_a_device_reports_no_device():
    """Aligned, valid arguments pass every check; without a GPU the last check before the launch
    answers KD_ERR_NO_DEVICE (nothing is dereferenced)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present: this call would launch")
    assert K.kd_eig3_sym(64, K.KD_F32, 10, 10, 128, None, None, K.KD_F32, None, None, None) == K.KD_ERR_NO_DEVICE


def test_option_checks():
    o = K.kd_opts_default()
    o.max_sweeps = 9
    assert K.kd_eig3_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F32, None, o, None) == K.KD_ERR_INVALID_ARG
    o = K.kd_opts_default()
    o.form = K.KD_FORM_MIXED
    assert K.kd_eig3_sym(64, K.KD_F64, 10, 10, None, None, None, K.KD_F64, None, o, None) == K.KD_ERR_UNSUPPORTED
    o = K.kd_opts_default()
    o.form = K.KD_FORM_PLAIN
    assert K.kd_eig3_sym(64, K.KD_BF16, 10, 10, None, None, None, K.KD_F32, None, o, None) == K.KD_ERR_UNSUPPORTED
    o = K.kd_opts_default()
    o.layout = 2
    assert K.kd_eig3_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F32, None, o, None) == K.KD_ERR_INVALID_ARG
    o.layout = K.KD_LAYOUT_AOS
    assert K.kd_eig2_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F32, o, None) == K.KD_ERR_UNSUPPORTED
    o = K.kd_opts_default()
    o.stats = 12
    assert K.kd_eig3_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F32, None, o, None) == K.KD_ERR_MISALIGNED
    for field in ("degen_tau", "triple_tau", "conv_kappa", "gap_mask"):
        for bad in (float("nan"), float("inf"), -float("inf")):
            o = K.kd_opts_default()
            setattr(o, field, bad)
            assert K.kd_eig3_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F32, None, o, None) == \
                K.KD_ERR_INVALID_ARG, (field, bad)
            assert K.kd_st_loss_fwd_noalloc(64, K.KD_F32, 10, 10, (1, 0, 0), 64, o, None) == K.KD_ERR_INVALID_ARG


def test_other_entry_points_reject_bad_arguments():
    assert K.kd_eig2_sym(64, K.KD_BF16, 10, 10, None, None, None, K.KD_BF16, None, None) == K.KD_ERR_UNSUPPORTED
    assert K.kd_eig2_sym(64, K.KD_F32, 10, 10, None, None, None, K.KD_F64, None, None) == K.KD_ERR_UNSUPPORTED
    assert K.kd_eig3_sym_adjoint(64, K.KD_F32, 10, 10, None, None, None, None, None, None) == K.KD_ERR_INVALID_ARG
    assert K.kd_eig3_sym_adjoint(64, K.KD_F32, 10, 10, None, None, 66, 64, None, None) == K.KD_ERR_MISALIGNED
    assert K.kd_eig2_sym_adjoint(64, K.KD_F32, 10, 10, None, None, None, None, None) == K.KD_ERR_INVALID_ARG
    assert K.kd_st_loss_fwd(64, K.KD_F64, 10, 10, (1, 0, 0), 64, 1024, 64, None, None) == K.KD_ERR_UNSUPPORTED
    assert K.kd_st_loss_fwd(64, K.KD_F32, 10, 10, (1, 0, 0), 64, 1024, None, None, None) == K.KD_ERR_INVALID_ARG
    assert K.kd_st_loss_bwd(64, K.KD_BF16, 10, 10, (1, 0, 0), 1.0, None, None, None) == K.KD_ERR_INVALID_ARG
    assert K.kd_st_loss_bwd(64, K.KD_F32, 0, 0, (1, 0, 0), 1.0, None, None, None) == K.KD_OK
    assert K.kd_st_loss_fwd_bwd(64, K.KD_F64, 10, 10, (1, 0, 0), 1.0, 64, 1024, 64, 64, None,
                                None) == K.KD_ERR_UNSUPPORTED
    assert K.kd_st_loss_fwd_bwd(64, K.KD_F32, 10, 10, (1, 0, 0), 1.0, 64, 1024, 64, None, None,
                                None) == K.KD_ERR_INVALID_ARG
    assert K.kd_st_loss_fwd_bwd(64, K.KD_F32, 10, 10, (1, 0, 0), 1.0, 64, 1024, 64, 66, None,
                                None) == K.KD_ERR_MISALIGNED


def test_noalloc_checks():
    """kd_st_loss_fwd_noalloc takes the same option checks as the other entry points and rejects a
    batch beyond its fixed scratch before touching a device."""
    call = K.kd_st_loss_fwd_noalloc
    w = (1, 0, 0)
    for field, value, expect in (("invariants", 3, K.KD_ERR_INVALID_ARG), ("invariants", -1, K.KD_ERR_INVALID_ARG), ("form", 3, K.KD_ERR_INVALID_ARG),
                                 ("max_sweeps", 9, K.KD_ERR_INVALID_ARG), ("layout", 2, K.KD_ERR_INVALID_ARG),
                                 ("stats", 12, K.KD_ERR_MISALIGNED), ("layout", K.KD_LAYOUT_AOS, K.KD_ERR_UNSUPPORTED)):
        o = K.kd_opts_default()
        setattr(o, field, value)
        assert call(64, K.KD_F32, 10, 10, w, 64, o, None) == expect, field
    assert call(64, K.KD_F64, 10, 10, w, 64, None, None) == K.KD_ERR_UNSUPPORTED
    assert call(64, K.KD_F32, 10, 10, w, 68, None, None) == K.KD_ERR_MISALIGNED
    assert call(64, K.KD_F32, 10, 10, w, None, None, None) == K.KD_ERR_INVALID_ARG
    big = 8192 * 16384 + 1
    assert call(64, K.KD_F32, big, big, w, 64, None, None) == K.KD_ERR_TOO_LARGE


def test_host_pipeline_checks():
    """kd_eig3_sym_host rejects bad arguments before enqueuing anything; the workspace size grows
    with chunk and stream count."""
    a = K.kd_eig3_host_workspace_bytes(K.KD_F32, 1000, 1)
    assert a >= 1000 * (6 * 4 + 36 * 4) and K.kd_eig3_host_workspace_bytes(K.KD_F32, 1000, 3) == 3 * a
    assert K.kd_eig3_host_workspace_bytes(K.KD_F64, 1000, 1) > a
    assert K.kd_eig3_host_workspace_bytes(K.KD_F32, 0, 1) == 0
    assert K.kd_eig3_host_workspace_bytes(K.KD_F32, 10, 17) == 0
    call = K.kd_eig3_sym_host
    # stream list missing / stream count out of range / chunk 0
    assert call(64, K.KD_F32, 10, None, None, None, 64, None, None, None, 4, 256, 1 << 20, None, None, 1) == \
        K.KD_ERR_INVALID_ARG
    assert call(64, K.KD_F32, 10, None, None, None, 64, None, None, None, 4, 256, 1 << 20, None, [None], 0) == \
        K.KD_ERR_INVALID_ARG
    assert call(64, K.KD_F32, 10, None, None, None, 64, None, None, None, 0, 256, 1 << 20, None, [None], 1) == \
        K.KD_ERR_INVALID_ARG
    # a cotangent without A_bar, and A_bar without a cotangent
    assert call(64, K.KD_F32, 10, 64, None, None, None, None, None, None, 4, 256, 1 << 20, None, [None], 1) == \
        K.KD_ERR_INVALID_ARG
    assert call(64, K.KD_F32, 10, None, None, None, None, None, None, 64, 4, 256, 1 << 20, None, [None], 1) == \
        K.KD_ERR_INVALID_ARG
    # FP64 needs FP64 outputs: checked by type; misaligned host output; misaligned workspace
    assert call(64, 7, 10, None, None, None, 64, None, None, None, 4, 256, 1 << 20, None, [None], 1) == \
        K.KD_ERR_UNSUPPORTED
    assert call(64, K.KD_F64, 10, None, None, None, 68, None, None, None, 4, 256, 1 << 20, None, [None], 1) == \
        K.KD_ERR_MISALIGNED
    assert call(64, K.KD_F32, 10, None, None, None, 64, None, None, None, 4, 128, 1 << 20, None, [None], 1) == \
        K.KD_ERR_MISALIGNED
    o = K.kd_opts_default()
    o.layout = K.KD_LAYOUT_AOS
    assert call(64, K.KD_F32, 10, None, None, None, 64, None, None, None, 4, 256, 1 << 20, o, [None], 1) == \
        K.KD_ERR_UNSUPPORTED
    o = K.kd_opts_default()
    o.form = K.KD_FORM_PLAIN
    assert call(64, K.KD_BF16, 10, None, None, None, 64, None, None, None, 4, 256, 1 << 20, o, [None], 1) == \
        K.KD_ERR_UNSUPPORTED
    # empty batch: nothing to do
    assert call(None, K.KD_F32, 0, None, None, None, None, None, None, None, 4, None, 0, None, [None], 1) == K.KD_OK
    # no output requested: nothing to do (no workspace needed, no copies)
    assert call(64, K.KD_F32, 10, None, None, None, None, None, None, None, 4, None, 0, None, [None], 1) == K.KD_OK


def test_library_is_built_for_sm_103a_only():
    from paper_1306_6291_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(_build.LIB)
