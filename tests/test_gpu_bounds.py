"""No kernel writes outside its batch: every output is a (k, ld) buffer with ld > n, pre-filled
with a canary value, and after each call the columns n..ld-1 of every plane (and the rows past n
of AoS records) must still hold the canary. Ragged sizes, including batches much smaller than one
block, exercise the tail handling of the grid-stride and unrolled loops."""
import math

import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import kdiag as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CANARY = 12345.5


def _buf(rows, ld, dtype=torch.float32):
    return torch.full((rows, ld), CANARY, device=DEV, dtype=dtype)


def _tail_intact(t, n):
    return bool((t[:, n:] == CANARY).all())


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n", [1, 33, 1000, 5003])
def test_3x3_forward_and_adjoint_stay_in_bounds(n):
    ld = n + 117
    A = torch.zeros(6, ld, device=DEV)
    A[:, :n] = W.sym3_normal(n, seed=n, device=DEV)
    for outs in ((True, True, True), (True, False, True), (True, True, False), (False, True, False)):
        lam, D, ang = _buf(3, ld), _buf(9, ld), _buf(3, ld)
        ptr = [t.data_ptr() if want else None for t, want in zip((lam, D, ang), outs)]
        assert K.kd_eig3_sym(A.data_ptr(), K.KD_F32, n, ld, ptr[0], ptr[1], ptr[2], K.KD_F32, None, None,
                             _stream()) == K.KD_OK
        torch.cuda.synchronize()
        for t, want in zip((lam, D, ang), outs):
            assert _tail_intact(t, n)
            if not want:
                assert bool((t == CANARY).all())
    g = torch.Generator(device=DEV).manual_seed(n)
    lb, Db, ab = (torch.randn(k, ld, generator=g, device=DEV) for k in (3, 9, 3))
    for use_ang in (False, True):
        Ab = _buf(6, ld)
        assert K.kd_eig3_sym_adjoint(A.data_ptr(), K.KD_F32, n, ld, lb.data_ptr(), Db.data_ptr(),
                                     ab.data_ptr() if use_ang else None, Ab.data_ptr(), None,
                                     _stream()) == K.KD_OK
        torch.cuda.synchronize()
        assert _tail_intact(Ab, n) and bool(torch.isfinite(Ab[:, :n]).all())


@pytest.mark.parametrize("n", [1, 33, 1000, 5003])
def test_2x2_forward_and_adjoint_stay_in_bounds(n):
    ld = n + 117
    A = torch.zeros(3, ld, device=DEV)
    A[:, :n] = W.sym2_normal_ties(n, seed=n, device=DEV)
    lam, phi, D = _buf(2, ld), _buf(1, ld), _buf(4, ld)
    assert K.kd_eig2_sym(A.data_ptr(), K.KD_F32, n, ld, lam.data_ptr(), phi.data_ptr(), D.data_ptr(), K.KD_F32,
                         None, _stream()) == K.KD_OK
    torch.cuda.synchronize()
    assert _tail_intact(lam, n) and _tail_intact(phi, n) and _tail_intact(D, n)
    g = torch.Generator(device=DEV).manual_seed(n)
    lb, pb = torch.randn(2, ld, generator=g, device=DEV), torch.randn(1, ld, generator=g, device=DEV)
    Ab = _buf(3, ld)
    assert K.kd_eig2_sym_adjoint(A.data_ptr(), K.KD_F32, n, ld, lb.data_ptr(), pb.data_ptr(), Ab.data_ptr(), None,
                                 _stream()) == K.KD_OK
    torch.cuda.synchronize()
    assert _tail_intact(Ab, n)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("n", [1, 33, 5003])
def test_loss_gradient_stays_in_bounds(n, dtype):
    ld = n + 117
    field = W.structure_tensor_field((32, 16, 12), seed=1, device=DEV)
    A = torch.zeros(6, ld, device=DEV, dtype=dtype)
    A[:, :n] = field[:, :n].to(dtype)
    wv = (1 / math.sqrt(3),) * 3
    ws = K.st_loss_workspace(n, torch.device(DEV))
    loss = torch.empty(2, device=DEV, dtype=torch.float64)
    Ab = _buf(6, ld, dtype)
    assert K.kd_st_loss_fwd_bwd(A.data_ptr(), K._DT[dtype], n, ld, wv, 1.0, ws.data_ptr(), ws.numel() * 8,
                                loss.data_ptr(), Ab.data_ptr(), None, _stream()) == K.KD_OK
    Ab2 = _buf(6, ld, dtype)
    assert K.kd_st_loss_bwd(A.data_ptr(), K._DT[dtype], n, ld, wv, 1.0, Ab2.data_ptr(), None,
                            _stream()) == K.KD_OK
    torch.cuda.synchronize()
    assert _tail_intact(Ab, n) and _tail_intact(Ab2, n)
    assert bool(torch.isfinite(loss).all())


@pytest.mark.parametrize("n", [1, 255, 256, 1000, 5003])
def test_aos_records_stay_in_bounds(n):
    pad = 37
    A = torch.zeros(n + pad, 6, device=DEV)
    A[:n] = W.sym3_normal(n, seed=n, device=DEV).t()
    lam, D, ang = (torch.full((n + pad, k), CANARY, device=DEV) for k in (3, 9, 3))
    o = K.kd_opts_default()
    o.layout = K.KD_LAYOUT_AOS
    assert K.kd_eig3_sym(A.data_ptr(), K.KD_F32, n, n, lam.data_ptr(), D.data_ptr(), ang.data_ptr(), K.KD_F32,
                         None, o, _stream()) == K.KD_OK
    g = torch.Generator(device=DEV).manual_seed(n)
    lb, Db = torch.randn(n + pad, 3, generator=g, device=DEV), torch.randn(n + pad, 9, generator=g, device=DEV)
    Ab = torch.full((n + pad, 6), CANARY, device=DEV)
    assert K.kd_eig3_sym_adjoint(A.data_ptr(), K.KD_F32, n, n, lb.data_ptr(), Db.data_ptr(), None, Ab.data_ptr(), o,
                                 _stream()) == K.KD_OK
    torch.cuda.synchronize()
    for t in (lam, D, ang, Ab):
        assert bool((t[n:] == CANARY).all())
        assert bool(torch.isfinite(t[:n]).all())


def test_batches_beyond_2_31_matrices():
    """n = 2^31 + 4097: the matrix index itself needs 64 bits (the other tests reach the 64-bit
    variants through large plane strides only). 3x3 eigenvalues (A 51.5 GB, lam 25.8 GB), then the
    2x2 forward (51.5 GB in all), each checked on matrices sampled across the batch, most of them
    past index 2^31, against the oracle. Skipped on a device with less than 100 GB free."""
    import numpy as np

    import oracle
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip(f"needs 100 GB of free device memory, {free / 1e9:.0f} GB free")
    n = (1 << 31) + 4097
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([np.arange(1000), np.arange(n - 3000, n),
                                    rng.integers(1 << 31, n, 4000), rng.integers(0, n, 4000)]))
    it = torch.as_tensor(idx, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(31)

    A = torch.empty(6, n, device=DEV)
    A.normal_(generator=g)
    lam = torch.full((3, n), CANARY, device=DEV)
    assert K.kd_eig3_sym(A.data_ptr(), K.KD_F32, n, n, lam.data_ptr(), None, None, K.KD_F32, None, None,
                         _stream()) == K.KD_OK
    torch.cuda.synchronize()
    Ar = A[:, it].t().double().cpu().numpy()
    lg = lam[:, it].t().double().cpu().numpy()
    del A, lam
    torch.cuda.empty_cache()
    lj, _, _ = oracle.jacobi3(Ar)
    fro = np.linalg.norm(oracle.unpack3(Ar), axis=(1, 2))
    assert np.max(np.abs(np.sort(lg, 1)[:, ::-1] - lj).max(1) / fro) < 2e-6

    A2 = torch.empty(3, n, device=DEV)
    A2.normal_(generator=g)
    lam2 = torch.full((2, n), CANARY, device=DEV)
    phi = torch.full((1, n), CANARY, device=DEV)
    assert K.kd_eig2_sym(A2.data_ptr(), K.KD_F32, n, n, lam2.data_ptr(), phi.data_ptr(), None, K.KD_F32, None,
                         _stream()) == K.KD_OK
    torch.cuda.synchronize()
    A2r = A2[:, it].t().double().cpu().numpy()
    l2 = lam2[:, it].t().double().cpu().numpy()
    p2 = phi[0, it].double().cpu().numpy()
    del A2, lam2, phi
    torch.cuda.empty_cache()
    lo, po = oracle.eig2(A2r)
    fro2 = np.sqrt(A2r[:, 0] ** 2 + A2r[:, 1] ** 2 + 2 * A2r[:, 2] ** 2)
    assert np.max(np.abs(l2 - lo) / fro2[:, None]) < 2e-6
    gap = np.abs(lo[:, 0] - lo[:, 1])
    assert np.max(np.abs(p2 - po) * gap / fro2) < 1e-6
