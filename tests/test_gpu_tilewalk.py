"""The 3x3 SoA kernels visit a batch in scrambled tiles of 1024 matrices (csrc/kd_soa.cuh,
TileWalk): every block takes tiles (b + kG) M mod T, and the threads of a partial last tile past
the end compute on clamped loads and store nothing. These tests check, on sizes around the tile
and grid boundaries, that every matrix is written exactly where it belongs and nothing past the
end of a plane (ld > n, canary-filled gaps), and that a matrix's results do not depend on where
it sits in the batch (the same instructions run for every position): the same matrices shifted
by an offset give identical bits."""
import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import kdiag as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CANARY = -12345.0
SHIFT = 777


def _fwd(A, n, ld, off):
    """Forward of matrices off .. off+n-1 of A (6, ld_a) written into canary-filled planes of
    stride ld."""
    lam, D, ang = (torch.full((k, ld), CANARY, device=DEV) for k in (3, 9, 3))
    Av = torch.full((6, ld), 0.0, device=DEV)
    Av[:, :n] = A[:, off:off + n]
    s = K.kd_eig3_sym(Av.data_ptr(), K.KD_F32, n, ld, lam.data_ptr(), D.data_ptr(), ang.data_ptr(), K.KD_F32,
                      None, None, torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_OK
    return lam, D, ang


def _adj(A, lb, Db, n, ld, off):
    Ab = torch.full((6, ld), CANARY, device=DEV)
    Av, lv, Dv = torch.zeros(6, ld, device=DEV), torch.zeros(3, ld, device=DEV), torch.zeros(9, ld, device=DEV)
    Av[:, :n], lv[:, :n], Dv[:, :n] = A[:, off:off + n], lb[:, off:off + n], Db[:, off:off + n]
    s = K.kd_eig3_sym_adjoint(Av.data_ptr(), K.KD_F32, n, ld, lv.data_ptr(), Dv.data_ptr(), None, Ab.data_ptr(),
                              None, torch.cuda.current_stream().cuda_stream)
    assert s == K.KD_OK
    return Ab


@pytest.mark.parametrize("n", [1, 1023, 1024, 1025, 152 * 1024 - 1, 152 * 1024 + 1, 3 * 152 * 1024 + 517])
def test_tile_walk_writes_each_matrix_once_and_is_position_independent(n):
    A, _ = W.sym3_precision(n + SHIFT, seed=n % 1000, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(7)
    lb, Db = torch.randn(3, n + SHIFT, generator=g, device=DEV), torch.randn(9, n + SHIFT, generator=g, device=DEV)
    ld = n + 61
    outs0 = _fwd(A, n, ld, 0) + (_adj(A, lb, Db, n, ld, 0),)
    outs1 = _fwd(A, n, ld, SHIFT) + (_adj(A, lb, Db, n, ld, SHIFT),)
    for P0, P1 in zip(outs0, outs1):
        # every entry of the n matrices written (no canary left), the gaps past n untouched
        assert not (P0[:, :n] == CANARY).any() and not (P1[:, :n] == CANARY).any()
        assert (P0[:, n:] == CANARY).all() and (P1[:, n:] == CANARY).all()
        # matrix SHIFT + j of the first call is matrix j of the second: identical bits
        if n > SHIFT:
            assert torch.equal(P0[:, SHIFT:n], P1[:, :n - SHIFT])
