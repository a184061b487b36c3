"""The mixed 2x2 + 3x3 batch as one CUDA graph (one launch per size captured from the C-ABI calls
on a PyTorch stream) gives the same results as eager calls, and replays on new inputs."""
import pytest
import torch

import workloads as W
from paper_1306_6291_gb300 import kdiag as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_mixed_batch_graph_matches_eager():
    n = 1 << 18
    A2 = W.sym2_normal_ties(n, seed=0, device=DEV)
    A3 = W.sym3_normal(n, seed=1, device=DEV)
    lam2, phi2, _ = K.eig2(A2)
    lam3, _, ang3, _ = K.eig3(A3, D=False)
    o_lam2, o_phi2 = torch.empty_like(lam2), torch.empty_like(phi2)
    o_lam3, o_ang3 = torch.empty_like(lam3), torch.empty_like(ang3)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            h = torch.cuda.current_stream().cuda_stream
            assert K.kd_eig2_sym(A2.data_ptr(), K.KD_F32, n, n, o_lam2.data_ptr(), o_phi2.data_ptr(), None,
                                 K.KD_F32, None, h) == K.KD_OK
            assert K.kd_eig3_sym(A3.data_ptr(), K.KD_F32, n, n, o_lam3.data_ptr(), None, o_ang3.data_ptr(),
                                 K.KD_F32, None, None, h) == K.KD_OK
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(o_lam2, lam2) and torch.equal(o_phi2, phi2)
    assert torch.equal(o_lam3, lam3) and torch.equal(o_ang3, ang3)
    # new inputs in the same buffers
    A2.copy_(W.sym2_normal_ties(n, seed=5, device=DEV))
    A3.copy_(W.sym3_normal(n, seed=6, device=DEV))
    g.replay()
    torch.cuda.synchronize()
    l2, p2, _ = K.eig2(A2)
    l3, _, a3, _ = K.eig3(A3, D=False)
    assert torch.equal(o_lam2, l2) and torch.equal(o_ang3, a3)


def test_mixed_3x3_half_full_size_sampled():
    """The mixed workload's 3x3 half at full size (2^25 N(0,1) matrices, lam + angles, the
    instantiation the graph launches), checked on sampled matrices against the long-double Jacobi
    definition oracle: eigenvalues, and eigenvectors and reconstruction through D = R1 R2 R3 of
    the returned angles (Eq. (6.5))."""
    import numpy as np

    import oracle
    from parity import definition_errors, euler_D, planes_to_rows

    n = 1 << 25
    A3 = W.sym3_normal(n, seed=1, device=DEV)
    lam, _, ang, _ = K.eig3(A3, D=False)
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([np.arange(128), np.arange(n - 128, n), rng.integers(0, n, 3000)]))
    it = torch.as_tensor(idx, device=DEV)
    Ar = planes_to_rows(A3[:, it])
    e = definition_errors(Ar, planes_to_rows(lam[:, it]), euler_D(planes_to_rows(ang[:, it])))
    assert np.max(e["lam"]) < 2e-6
    assert np.max(e["rec"]) < 4e-6
    assert np.max(e["ev"]) < 1e-5
