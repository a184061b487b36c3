"""Seeded synthetic inputs for the batched 2x2 / 3x3 symmetric eigenproblem.

This module is shared by the GPU path's tests/benchmark and by the oracle checks. It holds none
of the diagonalization arithmetic: it only draws random numbers and builds matrices. Every
generator takes a seed and a torch device and draws from ``torch.Generator(device)`` seeded with
it, so a given (seed, device) always gives the same batch.

Layout: structure-of-arrays planes, ``(6, n)`` for 3x3 = rows (A11, A22, A33, A12, A13, A23) and
``(3, n)`` for 2x2 = rows (A11, A22, A12), contiguous, so plane k starts at ``k * n`` elements.

Workloads (sizes are parameters; the benchmark and the tests pick them):

* ``sym3_uniform``          entries i.i.d. U[-1, 1] (the plain FP64 workload)
* ``sym3_precision``        R diag(lam) R^T with Haar R in four equal groups (lam ~ N(0,1); two
                            eigenvalues equal to 1e-6 relative; near-triple with spread 1e-7;
                            exactly diagonal), each matrix scaled by 10^u, u ~ U[-15, 15], FP32
* ``sym2_normal_ties``      2x2 entries N(0,1), 10% with A11 := A22
* ``sym3_normal``           3x3 entries N(0,1)
* ``sym3_normal_gapped``    3x3 entries N(0,1), resampled until every eigen-gap >= min_gap
* ``structure_tensor_field`` 3x3 structure tensors of a smoothed Gaussian random field, BF16
  (``structure_tensor_from_field`` is the differentiable field -> tensor step)
"""
from __future__ import annotations

import math

import torch

PLANES3 = ("A11", "A22", "A33", "A12", "A13", "A23")
PLANES2 = ("A11", "A22", "A12")


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def haar_rotations(n: int, gen: torch.Generator, device, dtype=torch.float64) -> torch.Tensor:
    """(n, 3, 3) rotations distributed by Haar measure on SO(3): the rotation of a unit
    quaternion whose four components are i.i.d. normal."""
    q = torch.randn(n, 4, generator=gen, device=device, dtype=dtype)
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
        2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
        2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y),
    ], dim=1).reshape(n, 3, 3)
    return R


def pack3(M: torch.Tensor) -> torch.Tensor:
    """(n, 3, 3) symmetric -> (6, n) SoA planes."""
    return torch.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]], 0).contiguous()


def soa_to_aos(P: torch.Tensor) -> torch.Tensor:
    """(k, n) SoA planes -> (n, k) rows (a copy)."""
    return P.t().contiguous()


def sym3_uniform(n: int, seed: int = 0, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """(6, n): entries i.i.d. uniform on [-1, 1]."""
    g = _gen(seed, device)
    u = torch.rand(6, n, generator=g, device=device, dtype=torch.float64)
    return (2 * u - 1).to(dtype).contiguous()


GROUPS = ("normal", "pair_1e-6", "triple_1e-7", "diagonal")


def sym3_precision(n: int, seed: int = 0, device="cpu", scale_exp: float = 15.0,
                   chunk: int = 1 << 22) -> tuple[torch.Tensor, torch.Tensor]:
    """(6, n) float32 and the group index (n,) int8 of each matrix.

    The batch is split in four equal contiguous groups (group k = rows [k n/4, (k+1) n/4)):
      0  lam_i ~ N(0,1) i.i.d.;
      1  lam = (a, a (1 + 1e-6), b), a, b ~ N(0,1): two eigenvalues equal to 1e-6 relative;
      2  lam_i = c (1 + 1e-7 (t_i - 1/2)), c ~ N(0,1), t_i ~ U[0,1]: spread about 1e-7 relative;
      3  A = diag(lam), lam_i ~ N(0,1): exactly diagonal (R = I).
    Groups 0-2 use A = R diag(lam) R^T with Haar R. Every matrix is then multiplied by 10^u,
    u ~ U[-scale_exp, scale_exp]. The matrix is formed in float64 and rounded once to float32.
    Generated in chunks to bound the float64 temporaries."""
    g = _gen(seed, device)
    out = torch.empty(6, n, device=device, dtype=torch.float32)
    grp = torch.empty(n, device=device, dtype=torch.int8)
    q = n // 4
    bounds = [0, q, 2 * q, 3 * q, n]
    for k in range(4):
        lo_k, hi_k = bounds[k], bounds[k + 1]
        for s in range(lo_k, hi_k, chunk):
            m = min(chunk, hi_k - s)
            if m <= 0:
                continue
            if k == 0:
                lam = torch.randn(m, 3, generator=g, device=device, dtype=torch.float64)
            elif k == 1:
                ab = torch.randn(m, 2, generator=g, device=device, dtype=torch.float64)
                lam = torch.stack([ab[:, 0], ab[:, 0] * (1 + 1e-6), ab[:, 1]], 1)
            elif k == 2:
                c = torch.randn(m, 1, generator=g, device=device, dtype=torch.float64)
                t = torch.rand(m, 3, generator=g, device=device, dtype=torch.float64)
                lam = c * (1 + 1e-7 * (t - 0.5))
            else:
                lam = torch.randn(m, 3, generator=g, device=device, dtype=torch.float64)
            if k < 3:
                R = haar_rotations(m, g, device)
                M = torch.einsum("nij,nj,nkj->nik", R, lam, R)
            else:
                M = torch.diag_embed(lam)
            u = (2 * torch.rand(m, generator=g, device=device, dtype=torch.float64) - 1) * scale_exp
            M = M * torch.pow(10.0, u)[:, None, None]
            out[:, s:s + m] = pack3(M).to(torch.float32)
            grp[s:s + m] = k
    return out, grp


def sym2_normal_ties(n: int, seed: int = 0, device="cpu", tie_frac: float = 0.1) -> torch.Tensor:
    """(3, n) float32: A11, A22, A12 ~ N(0,1); a random tie_frac of them get A11 := A22."""
    g = _gen(seed, device)
    A = torch.randn(3, n, generator=g, device=device, dtype=torch.float32)
    tie = torch.rand(n, generator=g, device=device) < tie_frac
    A[0] = torch.where(tie, A[1], A[0])
    return A.contiguous()


def sym3_normal(n: int, seed: int = 0, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """(6, n): entries i.i.d. N(0, 1)."""
    g = _gen(seed, device)
    return torch.randn(6, n, generator=g, device=device, dtype=torch.float64).to(dtype).contiguous()


def _jacobi_eigvals(P: torch.Tensor, sweeps: int = 10) -> torch.Tensor:
    """Eigenvalues (unsorted, (m, 3)) of float64 packed symmetric matrices P (6, m) by cyclic
    Jacobi rotations (textbook, elementwise over the batch) - used only to filter generated
    inputs."""
    a = [P[k].clone() for k in range(6)]            # a11 a22 a33 a12 a13 a23
    diag = {0: 0, 1: 1, 2: 2}
    off = {(0, 1): 3, (0, 2): 4, (1, 2): 5}
    for _ in range(sweeps):
        for (p, q), r in ((((0, 1)), 2), (((0, 2)), 1), (((1, 2)), 0)):
            apq = a[off[(p, q)]]
            app, aqq = a[diag[p]], a[diag[q]]
            d = aqq - app
            rr = torch.sqrt(d * d + 4 * apq * apq)
            den = d.abs() + rr
            num = torch.where(d < 0, -2 * apq, 2 * apq)
            t = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), torch.zeros_like(den))
            c = 1 / torch.sqrt(1 + t * t)
            s = t * c
            apr = a[off[tuple(sorted((p, r)))]]
            aqr = a[off[tuple(sorted((q, r)))]]
            a[diag[p]] = app - t * apq
            a[diag[q]] = aqq + t * apq
            a[off[(p, q)]] = torch.zeros_like(apq)
            a[off[tuple(sorted((p, r)))]] = c * apr - s * aqr
            a[off[tuple(sorted((q, r)))]] = s * apr + c * aqr
    return torch.stack([a[0], a[1], a[2]], 1)


def min_eigen_gap(P: torch.Tensor, chunk: int = 1 << 22) -> torch.Tensor:
    """Smallest |lam_i - lam_j| of each (6, n) matrix (float64 Jacobi eigenvalues)."""
    n = P.shape[1]
    out = torch.empty(n, device=P.device, dtype=torch.float64)
    for s in range(0, n, chunk):
        Q = P[:, s:s + chunk].to(torch.float64)
        w = torch.sort(_jacobi_eigvals(Q), dim=1).values
        out[s:s + chunk] = torch.minimum(w[:, 1] - w[:, 0], w[:, 2] - w[:, 1])
    return out


def sym3_normal_gapped(n: int, seed: int = 0, device="cpu", min_gap: float = 1e-3,
                       max_rounds: int = 50) -> torch.Tensor:
    """(6, n) float32, entries N(0,1); any matrix whose float32 entries have an eigen-gap below
    min_gap is redrawn (fresh N(0,1) entries) until none is left."""
    g = _gen(seed, device)
    A = torch.randn(6, n, generator=g, device=device, dtype=torch.float64).to(torch.float32)
    bad = torch.nonzero(min_eigen_gap(A) < min_gap).flatten()
    rounds = 0
    while bad.numel() > 0:
        rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("sym3_normal_gapped: resampling did not converge")
        A[:, bad] = torch.randn(6, bad.numel(), generator=g, device=device,
                                dtype=torch.float64).to(torch.float32)
        sub = min_eigen_gap(A[:, bad].contiguous())
        bad = bad[sub < min_gap]
    return A.contiguous()


def _gauss_fft_filter(shape, sigma: float, device) -> torch.Tensor:
    """Fourier transfer function of a periodic Gaussian blur with std sigma voxels, for rfftn."""
    ks = []
    for i, s in enumerate(shape):
        if i == len(shape) - 1:
            k = torch.fft.rfftfreq(s, device=device, dtype=torch.float64)
        else:
            k = torch.fft.fftfreq(s, device=device, dtype=torch.float64)
        ks.append(k)
    kx, ky, kz = torch.meshgrid(*ks, indexing="ij")
    return torch.exp(-2 * math.pi ** 2 * sigma ** 2 * (kx * kx + ky * ky + kz * kz)).to(torch.float32)


def structure_tensor_from_field(f: torch.Tensor, sigma_int: float = 2.0, dtype=None) -> torch.Tensor:
    """(6, X*Y*Z) structure tensors J = G_{sigma_int} * (grad f grad f^T) of a field f (X, Y, Z):
    central-difference gradient, products blurred with a periodic Gaussian of std sigma_int
    voxels (FFT). Differentiable in f (plain torch operations), so a loss on J can be
    back-propagated to the field. Returned in f's dtype unless ``dtype`` is given."""
    shape = tuple(f.shape)
    grads = [(torch.roll(f, -1, d) - torch.roll(f, 1, d)) * 0.5 for d in range(3)]
    Hi = _gauss_fft_filter(shape, sigma_int, f.device).to(f.dtype)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    comps = [torch.fft.irfftn(torch.fft.rfftn(grads[i] * grads[j]) * Hi, s=shape).reshape(-1) for i, j in pairs]
    J = torch.stack(comps, 0)
    return J if dtype is None else J.to(dtype)


def structure_tensor_field(shape=(512, 512, 256), seed: int = 0, device="cpu", sigma: float = 2.0,
                           sigma_int: float = 2.0, dtype=torch.bfloat16) -> torch.Tensor:
    """(6, X*Y*Z) structure tensors J = G_{sigma_int} * (grad f grad f^T) of a Gaussian random
    field f: white noise N(0,1) on a periodic grid, blurred with a Gaussian of std sigma voxels
    and normalised to unit variance; grad by central differences; each product blurred with a
    Gaussian of std sigma_int. Periodic boundaries throughout (FFT). Stored as ``dtype``."""
    g = _gen(seed, device)
    f = torch.randn(*shape, generator=g, device=device, dtype=torch.float32)
    H = _gauss_fft_filter(shape, sigma, device)
    f = torch.fft.irfftn(torch.fft.rfftn(f) * H, s=shape)
    f = (f - f.mean()) / f.std()
    grads = [(torch.roll(f, -1, d) - torch.roll(f, 1, d)) * 0.5 for d in range(3)]
    del f
    Hi = _gauss_fft_filter(shape, sigma_int, device)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    out = torch.empty(6, math.prod(shape), device=device, dtype=dtype)
    for k, (i, j) in enumerate(pairs):
        J = torch.fft.irfftn(torch.fft.rfftn(grads[i] * grads[j]) * Hi, s=shape)
        out[k] = J.reshape(-1).to(dtype)
    return out
