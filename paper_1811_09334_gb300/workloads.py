"""Seeded synthetic inputs for the randomized QLP path.

This module only builds test matrices A and Gaussian sketch matrices Omega.
It contains none of the factorization's arithmetic, so both the CUDA path and
the FP64 CPU oracle can be fed from it.

Matrix families
---------------
* ``low_rank_from_spectrum``: A = X diag(sigma) Y^T with X, Y orthonormal,
  taken from the QR of seeded N(0,1) matrices (the construction of the
  paper's Example 5.1 test matrices, Section 5).
* ``pds`` / ``eds``: the polynomially / exponentially decaying spectra of
  Example 5.1 (Section 5): the first t singular values are 1, then
  2^-s, 3^-s, ... (pds) or 2^-s, 2^-2s, ... (eds).
* ``c1`` ... ``c5``: the five workloads the benchmarks and parity tests use
  (RQLP FP64 2000x1000; ERQLP 8192^2; ERQLP 32768x16384 low rank plus noise;
  the differentiable 4096x2048 case; 512 uneven batched problems).

Seeds: the matrix of workload i (0-based) uses seed 1811 + i and the sketch of
trial t uses seed 9334 + t, both through numpy's PCG64 ``standard_normal``.
Large matrices can be finished on a CUDA device (``device=``): the Gaussian
entries still come from numpy, only the QR and the product run in torch.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_A = 1811
SEED_OMEGA = 9334


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded N(0,1) matrix (row-major)."""
    return _rng(seed).standard_normal((rows, cols)).astype(dtype, copy=False)


def omega(n: int, l: int, trial: int = 0) -> np.ndarray:
    """The n x l Gaussian sketch matrix of trial ``trial`` (FP64)."""
    return gaussian(n, l, SEED_OMEGA + trial)


def _orthonormal_np(G: np.ndarray) -> np.ndarray:
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def low_rank_from_spectrum(m: int, n: int, sigma: np.ndarray, seed: int,
                           device: Optional[str] = None, out_dtype=np.float64,
                           qr_float32: bool = False):
    """A = X diag(sigma) Y^T, X (m x r) and Y (n x r) orthonormal, r = len(sigma).

    Returns a numpy array, or a torch tensor on ``device`` if one is given.
    qr_float32 (device only) takes the QR of the Gaussian factors in FP32 for
    speed; X and Y are then orthonormal to about 1e-6, i.e. A's singular
    values are sigma to that relative accuracy.
    """
    r = len(sigma)
    rng = _rng(seed)
    GX = rng.standard_normal((m, r))
    GY = rng.standard_normal((n, r))
    if device is None:
        X = _orthonormal_np(GX)
        Y = _orthonormal_np(GY)
        A = (X * sigma[None, :]) @ Y.T
        return A.astype(out_dtype, copy=False)
    import torch
    tdt = torch.float64 if out_dtype == np.float64 else torch.float32
    def orth(G):
        try:
            Gt = torch.from_numpy(G).to(device)
            if qr_float32:
                Gt = Gt.float()
            Q, R = torch.linalg.qr(Gt)
            s = torch.sign(torch.diagonal(R))
            s[s == 0] = 1.0
            return (Q * s).double()
        except RuntimeError:
            # torch's device linear algebra can be unavailable (e.g. under a
            # profiler); the same construction then runs on the host.
            return torch.from_numpy(_orthonormal_np(G)).to(device)
    X = orth(GX)
    del GX
    Y = orth(GY)
    del GY
    sig = torch.from_numpy(np.ascontiguousarray(sigma)).to(device)
    A = (X * sig[None, :]) @ Y.T
    return A.to(tdt).contiguous()


def pds_spectrum(n: int, t: int, s: float) -> np.ndarray:
    """Polynomially decaying spectrum of Example 5.1: t ones, then j^-s, j = 2.."""
    tail = np.arange(2, n - t + 2, dtype=np.float64) ** (-s)
    return np.concatenate([np.ones(t), tail])[:n]


def eds_spectrum(n: int, t: int, s: float) -> np.ndarray:
    """Exponentially decaying spectrum of Example 5.1: t ones, then 2^(-i s)."""
    tail = 2.0 ** (-s * np.arange(1, n - t + 1, dtype=np.float64))
    return np.concatenate([np.ones(t), tail])[:n]


@dataclasses.dataclass
class Problem:
    """One factorization problem: A (m x n), target rank k, oversampling p."""
    name: str
    A: object
    sigma: Optional[np.ndarray]
    k: int
    p: int
    q: int
    d: int
    pivot2: int

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def n(self):
        return self.A.shape[1]

    @property
    def l(self):
        return self.k + self.p


def c1(m: int = 2000, n: int = 1000, k: int = 20, p: int = 10, device=None) -> Problem:
    """RQLP, q = 0, FP64: sigma_j = j^-2, X (m x n), Y (n x n) orthonormal."""
    sigma = np.arange(1, n + 1, dtype=np.float64) ** -2.0
    A = low_rank_from_spectrum(m, n, sigma, SEED_A + 0, device=device)
    return Problem("c1_rqlp_fp64_%dx%d" % (m, n), A, sigma, k, p, 0, 1, 1)


def c2(m: int = 8192, n: int = 8192, k: int = 100, p: int = 10, q: int = 1,
       d: int = 2, device=None) -> Problem:
    """ERQLP: sigma_j = 10^(-j/100), exponential decay, m = n = 8192."""
    r = min(m, n)
    sigma = 10.0 ** (-np.arange(1, r + 1, dtype=np.float64) / 100.0)
    A = low_rank_from_spectrum(m, n, sigma, SEED_A + 1, device=device)
    return Problem("c2_erqlp_%dx%d" % (m, n), A, sigma, k, p, q, d, 0)


def c3(m: int = 32768, n: int = 16384, r: int = 300, k: int = 200, p: int = 10,
       noise: float = 1e-4, device=None) -> Problem:
    """ERQLP q = 2: G1 diag(1/j) G2^T + noise * N(0,1), FP32 storage.

    G1 (m x r) and G2 (n x r) are N(0,1)/sqrt(dim); the spectrum is therefore
    only approximately 1/j and sigma is not returned exactly (None).
    """
    rng = _rng(SEED_A + 2)
    G1 = rng.standard_normal((m, r)) / np.sqrt(m)
    G2 = rng.standard_normal((n, r)) / np.sqrt(n)
    sig = 1.0 / np.arange(1, r + 1, dtype=np.float64)
    if device is None:
        A = (G1 * sig[None, :]) @ G2.T
        A += noise * rng.standard_normal((m, n))
        A = A.astype(np.float32)
    else:
        import torch
        g1 = torch.from_numpy(G1 * sig[None, :]).to(device)
        g2 = torch.from_numpy(G2).to(device)
        A = (g1 @ g2.T)
        del g1, g2
        # the noise is drawn in row slabs to bound host memory
        slab = 2048
        for i0 in range(0, m, slab):
            i1 = min(m, i0 + slab)
            A[i0:i1] += noise * torch.from_numpy(rng.standard_normal((i1 - i0, n))).to(device)
        A = A.to(torch.float32).contiguous()
    return Problem("c3_erqlp_%dx%d_fp32" % (m, n), A, None, k, p, 2, 2, 0)


def c4(m: int = 4096, n: int = 2048, k: int = 64, p: int = 8, device=None) -> Problem:
    """Differentiable case: A = N(0,1) diag(2^(-j/256)), FP32."""
    G = gaussian(m, n, SEED_A + 3)
    A = (G * 2.0 ** (-np.arange(n, dtype=np.float64) / 256.0)[None, :]).astype(np.float32)
    if device is not None:
        import torch
        A = torch.from_numpy(A).to(device)
    return Problem("c4_rqlp_grad_%dx%d" % (m, n), A, None, k, p, 1, 1, 1)


def c5_shapes(count: int = 512, mmax: int = 4096, seed: int = SEED_A + 4):
    """Shapes (m, n, k) of the batched workload: m ~ U[256, mmax], n ~ U[128, m], k ~ U[8, 64]."""
    rng = _rng(seed)
    shapes = []
    for _ in range(count):
        m = int(rng.integers(256, mmax + 1))
        n = int(rng.integers(128, m + 1))
        k = int(rng.integers(8, 65))
        shapes.append((m, n, k))
    return shapes


def c5_matrix(i: int, m: int, n: int, device=None, fast: bool = False):
    """Matrix i of the batched workload: X diag(j^-1.5) Y^T (fast: FP32 QR on the device)."""
    r = min(m, n)
    sigma = np.arange(1, r + 1, dtype=np.float64) ** -1.5
    return low_rank_from_spectrum(m, n, sigma, SEED_A + 100 + i, device=device,
                                  qr_float32=fast), sigma


def w6(kind: str, n: int, t: int = 30, s: Optional[float] = None, seed: int = SEED_A + 5,
       device=None) -> Problem:
    """Paper-shaped workload (Example 5.1, Tables 1-2): m = n, k = 120, p = 5."""
    if kind == "pds":
        sigma = pds_spectrum(n, t, 2.0 if s is None else s)
    elif kind == "eds":
        sigma = eds_spectrum(n, t, 1.0 / 20.0 if s is None else s)
    else:
        raise ValueError(kind)
    A = low_rank_from_spectrum(n, n, sigma, seed, device=device)
    return Problem("w6_%s_%d" % (kind, n), A, sigma, 120, 5, 0, 2, 0)
