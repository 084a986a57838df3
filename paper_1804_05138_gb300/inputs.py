"""Seeded synthetic inputs for randomized QRCP: test matrices and explicit sketches.

This module holds no step of the factorization; it only draws matrices.  Both the
test suite's oracle comparisons and the benchmark take their inputs from here, so
that the CUDA path and the CPU oracle see the same data.

Recipes (numpy PCG64 ``default_rng(seed)`` unless stated):
  * ``haar(n_rows, n_cols, seed)``: Q of the QR of an N(0,1) matrix, columns scaled
    by sign(diag R) (Mezzadri 2007), i.e. Haar-distributed orthonormal columns.
  * ``spectrum_matrix(m, n, sigma, seed_u, seed_v)``: U diag(sigma) V^T with Haar U, V.
  * ``gaussian(m, n, seed)``: i.i.d. N(0,1) entries.
  * ``rank_r_product(m, n, r, seed1, seed2)``: G1 G2 with G1 m x r, G2 r x n, N(0,1).
  * ``kahan(n, c)``: diag(s^0..s^{n-1}) (I - c * strictly-upper ones), s = sqrt(0.9999 - c^2)
    (the paper's Sec. V-B parameters).
  * ``gaussian_sketch(l, m, seed)``: an explicit N(0,1) sketching matrix, row-major l x m,
    for the entry point that takes Omega as an input.
Spectra are indexed from 1 (sigma_1 is the largest), as the paper's sigma_j notation.
Large inputs for the benchmark are drawn on the GPU with torch (``*_torch``) by the
same recipe; their values differ from the numpy draws, which only size-limited tests use.
"""
from __future__ import annotations

import numpy as np


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((m, n)))


def haar(n_rows: int, n_cols: int, seed: int) -> np.ndarray:
    G = np.random.default_rng(seed).standard_normal((n_rows, n_cols))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def spectrum_matrix(m: int, n: int, sigma: np.ndarray, seed_u: int = 1, seed_v: int = 2,
                    rank_cap: int | None = None) -> np.ndarray:
    """U diag(sigma) V^T with Haar U, V; ``rank_cap`` keeps only the leading triplets."""
    r = min(m, n, len(sigma))
    if rank_cap is not None:
        r = min(r, rank_cap)
    U = haar(m, r, seed_u)
    V = haar(n, r, seed_v)
    return np.asfortranarray((U * np.asarray(sigma[:r])) @ V.T)


def rank_r_product(m: int, n: int, r: int, seed1: int = 1, seed2: int = 2) -> np.ndarray:
    G1 = np.random.default_rng(seed1).standard_normal((m, r))
    G2 = np.random.default_rng(seed2).standard_normal((r, n))
    return np.asfortranarray(G1 @ G2)


def kahan(n: int, c: float = 0.285) -> np.ndarray:
    s = np.sqrt(0.9999 - c * c)
    K = np.eye(n) - c * np.triu(np.ones((n, n)), 1)
    return np.asfortranarray(np.diag(s ** np.arange(n)) @ K)


def gaussian_sketch(l: int, m: int, seed: int) -> np.ndarray:
    """Explicit Omega (row-major l x m) for the explicit-sketch entry point."""
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal((l, m)))


# ---------------------------------------------------------------- spectra of the workloads
def sigma_log_decay(n: int, decades: float = 6.0) -> np.ndarray:
    """sigma_i = 10^(-decades * i / n), i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return 10.0 ** (-decades * i / n)


def sigma_exp_decay(n: int, scale: float) -> np.ndarray:
    """sigma_i = exp(-i / scale), i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.exp(-i / scale)


def sigma_inverse_square(n: int) -> np.ndarray:
    """sigma_i = 1 / (1 + i)^2, i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return 1.0 / (1.0 + i) ** 2


def batched_shapes(count: int = 512, seed: int = 0, p: int = 8):
    """Uneven batch: m ~ U[256,4096], n ~ U[128, min(m,2048)], k ~ U[16,256] clipped to n,
    drawn per matrix in the order (m, n, k) from default_rng(seed); integers inclusive."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(256, 4096, endpoint=True))
        n = int(rng.integers(128, min(m, 2048), endpoint=True))
        k = min(int(rng.integers(16, 256, endpoint=True)), n)
        out.append((m, n, k))
    return out


# ---------------------------------------------------------------- GPU-side draws (torch)
def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def gaussian_torch(m: int, n: int, seed: int, device="cuda", dtype=None):
    """i.i.d. N(0,1), column-major m x n (returned as the transpose view of an n x m tensor)."""
    import torch
    dtype = dtype or torch.float64
    g = _torch_gen(seed, device)
    return torch.randn((n, m), generator=g, device=device, dtype=dtype).t()


def haar_torch(n_rows: int, n_cols: int, seed: int, device="cuda"):
    import torch
    g = _torch_gen(seed, device)
    G = torch.randn((n_rows, n_cols), generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return Q * d


def spectrum_matrix_torch(m: int, n: int, sigma, seed_u: int = 1, seed_v: int = 2, device="cuda",
                          dtype=None, rank_cap: int | None = None):
    """U diag(sigma) V^T drawn on the device in FP64, stored column-major in ``dtype``.

    ``rank_cap`` keeps only the leading singular triplets: used when sigma beyond the cap is
    below the storage precision relative to sigma_1 (the dropped part is under one rounding
    of the stored entries)."""
    import torch
    dtype = dtype or torch.float64
    r = min(m, n, len(sigma))
    if rank_cap is not None:
        r = min(r, rank_cap)
    U = haar_torch(m, r, seed_u, device)
    V = haar_torch(n, r, seed_v, device)
    s = torch.as_tensor(np.asarray(sigma[:r]), device=device, dtype=torch.float64)
    A = (V * s) @ U.t()          # n x m row-major == m x n column-major
    return A.to(dtype).t()


def rank_r_product_torch(m: int, n: int, r: int, seed1: int = 1, seed2: int = 2, device="cuda", dtype=None):
    import torch
    dtype = dtype or torch.float64
    g1 = _torch_gen(seed1, device)
    g2 = _torch_gen(seed2, device)
    G1 = torch.randn((m, r), generator=g1, device=device, dtype=torch.float64)
    G2 = torch.randn((r, n), generator=g2, device=device, dtype=torch.float64)
    return (G2.t() @ G1.t()).to(dtype).t()
