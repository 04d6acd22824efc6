"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers. It holds none of the method's
arithmetic (no graphs, no Laplacians, no solver steps), so both the FP64
oracle and the CUDA path can take their inputs from it without sharing any
of the computation under test.

Recipe (data model of Sec. II: Y = X_bar + E with X_bar low-rank on graphs,
E noise plus sparse gross errors; the cluster structure follows the
clustering experiments of Sec. VII):

* U in R^{p x r} with i.i.d. N(0, 1) entries.
* C cluster centres mu_1..mu_C in R^r, i.i.d. N(0, 1).
* Column labels j mod C, then a seeded shuffle (balanced clusters).
* Latent columns z_j = mu_{label(j)} + spread * N(0, I_r).
* X_bar = U Z scaled to unit RMS.
* Y = X_bar + noise * N(0, 1) entrywise.
* Each entry is independently replaced, with probability ``frac``, by a
  U(-1, 1) gross error.

The numpy path (``make_instance``) draws in FP64 and returns FP32 arrays.
``make_instance_torch`` follows the same recipe with torch's generator on
any device; it exists for the 8 GB workload, which is too large to build
on the host in reasonable time.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_instance", "make_instance_torch", "CONFIGS", "batched_instances",
           "heldout_entries", "latent_points"]


def make_instance(seed: int, p: int, n: int, r: int, C: int, frac: float,
                  noise: float = 0.01, spread: float = 0.1):
    """Return (Y, X_bar, labels): Y float32 (p, n), X_bar float64 (p, n)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((p, r))
    centres = rng.standard_normal((C, r))
    labels = rng.permutation(np.arange(n) % C)
    Z = centres[labels].T + spread * rng.standard_normal((r, n))
    Xb = U @ Z
    Xb /= np.sqrt(np.mean(Xb * Xb))
    Y = Xb + noise * rng.standard_normal((p, n))
    mask = rng.random((p, n)) < frac
    Y[mask] = rng.uniform(-1.0, 1.0, int(mask.sum()))
    return Y.astype(np.float32), Xb, labels


def make_instance_torch(seed: int, p: int, n: int, r: int, C: int, frac: float,
                        noise: float = 0.01, spread: float = 0.1,
                        device: str = "cuda", chunk_rows: int = 2048):
    """Same recipe as :func:`make_instance`, drawn with torch on ``device``.

    Returns Y as a float32 (p, n) tensor on ``device``. Rows are produced in
    chunks so that peak extra memory stays a few chunk sizes.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    U = torch.randn(p, r, generator=g, device=device, dtype=torch.float32)
    centres = torch.randn(C, r, generator=g, device=device, dtype=torch.float32)
    labels = torch.arange(n, device=device) % C
    labels = labels[torch.randperm(n, generator=g, device=device)]
    Z = centres[labels].T + spread * torch.randn(r, n, generator=g, device=device)
    # unit RMS of U Z: E[(UZ)_ij^2] over the drawn U, Z computed exactly as
    # trace(U^T U Z Z^T) / (p n) without forming U Z twice.
    ms = float(((U.double().T @ U.double()) * (Z.double() @ Z.double().T)).sum()) / (p * n)
    scale = 1.0 / ms ** 0.5
    Y = torch.empty(p, n, device=device, dtype=torch.float32)
    for r0 in range(0, p, chunk_rows):
        r1 = min(p, r0 + chunk_rows)
        blk = (U[r0:r1] @ Z) * scale
        blk += noise * torch.randn(r1 - r0, n, generator=g, device=device)
        mask = torch.rand(r1 - r0, n, generator=g, device=device) < frac
        gross = torch.rand(r1 - r0, n, generator=g, device=device) * 2.0 - 1.0
        Y[r0:r1] = torch.where(mask, gross, blk)
    return Y


# Single-instance workloads by size: shapes, ranks, cluster counts,
# corruption, graph K, sampling fractions, FISTA iteration counts and gamma
# values (the 64-instance workload is batched_instances below).
CONFIGS = {
    "small_256x512": dict(p=256, n=512, r=5, C=4, frac=0.05, K=10, fr=0.5, fc=0.5,
               J=200, gamma_r=1.0, gamma_c=1.0, cg_tol=1e-6),
    "bench_10304x1000": dict(p=10304, n=1000, r=10, C=10, frac=0.05, K=10, fr=0.25, fc=0.25,
               J=300, gamma_r=1.0, gamma_c=1.0, cg_tol=1e-6),
    "large_20000x100000": dict(p=20000, n=100000, r=20, C=50, frac=0.02, K=10, fr=0.1, fc=0.1,
               J=300, gamma_r=1.0, gamma_c=1.0, cg_tol=1e-6),
}


def batched_instances(count: int = 64, seed: int = 1000):
    """Sizes and gammas of the batched workload: p ~ U[500, 8000],
    n ~ U[200, 5000], rank ~ U{3..15}, gamma_r x gamma_c over an 8-point log
    grid on [0.1, 10] (all 64 pairs for count=64)."""
    rng = np.random.default_rng(seed)
    grid = np.logspace(-1, 1, 8)
    out = []
    for i in range(count):
        p = int(rng.integers(500, 8001))
        n = int(rng.integers(200, 5001))
        r = int(rng.integers(3, 16))
        out.append(dict(seed=seed + i, p=p, n=n, r=r, C=r, frac=0.05, K=10,
                        fr=0.25, fc=0.25, J=300,
                        gamma_r=float(grid[i % 8]), gamma_c=float(grid[(i // 8) % 8])))
    return out


def heldout_entries(seed: int, p: int, n: int, count: int, omega_r, omega_c):
    """`count` distinct entries (i, j) of a p x n matrix drawn uniformly among
    those outside the sampled block omega_r x omega_c (the held-out entries
    of a reconstruction loss). Returns (rows, cols) as int32 arrays."""
    rng = np.random.default_rng(seed)
    inside = np.zeros((p, n), dtype=bool)
    inside[np.ix_(np.asarray(omega_r), np.asarray(omega_c))] = True
    cand = np.flatnonzero(~inside.ravel())
    pick = np.sort(rng.choice(cand, size=min(count, cand.size), replace=False))
    return (pick // n).astype(np.int32), (pick % n).astype(np.int32)


def latent_points(seed: int, N: int, dim: int = 20, C: int = 1, spread: float = 0.1):
    """N seeded points in R^dim (float32), in C balanced clusters: centres
    i.i.d. N(0, 1), labels j mod C shuffled, point = centre + spread N(0, I)
    (C = 1: one N(0, I) cloud, spread ignored). The same model as the latent
    rows of U (C = 1) and columns of Z (C > 1) of ``make_instance``, for
    graphs whose size matches a workload but whose points are cheap to
    search."""
    rng = np.random.default_rng(seed)
    if C <= 1:
        return rng.standard_normal((N, dim)).astype(np.float32)
    centres = rng.standard_normal((C, dim))
    labels = rng.permutation(np.arange(N) % C)
    return (centres[labels] + spread * rng.standard_normal((N, dim))).astype(np.float32)
