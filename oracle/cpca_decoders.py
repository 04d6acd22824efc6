"""FP64 restatements of the paper's other decoders (test infrastructure only).

Alternate decoder (Sec. V-B, Eq. alternatedecoder): the full low-rank
matrix X (p x n) minimising

    |M_r X M_c - X~|_F^2 + gc_bar tr(X L_c X^T) + gr_bar tr(X^T L_r X),

with M_r the rho_r x p row-selection matrix of Omega_r and M_c the
n x rho_c column-selection matrix of Omega_c (Sec. III, Eq. Mc). The
paper leaves gr_bar and gc_bar to the user (Theorem 2 ties them to a gamma
and the spectral gaps). Setting the gradient to zero (L_r, L_c symmetric)
gives the normal equations

    D_r X D_c + gc_bar X L_c + gr_bar L_r X = M_r^T X~ M_c^T,

D_r = M_r^T M_r and D_c = M_c M_c^T the 0/1 diagonals of the sampled rows
and columns; the oracle solves them exactly (sparse direct solve of the
Kronecker form), since the objective is a convex quadratic whose
minimiser is that solution. Parity pinned by tests/test_oracle_decoders.py:
closed form (full sampling, no regularisation), vanishing central
differences of the objective as written above, an independent stacked
least-squares solve through incidence factors L = G^T G, and the
transpose symmetry of the problem.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = ["selection_matrix", "alternate_objective", "alternate_decode"]


def selection_matrix(omega: np.ndarray, N: int) -> sp.csr_matrix:
    """M (len(omega) x N): row t has a one in column omega[t] (Eq. Mc)."""
    omega = np.asarray(omega, dtype=np.int64)
    m = len(omega)
    return sp.csr_matrix((np.ones(m), (np.arange(m), omega)), shape=(m, N))


def alternate_objective(X, Xt, omega_r, omega_c, Lr, Lc, gr_bar: float, gc_bar: float) -> float:
    """The objective of Eq. (alternatedecoder) at X, term by term."""
    X = np.asarray(X, dtype=np.float64)
    p, n = X.shape
    Mr = selection_matrix(omega_r, p)        # rho_r x p
    Mc = selection_matrix(omega_c, n).T      # n x rho_c
    fit = Mr @ X @ Mc - np.asarray(Xt, dtype=np.float64)
    Lr = sp.csr_matrix(Lr)
    Lc = sp.csr_matrix(Lc)
    return float(np.sum(fit * fit) + gc_bar * np.trace(X @ (Lc @ X.T)) + gr_bar * np.trace(X.T @ (Lr @ X)))


def alternate_decode(Xt, omega_r, omega_c, p: int, n: int, Lr, Lc, gr_bar: float, gc_bar: float):
    """Exact minimiser of Eq. (alternatedecoder): the normal equations in
    Kronecker form on vec(X) taken row by row (index i * n + j),

        (D_r kron D_c + gc_bar I_p kron L_c^T + gr_bar L_r kron I_n) vec(X)
            = vec(M_r^T X~ M_c^T),

    solved by a sparse direct factorisation. Returns X (p x n)."""
    Mr = selection_matrix(omega_r, p)
    Mc = selection_matrix(omega_c, n).T
    Dr = (Mr.T @ Mr).tocsr()
    Dc = (Mc @ Mc.T).tocsr()
    Lr = sp.csr_matrix(Lr, dtype=np.float64)
    Lc = sp.csr_matrix(Lc, dtype=np.float64)
    A = (sp.kron(Dr, Dc) + gc_bar * sp.kron(sp.identity(p), Lc.T) + gr_bar * sp.kron(Lr, sp.identity(n))).tocsc()
    B = Mr.T @ sp.csr_matrix(np.asarray(Xt, dtype=np.float64)) @ Mc.T
    x = spla.spsolve(A, np.asarray(B.todense()).reshape(-1))
    return np.asarray(x).reshape(p, n)
