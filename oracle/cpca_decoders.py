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

Approximate decoders 2 and 3 (appendix, "Other Approximate Decoders"):
with the full data Y available, only one subspace is upsampled (Lemma 1,
Eq. Uupsample, then unit columns as in Algorithm 2 step 4) and
X = U U^T Y (decoder 2) or X = Y V V^T (decoder 3). Pinned by the exact
recovery of exactly low-rank data when every row (column) is sampled, by
the paper's V-route X = U Sigma~ c V^T with V = Y^T U Sigma~^-1 / c, and by
the symmetry between the two decoders under transposition.

Clustering decoder (Sec. V-D, Algorithm 3): k-means on the columns of X~
(rho_c points in R^{rho_r}) gives one-hot labels C~ (rho_c x k); every
column of C is the minimiser of c^T L_c c subject to c(Omega_c) = c~
(Lemma 1, by PCG); each node takes the label of the largest entry of its
row (ties: the lowest label). The paper does not say how k-means starts or
stops; the reading is Lloyd's iteration from k distinct columns drawn with
the sampling generator (stream KMEANS_STREAM, ascending index order),
nearest centre by squared Euclidean distance (ties: the lowest centre),
centres the means of their points (an empty cluster keeps its centre),
until no assignment changes. Pinned by well-separated blobs (the
generating partition, up to a relabelling), Lloyd's fixed point at the end
(every point at its nearest centre, centres at their means), the
non-increasing k-means objective, and graphs made of components whose
sampled nodes share a label (every node of a component gets that label).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .cpca_oracle import pcg, sample_indices, svd_rank, upsample_subspace

__all__ = ["selection_matrix", "alternate_objective", "alternate_decode", "approx_decode_projected",
           "kmeans_columns", "cluster_decode", "KMEANS_STREAM"]

KMEANS_STREAM = 5  # SplitMix64 stream of the k-means initial centres


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


def alternate_decode(Xt, omega_r, omega_c, p: int, n: int, Lr, Lc, gr_bar: float, gc_bar: float,
                     tol: float | None = None):
    """Minimiser of Eq. (alternatedecoder): the normal equations in
    Kronecker form on vec(X) taken row by row (index i * n + j),

        (D_r kron D_c + gc_bar I_p kron L_c^T + gr_bar L_r kron I_n) vec(X)
            = vec(M_r^T X~ M_c^T),

    solved by a sparse direct factorisation (tol None; exact, for small
    sizes: the factors fill in quickly) or by this oracle's FP64 Jacobi PCG
    to relative residual tol (the same system; for larger test sizes).
    Returns X (p x n)."""
    Mr = selection_matrix(omega_r, p)
    Mc = selection_matrix(omega_c, n).T
    Dr = (Mr.T @ Mr).tocsr()
    Dc = (Mc @ Mc.T).tocsr()
    Lr = sp.csr_matrix(Lr, dtype=np.float64)
    Lc = sp.csr_matrix(Lc, dtype=np.float64)
    A = (sp.kron(Dr, Dc) + gc_bar * sp.kron(sp.identity(p), Lc.T) + gr_bar * sp.kron(Lr, sp.identity(n))).tocsc()
    B = Mr.T @ sp.csr_matrix(np.asarray(Xt, dtype=np.float64)) @ Mc.T
    b = np.asarray(B.todense()).reshape(-1)
    if tol is None:
        x = spla.spsolve(A, b)
    else:
        x, _, _ = pcg(A.tocsr(), b, tol=tol, maxit=100 * p * n)
    return np.asarray(x).reshape(p, n)


def approx_decode_projected(Y, Xt, omega_r, omega_c, Lr, Lc, side: int, ratio: float = 0.1,
                            tol: float = 1e-6, k_override: int | None = None, maxit: int | None = None):
    """Approximate decoder 2 (side 0) or 3 (side 1). Steps: SVD of X~ and
    the rank k (Algorithm 2 steps 1-2); upsample U~ on L_r (side 0) or V~ on
    L_c (side 1) (Lemma 1); unit columns (Algorithm 2 step 4); then
    X = U (U^T Y) or X = (Y V) V^T. Returns (X, basis, k)."""
    Y = np.asarray(Y, dtype=np.float64)
    Ut, s, Vh, k = svd_rank(Xt, ratio)
    if k_override is not None:
        k = int(k_override)
    if side == 0:
        B, _, _ = upsample_subspace(Lr, omega_r, Ut[:, :k], tol, maxit)
    else:
        B, _, _ = upsample_subspace(Lc, omega_c, Vh[:k].T, tol, maxit)
    B = B / np.linalg.norm(B, axis=0, keepdims=True)
    X = B @ (B.T @ Y) if side == 0 else (Y @ B) @ B.T
    return X, B, k


def kmeans_columns(Xt, k: int, seed: int = 0, max_iter: int = 100):
    """Lloyd's k-means on the columns of X~ (see the module docstring).
    Returns (labels (rho_c,), centres (k x rho_r), assignment steps,
    objective after each assignment step)."""
    P = np.asarray(Xt, dtype=np.float64).T  # rho_c points, one per row
    m = P.shape[0]
    C = P[sample_indices(seed, m, k, KMEANS_STREAM)].copy()
    labels = None
    objective = []
    steps = 0
    for _ in range(max_iter):
        d = np.zeros((m, k))
        for c in range(k):
            diff = P - C[c]
            d[:, c] = np.sum(diff * diff, axis=1)
        new = np.argmin(d, axis=1)  # first minimum: the lowest centre on ties
        steps += 1
        objective.append(float(d[np.arange(m), new].sum()))
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for c in range(k):
            members = labels == c
            if members.any():
                C[c] = P[members].mean(axis=0)
    return labels, C, steps, objective


def cluster_decode(Xt, omega_c, n: int, Lc, k: int, seed: int = 0, tol: float = 1e-6,
                   kmeans_iters: int = 100, maxit: int | None = None):
    """Algorithm 3. Returns (labels (n,), C (n x k), k-means labels of X~'s
    columns)."""
    lab_t, _, _, _ = kmeans_columns(Xt, k, seed, kmeans_iters)
    Ct = np.zeros((len(lab_t), k))
    Ct[np.arange(len(lab_t)), lab_t] = 1.0
    C, _, _ = upsample_subspace(Lc, omega_c, Ct, tol, maxit)
    return np.argmax(C, axis=1), C, lab_t
