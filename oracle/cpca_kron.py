"""FP64 Kron reduction of a graph Laplacian (test infrastructure only).

Sec. IV-A ("Graphs for Compressed data") offers, as the alternative to new
kNN graphs on the sampled matrix, the Kron reduction of the full graphs
onto the sampled nodes Omega (complement Omega-bar):

    L~ = L(Omega, Omega) - L(Omega, Omega-bar) L(Omega-bar, Omega-bar)^-1 L(Omega-bar, Omega),

the Schur complement of the unsampled block. The oracle is that definition
written out: the unsampled block is factorised once (sparse LU) and solved
for the dense right-hand side L(Omega-bar, Omega); the result is dense
(rho x rho). The unsampled block is invertible exactly when every
connected component of the graph holds a sampled node (the same condition
as Lemma 1's); otherwise the reduction is undefined and ValueError is
raised. The paper applies the reduction to "the" Laplacian; it is applied
here to whichever Laplacian the solver uses (normalised by default,
combinatorial on request), since a Schur complement does not depend on how
the matrix was made.

Pinned by tests/test_oracle_kron.py against the series and star-mesh
closed forms of electrical networks, the preservation of effective
resistances between kept nodes (from the pseudo-inverse of the full
Laplacian), the minimum-energy characterisation (an independent
least-squares solve through the incidence factor L = G^T G), the quotient
property (two reductions in a row equal one), the connectivity statement
the paper cites (Theorem III.4 of Dorfler and Bullo: two kept nodes are
coupled exactly when a path joins them through unsampled nodes only), and
Laplacian invariants (symmetry, zero row sums, non-positive off-diagonal
entries, positive semidefiniteness, the null vector D^1/2 1 of L_n).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

__all__ = ["kron_reduce", "kron_reduce_csr"]


def _check_components(L, omega: np.ndarray) -> None:
    """Every connected component of L's graph must contain a sampled node."""
    N = L.shape[0]
    A = sp.csr_matrix(L)
    A = A - sp.diags(A.diagonal())
    A.eliminate_zeros()
    ncomp, comp = csg.connected_components(A, directed=False)
    has = np.zeros(ncomp, dtype=bool)
    has[comp[omega]] = True
    if not has.all():
        raise ValueError("Kron reduction: a connected component holds no sampled node")


def kron_reduce(L, omega: np.ndarray) -> np.ndarray:
    """Dense FP64 Schur complement L~ (rho x rho) of L onto the sorted
    sampled nodes omega (Sec. IV-A)."""
    L = sp.csr_matrix(L, dtype=np.float64)
    N = L.shape[0]
    omega = np.asarray(omega, dtype=np.int64)
    if omega.size == 0 or np.any(np.diff(omega) <= 0) or omega[0] < 0 or omega[-1] >= N:
        raise ValueError("omega must be sorted, distinct and in range")
    _check_components(L, omega)
    abar = np.setdiff1d(np.arange(N), omega)
    L_bb = L[omega][:, omega].toarray()
    if abar.size == 0:
        return L_bb
    L_aa = L[abar][:, abar].tocsc()
    L_ab = L[abar][:, omega].toarray()
    L_ba = L[omega][:, abar]
    T = spla.splu(L_aa).solve(L_ab)
    return L_bb - L_ba @ T


def kron_reduce_csr(L, omega: np.ndarray) -> sp.csr_matrix:
    """kron_reduce as a CSR matrix with every entry stored (the dense
    pattern the FISTA kernels receive)."""
    Lt = kron_reduce(L, omega)
    rho = Lt.shape[0]
    return sp.csr_matrix((Lt.ravel(), np.tile(np.arange(rho), rho), np.arange(0, rho * rho + 1, rho)),
                         shape=(rho, rho))
