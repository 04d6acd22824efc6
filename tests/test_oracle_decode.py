"""Pins for the oracle's approximate decoder (Sec. V-C, Lemma 1, Algorithm 2).

Ties: a dense Kronecker-form solve, a sparse direct solve, the variational
definition of Lemma 1 (no feasible perturbation lowers the energy), the
regularised closed forms of Sec. V-C as gamma' -> 0, Eckart-Young under full
sampling, exact recovery of a constant matrix, and component-wise constant
extension for the combinatorial Laplacian.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle as O


def _graph(N, seed, lap=O.LAP_NORMALIZED, K=4):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((N, 3))
    L, *_ = O.knn_graph(P, K, lap)
    return L


def test_pcg_matches_direct_solve():
    L = _graph(60, 0, O.LAP_COMBINATORIAL)
    A = sp.csr_matrix(L[5:][:, 5:])
    B = np.random.default_rng(1).standard_normal((55, 3))
    X, its, res = O.pcg(A, B, tol=1e-12)
    assert np.allclose(X, spl.spsolve(sp.csc_matrix(A), B), rtol=1e-9, atol=1e-10)
    assert np.all(res <= 1e-12)


@pytest.mark.parametrize("lap", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
def test_upsample_matches_kronecker_solve(lap):
    N, k = 30, 3
    L = _graph(N, 2, lap).toarray()
    om = O.sample_indices(5, N, 8, 0)
    R = np.random.default_rng(3).standard_normal((len(om), k))
    S, *_ = O.upsample_subspace(sp.csr_matrix(L), om, R, tol=1e-13)
    a = np.setdiff1d(np.arange(N), om)
    # (I_k kron L_aa) vec(S_a) = -vec(L_ab R), column-major vec
    Akron = np.kron(np.eye(k), L[np.ix_(a, a)])
    rhs = -(L[np.ix_(a, om)] @ R).reshape(-1, order="F")
    Sa = np.linalg.solve(Akron, rhs).reshape(len(a), k, order="F")
    assert np.allclose(S[a], Sa, rtol=1e-9, atol=1e-11)
    assert np.array_equal(S[om], R)  # constraint M S = R holds exactly


def test_upsample_minimises_energy():
    # Lemma 1: S minimises tr(S^T L S) over S with S(omega,:) = R.
    N = 40
    L = _graph(N, 4).toarray()
    om = O.sample_indices(9, N, 10, 0)
    R = np.random.default_rng(5).standard_normal((10, 2))
    S, *_ = O.upsample_subspace(sp.csr_matrix(L), om, R, tol=1e-14)
    E0 = np.trace(S.T @ L @ S)
    rng = np.random.default_rng(6)
    a = np.setdiff1d(np.arange(N), om)
    for _ in range(20):
        D = np.zeros_like(S)
        D[a] = 1e-3 * rng.standard_normal((len(a), 2))
        assert np.trace((S + D).T @ L @ (S + D)) > E0


def test_regularised_closed_form_limit():
    # Sec. V-C: U = (M_r^T M_r + g' L_r)^{-1} M_r^T U~ tends to Lemma 1 as g' -> 0.
    N = 35
    L = _graph(N, 7).toarray()
    om = O.sample_indices(2, N, 9, 0)
    R = np.random.default_rng(8).standard_normal((9, 2))
    M = np.zeros((9, N))
    M[np.arange(9), om] = 1.0
    g = 1e-8
    Ureg = np.linalg.solve(M.T @ M + g * L, M.T @ R)
    S, *_ = O.upsample_subspace(sp.csr_matrix(L), om, R, tol=1e-14)
    assert np.allclose(Ureg, S, rtol=1e-5, atol=1e-6)


def test_full_sampling_is_truncated_svd():
    # Omega = everything: U = U~, V = V~, Sigma = Sigma~, so X is the best
    # rank-k approximation of X~ (Eckart-Young): |X~ - X|_F^2 = sum_{i>k} s_i^2.
    rng = np.random.default_rng(9)
    Xt = rng.standard_normal((20, 3)) @ np.diag([10.0, 5.0, 2.0]) @ rng.standard_normal((3, 25))
    Xt += 0.01 * rng.standard_normal(Xt.shape)
    Lr, Lc = _graph(20, 10), _graph(25, 11)
    d = O.approx_decode(Xt, np.arange(20), np.arange(25), 20, 25, Lr, Lc)
    s = np.sqrt(np.clip(np.linalg.eigvalsh(Xt.T @ Xt), 0, None))[::-1]
    k = int(np.sum(s / s[0] >= 0.1))
    assert d["k"] == k == 3
    assert np.sum((Xt - d["X"]) ** 2) == pytest.approx(np.sum(s[k:] ** 2), rel=1e-8)
    assert np.linalg.matrix_rank(d["X"], tol=1e-8 * s[0]) == k


def test_constant_matrix_recovered_exactly():
    # Combinatorial L annihilates constants, so the harmonic extension of a
    # constant subspace vector is constant; with the scale of step 5 the
    # decoder returns the all-ones matrix from its sampled corner.
    p, n = 30, 40
    Lr, Lc = _graph(p, 12, O.LAP_COMBINATORIAL), _graph(n, 13, O.LAP_COMBINATORIAL)
    om_r, om_c = O.sample_indices(1, p, 10, 0), O.sample_indices(1, n, 12, 1)
    d = O.approx_decode(np.ones((10, 12)), om_r, om_c, p, n, Lr, Lc, tol=1e-13)
    assert d["k"] == 1
    assert np.allclose(d["X"], 1.0, rtol=1e-9)


def test_component_constant_extension():
    # Two disconnected components; values constant per component on the
    # sampled nodes extend as the same constants (combinatorial L).
    rng = np.random.default_rng(14)
    P = np.vstack([rng.standard_normal((20, 2)), 100.0 + rng.standard_normal((20, 2))])
    L, *_ = O.knn_graph(P, 4, O.LAP_COMBINATORIAL)
    om = np.array([0, 3, 7, 21, 30])
    R = np.array([[2.0], [2.0], [2.0], [-5.0], [-5.0]])
    S, *_ = O.upsample_subspace(L, om, R, tol=1e-13)
    assert np.allclose(S[:20], 2.0) and np.allclose(S[20:], -5.0)


def test_decoder_scale_factor():
    # Step 5 scales Sigma~ by sqrt(n p / (rho_r rho_c (1 - delta))).
    p, n = 30, 40
    Lr, Lc = _graph(p, 12, O.LAP_COMBINATORIAL), _graph(n, 13, O.LAP_COMBINATORIAL)
    om_r, om_c = O.sample_indices(1, p, 10, 0), O.sample_indices(1, n, 12, 1)
    d0 = O.approx_decode(np.ones((10, 12)), om_r, om_c, p, n, Lr, Lc, tol=1e-13)
    d1 = O.approx_decode(np.ones((10, 12)), om_r, om_c, p, n, Lr, Lc, tol=1e-13, delta=0.75)
    assert d0["sigma"][0] == pytest.approx(math.sqrt(p * n), rel=1e-12)
    assert np.allclose(d1["X"], 2.0 * d0["X"], rtol=1e-12)
