"""Pins for the oracle's FRPCAG objective and FISTA (Sec. IV-B, Algorithm 1).

The minimiser is tied to: a two-node closed form, an independent
bound-constrained solve of the same convex problem (L-BFGS-B on a split
formulation with a dense Kronecker operator), the l1 subgradient optimality
conditions, the gamma = 0 special case, and the Beck-Teboulle rate bound.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import oracle as O


def _two_node(y1, y2, gamma):
    Yt = np.array([[y1], [y2]])
    Lr = sp.csr_matrix(np.array([[1.0, -1.0], [-1.0, 1.0]]))
    Lc = sp.csr_matrix(np.zeros((1, 1)))
    return Yt, Lr, Lc


@pytest.mark.parametrize("y2,gamma,fstar", [
    (3.0, 1.0, 3.0 - 0.25),     # d > 1/(2 gamma): F* = d - 1/(4 gamma)
    (0.3, 1.0, 0.09),           # d <= 1/(2 gamma): X* = Y~, F* = gamma d^2
    (2.0, 4.0, 2.0 - 1.0 / 16),
])
def test_two_node_closed_form(y2, gamma, fstar):
    Yt, Lr, Lc = _two_node(0.0, y2, gamma)
    lam = O.fista_step(gamma, 0.0, 2.0, 0.0)
    assert lam == pytest.approx(1.0 / (4.0 * gamma))
    X, _ = O.frpcag_fista(Yt, Lr, Lc, gamma, 0.0, lam, 5000)
    F = O.frpcag_objective(X, Yt, Lr, Lc, gamma, 0.0)
    assert F == pytest.approx(fstar, rel=1e-9, abs=1e-12)


def test_gamma_zero_returns_data():
    rng = np.random.default_rng(0)
    Yt = rng.standard_normal((12, 17))
    Lr, *_ = O.knn_graph(Yt, 3)
    Lc, *_ = O.knn_graph(Yt.T, 3)
    lam = O.fista_step(0.0, 0.0, 1.3, 1.7)
    X, info = O.frpcag_fista(Yt, Lr, Lc, 0.0, 0.0, lam, 25)
    assert np.array_equal(X, Yt) and info["iters"] == 25


def _small_problem(seed=4, rr=6, rc=7):
    rng = np.random.default_rng(seed)
    Yt = rng.standard_normal((rr, rc))
    Yt[rng.random((rr, rc)) < 0.2] += 3.0
    Lr, *_ = O.knn_graph(Yt, 2)
    Lc, *_ = O.knn_graph(Yt.T, 2)
    return Yt, Lr, Lc


def _independent_minimum(Yt, Lr, Lc, gr, gc):
    """Same convex problem, different method: X = Y~ - A + B with A, B >= 0,
    F = sum(A + B) + vec(X)^T Q vec(X), Q = gc (L_c kron I) + gr (I kron L_r)
    built densely (column-major vec), minimised by L-BFGS-B."""
    rr, rc = Yt.shape
    Q = gc * np.kron(Lc.toarray(), np.eye(rr)) + gr * np.kron(np.eye(rc), Lr.toarray())
    y = Yt.reshape(-1, order="F")
    m = y.size

    def f(z):
        a, b = z[:m], z[m:]
        x = y - a + b
        Qx = Q @ x
        return a.sum() + b.sum() + x @ Qx, np.concatenate([1 - 2 * Qx, 1 + 2 * Qx])

    r = so.minimize(f, np.zeros(2 * m), jac=True, method="L-BFGS-B",
                    bounds=[(0, None)] * (2 * m),
                    options=dict(maxiter=50000, ftol=1e-16, gtol=1e-13, maxcor=50))
    return r.fun


def test_matches_independent_solver():
    Yt, Lr, Lc = _small_problem()
    gr, gc = 0.7, 1.3
    lam = O.fista_step(gr, gc, O.power_norm(Lr, 2000), O.power_norm(Lc, 2000))
    X, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, 20000)
    F = O.frpcag_objective(X, Yt, Lr, Lc, gr, gc)
    Fi = _independent_minimum(Yt, Lr, Lc, gr, gc)
    assert F == pytest.approx(Fi, rel=1e-8)


def test_l1_optimality_conditions():
    # At a minimiser of |Y~ - X|_1 + g(X): -grad g(X)_ij = -sgn(X_ij - Y~_ij)
    # where X_ij != Y~_ij and |grad g(X)_ij| <= 1 where X_ij = Y~_ij, with
    # grad g built here from the dense trace form d/dX [gc tr(X Lc X^T) + gr tr(X^T Lr X)].
    Yt, Lr, Lc = _small_problem(seed=5, rr=9, rc=11)
    gr, gc = 0.4, 0.9
    lam = O.fista_step(gr, gc, O.power_norm(Lr, 2000), O.power_norm(Lc, 2000))
    X, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, 20000)
    Lrd, Lcd = Lr.toarray(), Lc.toarray()
    G = gc * (X @ (Lcd + Lcd.T)) + gr * ((Lrd + Lrd.T) @ X)
    on = np.abs(X - Yt) > 1e-9
    assert np.max(np.abs(G[on] - np.sign(Yt - X)[on])) < 1e-4
    assert np.max(np.maximum(np.abs(G[~on]) - 1.0, 0.0), initial=0.0) < 1e-4
    assert on.any() and (~on).any()


def test_rate_bound():
    # Beck & Teboulle (2009), Thm 4.4: F(S_j) - F* <= 2 L |S_0 - X*|^2 / (j+1)^2
    Yt, Lr, Lc = _small_problem(seed=6, rr=8, rc=10)
    gr, gc = 1.0, 1.0
    nr, nc = O.power_norm(Lr, 3000), O.power_norm(Lc, 3000)
    beta = 2 * gr * nr + 2 * gc * nc
    lam = 1.0 / beta
    Xs, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, 30000)
    Fs = O.frpcag_objective(Xs, Yt, Lr, Lc, gr, gc)
    R2 = np.sum((Yt - Xs) ** 2)
    for j in (1, 2, 5, 10, 50, 200):
        Xj, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, j)
        gap = O.frpcag_objective(Xj, Yt, Lr, Lc, gr, gc) - Fs
        assert gap <= 2 * beta * R2 / (j + 1) ** 2 + 1e-9


def test_stopping_rule_stops_early():
    Yt, Lr, Lc = _small_problem(seed=7)
    lam = O.fista_step(1, 1, O.power_norm(Lr), O.power_norm(Lc))
    X, info = O.frpcag_fista(Yt, Lr, Lc, 1.0, 1.0, lam, 100000, eps=1e-12)
    assert info["iters"] < 100000 and info["rel_change"] < 1e-12
