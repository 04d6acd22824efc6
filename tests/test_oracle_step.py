"""Pins for the step-size reading (Sec. IV-B: lambda = 1/beta',
beta' = 2 gamma_c |L_c|_2 + 2 gamma_r |L_r|_2) at the workloads' sizes.

|L|_2 is the Rayleigh quotient after 200 power iterations from the seeded
start vector (oracle.power_norm; the library computes the same estimate).
A Rayleigh quotient never exceeds the largest eigenvalue, so beta' can fall
below the Lipschitz constant beta of the smooth part. These tests measure
that gap against ARPACK (scipy eigsh) on the compressed graphs of the
10304 x 1000 workload and of a 2000 x 10000 sampled matrix of the 8 GB
workload's model, and pin the consequence: FISTA with a step up to 1%
above 1/beta reaches the same minimiser as with the exact step.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import gen
import oracle as O
from tests._oracle_knn import oracle_knn_graph


def _lam_max(L):
    return float(sla.eigsh(L, k=1, which="LA", tol=1e-14)[0][0])


def _gap(L, stream):
    lm = _lam_max(L)
    rq = O.power_norm(L, 200, 0, stream)
    return lm, rq, (lm - rq) / lm


def test_power_estimate_at_10304x1000():
    cfg = gen.CONFIGS["bench_10304x1000"]
    Y, _, _ = gen.make_instance(0, cfg["p"], cfg["n"], cfg["r"], cfg["C"], cfg["frac"])
    rr, rc = int(cfg["p"] * cfg["fr"] + 0.5), int(cfg["n"] * cfg["fc"] + 0.5)
    Yt = Y[np.ix_(O.sample_indices(0, cfg["p"], rr, 0), O.sample_indices(0, cfg["n"], rc, 1))]
    for P, stream in ((Yt, 2), (Yt.T, 3)):
        L, *_ = oracle_knn_graph(P, cfg["K"])
        lm, rq, gap = _gap(L, stream)
        assert rq <= lm * (1 + 1e-12)  # a Rayleigh quotient
        assert 0.0 <= gap < 2e-3      # measured 1.4e-3 (rows), 1.0e-3 (columns)
        # more iterations close the gap (the estimate converges to |L|_2)
        assert (lm - O.power_norm(L, 1000, 0, stream)) / lm < gap / 10


def test_power_estimate_at_2000x10000():
    Yt, _, _ = gen.make_instance(0, 2000, 10000, 20, 50, 0.02)
    for P, stream in ((Yt, 2), (Yt.T, 3)):
        L, *_ = oracle_knn_graph(P, 10)
        lm, rq, gap = _gap(L, stream)
        assert rq <= lm * (1 + 1e-12)
        assert 0.0 <= gap < 1e-2      # measured 7.0e-3 (rows), 2.1e-3 (columns)


@pytest.mark.parametrize("under", [0.0, 0.01])
def test_step_slightly_above_one_over_beta_reaches_the_minimiser(under):
    """beta' = (1 - under) beta: the same objective at convergence and the
    l1 optimality conditions, as with the exact step. (On each eigen-
    direction of the quadratic part, FISTA's momentum recurrence keeps its
    roots inside the unit circle for steps below 4/(3 beta).)"""
    rng = np.random.default_rng(21)
    Yt = rng.standard_normal((9, 12))
    Yt[rng.random(Yt.shape) < 0.2] += 3.0
    Lr, *_ = O.knn_graph(Yt, 3)
    Lc, *_ = O.knn_graph(Yt.T, 3)
    gr, gc = 0.8, 1.1
    beta = 2 * gr * np.linalg.eigvalsh(Lr.toarray()).max() + 2 * gc * np.linalg.eigvalsh(Lc.toarray()).max()
    X0, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, 1.0 / beta, 20000)
    X, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, 1.0 / ((1.0 - under) * beta), 20000)
    F0 = O.frpcag_objective(X0, Yt, Lr, Lc, gr, gc)
    assert O.frpcag_objective(X, Yt, Lr, Lc, gr, gc) == pytest.approx(F0, rel=1e-10)
    Lrd, Lcd = Lr.toarray(), Lc.toarray()
    G = 2 * gc * (X @ Lcd) + 2 * gr * (Lrd @ X)
    on = np.abs(X - Yt) > 1e-9
    assert np.max(np.abs(G[on] - np.sign(Yt - X)[on])) < 1e-6
    assert np.max(np.maximum(np.abs(G[~on]) - 1.0, 0.0), initial=0.0) < 1e-6
