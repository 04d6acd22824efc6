"""Pins for the C restatement of Algorithm 1 (oracle/fista_c.c).

It must reproduce the numpy oracle (itself pinned in test_oracle_fista.py
against closed forms, an independent solve and the KKT conditions): same
iterates on small problems of both Laplacian kinds, with and without the
stopping rule, for any thread count; gamma = 0 returns Y~ exactly.
"""
import numpy as np
import pytest

import oracle as O
from oracle.cpca_fista_c import frpcag_fista_c


def _problem(seed, rr, rc, lap):
    rng = np.random.default_rng(seed)
    Yt = rng.standard_normal((rr, rc))
    Yt[rng.random((rr, rc)) < 0.1] += 3.0
    Lr, *_ = O.knn_graph(Yt, 4, lap)
    Lc, *_ = O.knn_graph(Yt.T, 5, lap)
    return Yt, Lr, Lc


@pytest.mark.parametrize("lap", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
@pytest.mark.parametrize("eps", [0.0, 1e-9])
def test_matches_numpy_oracle(lap, eps):
    Yt, Lr, Lc = _problem(3, 37, 53, lap)
    lam = O.fista_step(1.3, 0.7, O.power_norm(Lr, 200, 0, 2), O.power_norm(Lc, 200, 0, 3))
    a, ia = O.frpcag_fista(Yt, Lr, Lc, 1.3, 0.7, lam, 150, eps)
    b, ib = frpcag_fista_c(Yt, Lr, Lc, 1.3, 0.7, lam, 150, eps, threads=3)
    assert ia["iters"] == ib["iters"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    assert ib["rel_change"] == pytest.approx(ia["rel_change"], rel=1e-9)


def test_thread_count_does_not_change_iterates():
    Yt, Lr, Lc = _problem(5, 64, 41, O.LAP_NORMALIZED)
    lam = O.fista_step(1.0, 1.0, O.power_norm(Lr, 200, 0, 2), O.power_norm(Lc, 200, 0, 3))
    a, _ = frpcag_fista_c(Yt, Lr, Lc, 1.0, 1.0, lam, 60, threads=1)
    b, _ = frpcag_fista_c(Yt, Lr, Lc, 1.0, 1.0, lam, 60, threads=4)
    assert np.array_equal(a, b)


def test_gamma_zero_returns_data():
    Yt, Lr, Lc = _problem(7, 12, 17, O.LAP_NORMALIZED)
    X, info = frpcag_fista_c(Yt, Lr, Lc, 0.0, 0.0, 1.0, 25)
    assert np.array_equal(X, Yt) and info["iters"] == 25


def test_one_sided_products():
    """Only one of the two graph terms active: each product alone against
    the numpy oracle's scipy product."""
    Yt, Lr, Lc = _problem(9, 20, 30, O.LAP_COMBINATORIAL)
    for gr, gc in ((1.0, 0.0), (0.0, 1.0)):
        lam = O.fista_step(gr, gc, O.power_norm(Lr, 200, 0, 2), O.power_norm(Lc, 200, 0, 3))
        a, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, 40)
        b, _ = frpcag_fista_c(Yt, Lr, Lc, gr, gc, lam, 40)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
