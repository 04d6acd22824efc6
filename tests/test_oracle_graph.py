"""Pins for the oracle's sampling, kNN, kernel width and Laplacians.

Each check ties the oracle to something other than itself: hand-derived
values (tests/golden), scipy's exact k-d tree, the published SplitMix64
outputs, and the algebraic invariants of Laplacians (Sec. I).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial import cKDTree

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_splitmix64_published_outputs(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "splitmix64.json")))
    # state0 = seed ^ (gamma * (stream + 1)); choose seed so that state0 = 0
    outs = O.splitmix64_outputs(O.GOLDEN_GAMMA, 0, 3)
    assert [f"{x:016x}" for x in outs] == g["outputs_hex"]


def test_sample_indices_basic():
    om = O.sample_indices(7, 1000, 250, 0)
    assert len(om) == 250 and len(set(om.tolist())) == 250
    assert np.all(np.diff(om) > 0) and om.min() >= 0 and om.max() < 1000
    assert not np.array_equal(om, O.sample_indices(7, 1000, 250, 1))
    assert np.array_equal(O.sample_indices(3, 10, 10, 0), np.arange(10))
    assert len(O.sample_indices(3, 10, 0, 0)) == 0


def test_sample_indices_uniform():
    # Uniform without replacement (Eq. Mc): each index is included with
    # probability rho/N; chi-square over 4000 draws of 5 out of 20.
    N, rho, T = 20, 5, 4000
    cnt = np.zeros(N)
    for s in range(T):
        cnt[O.sample_indices(s, N, rho, 0)] += 1
    exp = T * rho / N
    chi2 = np.sum((cnt - exp) ** 2 / exp)
    assert chi2 < 45.3  # 99.9% quantile of chi2 with 19 dof
    # pairs are uniform too: a fixed pair appears with prob rho(rho-1)/(N(N-1))
    pair = sum(1 for s in range(T) if {0, 1} <= set(O.sample_indices(s, N, rho, 0).tolist()))
    pexp = T * rho * (rho - 1) / (N * (N - 1))
    assert abs(pair - pexp) < 4.5 * math.sqrt(pexp)


def test_sample_matrix_is_index_gather():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((9, 13))
    om_r, om_c = np.array([1, 4, 8]), np.array([0, 2, 3, 12])
    assert np.array_equal(O.sample_matrix(Y, om_r, om_c), Y[np.ix_(om_r, om_c)])


@pytest.mark.parametrize("case", range(3))
def test_graph_hand_derived(golden_dir, case):
    g = json.load(open(os.path.join(golden_dir, "graph_1d.json")))["cases"][case]
    P = np.array(g["points"])
    K = g["K"]
    idx, d2 = O.knn_bruteforce(P, K)
    assert idx.tolist() == g["knn"]
    assert np.allclose(d2, g["knn_d2"], rtol=0, atol=0)
    s2 = O.sigma2_mean(d2)
    assert s2 == pytest.approx(g["sigma2"], rel=1e-15)
    N = len(P)
    for lap in (O.LAP_COMBINATORIAL, O.LAP_NORMALIZED):
        L, W = O.laplacian_from_knn(idx, d2, N, s2, lap)
        Wd = np.zeros((N, N))
        for key, dd in g["edges_d2"].items():
            a, b = map(int, key.split("-"))
            Wd[a, b] = Wd[b, a] = math.exp(-dd / g["sigma2"])
        assert np.allclose(W.toarray(), Wd, rtol=1e-15, atol=0)
        deg = Wd.sum(1)
        Ld = np.diag(deg) - Wd
        if lap == O.LAP_NORMALIZED:
            Ld = Ld / np.sqrt(np.outer(deg, deg))
        assert np.allclose(L.toarray(), Ld, rtol=1e-14, atol=1e-15)


def test_knn_matches_kdtree():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((300, 7))
    idx, d2 = O.knn_bruteforce(P, 10)
    dist, ref = cKDTree(P).query(P, 11)
    assert np.array_equal(ref[:, 0], np.arange(300))
    assert np.array_equal(idx, ref[:, 1:])
    assert np.allclose(d2, dist[:, 1:] ** 2, rtol=1e-12)


def test_knn_query_blocked_matches_kdtree():
    """The blocked single-query search (used on point sets too large to
    difference at once), including a float32 point set read through a
    transposed view, against a k-d tree; ragged last block."""
    rng = np.random.default_rng(2)
    P32 = rng.standard_normal((9, 333)).astype(np.float32)
    P = P32.T  # 333 points of dimension 9, a non-contiguous view
    dist, ref = cKDTree(P.astype(np.float64)).query(P.astype(np.float64), 13)
    for i in (0, 17, 332):
        idx, d2 = O.knn_query_blocked(P, i, 11, block=64)
        assert np.array_equal(idx, ref[i, 1:13])
        assert np.allclose(d2, dist[i, 1:13] ** 2, rtol=1e-12)


@pytest.mark.parametrize("lap", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
def test_laplacian_invariants(lap):
    rng = np.random.default_rng(2)
    P = rng.standard_normal((120, 5))
    L, W, idx, d2, s2 = O.knn_graph(P, 6, lap)
    Ld = L.toarray()
    assert np.array_equal(Ld, Ld.T)
    ev = np.linalg.eigvalsh(Ld)
    assert ev.min() > -1e-12
    deg = np.asarray(W.sum(1)).ravel()
    assert np.all(W.diagonal() == 0)
    if lap == O.LAP_COMBINATORIAL:
        assert np.abs(Ld.sum(1)).max() < 1e-12          # zero row sums
    else:
        assert np.abs(Ld @ np.sqrt(deg)).max() < 1e-12  # D^1/2 1 spans the null space
        assert np.allclose(np.diag(Ld), 1.0)
        assert ev.max() <= 2.0 + 1e-12
    # every directed kNN edge is present with the Gaussian weight, both ways
    for i in range(0, 120, 17):
        for k in range(6):
            j = idx[i, k]
            assert W[i, j] == W[j, i] == pytest.approx(math.exp(-d2[i, k] / s2), rel=1e-15)
    # and nothing else: edge count equals the size of the OR-symmetrised set
    und = {(min(i, int(j)), max(i, int(j))) for i in range(120) for j in idx[i]}
    assert W.nnz == 2 * len(und)


def test_power_norm_matches_eigvalsh():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((200, 4))
    for lap in (O.LAP_NORMALIZED, O.LAP_COMBINATORIAL):
        L, *_ = O.knn_graph(P, 8, lap)
        lmax = np.linalg.eigvalsh(L.toarray()).max()
        assert O.power_norm(L, 3000, 0) == pytest.approx(lmax, rel=1e-7)
