"""Pins of the alternate-decoder oracle (Sec. V-B, Eq. alternatedecoder)
against facts that do not reuse its normal equations."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import cpca_decoders as D


def _ring_graph(N: int, rng, extra: int = 4):
    """Connected symmetric weights: a ring plus a few random chords."""
    W = np.zeros((N, N))
    for i in range(N):
        w = rng.uniform(0.2, 1.0)
        W[i, (i + 1) % N] = W[(i + 1) % N, i] = w
    for _ in range(extra):
        i, j = rng.choice(N, 2, replace=False)
        w = rng.uniform(0.2, 1.0)
        W[i, j] = W[j, i] = w
    return W


def _incidence(W, lap_type):
    """G with G^T G = the Laplacian of W: one row per edge i < j,
    sqrt(w_ij) (e_i / s_i - e_j / s_j), s = sqrt(degree) for the
    normalised Laplacian and 1 for the combinatorial one."""
    N = W.shape[0]
    deg = W.sum(axis=1)
    s = np.sqrt(deg) if lap_type == O.LAP_NORMALIZED else np.ones(N)
    rows = []
    for i in range(N):
        for j in range(i + 1, N):
            if W[i, j] > 0:
                g = np.zeros(N)
                g[i] = 1.0 / s[i]
                g[j] = -1.0 / s[j]
                rows.append(np.sqrt(W[i, j]) * g)
    return np.array(rows)


def _problem(seed, p=6, n=5, rr=3, rc=3, lap_type=O.LAP_NORMALIZED):
    rng = np.random.default_rng(seed)
    Wr, Wc = _ring_graph(p, rng), _ring_graph(n, rng)
    Lr = O.laplacian_from_weights(sp.csr_matrix(Wr), lap_type)
    Lc = O.laplacian_from_weights(sp.csr_matrix(Wc), lap_type)
    om_r = np.sort(rng.choice(p, rr, replace=False))
    om_c = np.sort(rng.choice(n, rc, replace=False))
    Xt = rng.standard_normal((rr, rc))
    return dict(Wr=Wr, Wc=Wc, Lr=Lr, Lc=Lc, om_r=om_r, om_c=om_c, Xt=Xt, p=p, n=n)


def test_full_sampling_without_regularisation_returns_the_samples():
    rng = np.random.default_rng(0)
    p, n = 5, 4
    Xt = rng.standard_normal((p, n))
    L = O.laplacian_from_weights(sp.csr_matrix(_ring_graph(p, rng)))
    M = O.laplacian_from_weights(sp.csr_matrix(_ring_graph(n, rng)))
    X = D.alternate_decode(Xt, np.arange(p), np.arange(n), p, n, L, M, 0.0, 0.0)
    np.testing.assert_allclose(X, Xt, rtol=0, atol=1e-13)


@pytest.mark.parametrize("lap_type", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
def test_objective_is_stationary_at_the_solution(lap_type):
    q = _problem(1, lap_type=lap_type)
    gr, gc = 0.7, 1.3
    X = D.alternate_decode(q["Xt"], q["om_r"], q["om_c"], q["p"], q["n"], q["Lr"], q["Lc"], gr, gc)
    f = lambda Z: D.alternate_objective(Z, q["Xt"], q["om_r"], q["om_c"], q["Lr"], q["Lc"], gr, gc)
    f0 = f(X)
    h = 1e-4
    for i in range(q["p"]):
        for j in range(q["n"]):
            E = np.zeros_like(X)
            E[i, j] = h
            g = (f(X + E) - f(X - E)) / (2 * h)  # exact for a quadratic up to rounding
            assert abs(g) < 1e-8
            assert f(X + E) > f0 and f(X - E) > f0  # strict minimum (positive definite)


@pytest.mark.parametrize("lap_type", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
def test_matches_stacked_least_squares_through_incidence_factors(lap_type):
    """tr(X L_c X^T) = |X G_c^T|^2 and tr(X^T L_r X) = |G_r X|^2, so the
    objective is one linear least-squares problem in vec(X)."""
    q = _problem(2, p=7, n=6, rr=4, rc=3, lap_type=lap_type)
    gr, gc = 0.4, 2.0
    Gr, Gc = _incidence(q["Wr"], lap_type), _incidence(q["Wc"], lap_type)
    np.testing.assert_allclose(Gr.T @ Gr, q["Lr"].toarray(), atol=1e-12)
    np.testing.assert_allclose(Gc.T @ Gc, q["Lc"].toarray(), atol=1e-12)
    p, n = q["p"], q["n"]
    blocks, rhs = [], []
    for a, i in enumerate(q["om_r"]):          # sampled entries: X[i, j] - Xt[a, b]
        for b, j in enumerate(q["om_c"]):
            row = np.zeros(p * n)
            row[i * n + j] = 1.0
            blocks.append(row)
            rhs.append(q["Xt"][a, b])
    for i in range(p):                          # sqrt(gc) (X G_c^T)[i, e]
        for e in range(Gc.shape[0]):
            row = np.zeros(p * n)
            row[i * n:(i + 1) * n] = np.sqrt(gc) * Gc[e]
            blocks.append(row)
            rhs.append(0.0)
    for e in range(Gr.shape[0]):                # sqrt(gr) (G_r X)[e, j]
        for j in range(n):
            row = np.zeros(p * n)
            row[j::n] = np.sqrt(gr) * Gr[e]
            blocks.append(row)
            rhs.append(0.0)
    x, *_ = np.linalg.lstsq(np.array(blocks), np.array(rhs), rcond=None)
    X = D.alternate_decode(q["Xt"], q["om_r"], q["om_c"], p, n, q["Lr"], q["Lc"], gr, gc)
    np.testing.assert_allclose(X, x.reshape(p, n), rtol=0, atol=1e-10)


def test_transposed_problem_gives_the_transposed_solution():
    q = _problem(3, p=6, n=8, rr=2, rc=5)
    gr, gc = 0.9, 0.3
    X = D.alternate_decode(q["Xt"], q["om_r"], q["om_c"], q["p"], q["n"], q["Lr"], q["Lc"], gr, gc)
    XT = D.alternate_decode(q["Xt"].T, q["om_c"], q["om_r"], q["n"], q["p"], q["Lc"], q["Lr"], gc, gr)
    np.testing.assert_allclose(XT, X.T, rtol=0, atol=1e-12)


def test_pcg_mode_matches_the_direct_solve():
    q = _problem(4, p=12, n=9, rr=5, rc=4)
    X0 = D.alternate_decode(q["Xt"], q["om_r"], q["om_c"], q["p"], q["n"], q["Lr"], q["Lc"], 1.0, 1.0)
    X1 = D.alternate_decode(q["Xt"], q["om_r"], q["om_c"], q["p"], q["n"], q["Lr"], q["Lc"], 1.0, 1.0, tol=1e-13)
    np.testing.assert_allclose(X1, X0, rtol=0, atol=1e-10 * np.abs(X0).max())


# ---------------------------------------------- approximate decoders 2 and 3
def _lowrank(seed, p, n, r):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((p, r)) @ rng.standard_normal((r, n))


def _graph_of(points, K=4):
    L, *_ = O.knn_graph(points, K)
    return L


@pytest.mark.parametrize("side", [0, 1])
def test_projected_decoders_recover_exactly_lowrank_data_when_one_side_is_fully_sampled(side):
    p, n, r = 30, 24, 3
    Y = _lowrank(5, p, n, r)
    Lr, Lc = _graph_of(Y), _graph_of(Y.T)
    rng = np.random.default_rng(6)
    if side == 0:   # every row sampled: U~ spans Y's column space, no upsampling
        om_r, om_c = np.arange(p), np.sort(rng.choice(n, 10, replace=False))
    else:           # every column sampled
        om_r, om_c = np.sort(rng.choice(p, 12, replace=False)), np.arange(n)
    Xt = Y[np.ix_(om_r, om_c)]
    X, B, k = D.approx_decode_projected(Y, Xt, om_r, om_c, Lr, Lc, side, ratio=1e-6)
    assert k == r
    np.testing.assert_allclose(X, Y, rtol=0, atol=1e-10 * np.abs(Y).max())


def test_decoder2_equals_the_papers_v_route():
    """X = U Sigma~ c V^T with V = Y^T U Sigma~^-1 / c, c = sqrt(n p / (rho_r rho_c))."""
    p, n = 28, 20
    rng = np.random.default_rng(8)
    Y = _lowrank(9, p, n, 4) + 0.01 * rng.standard_normal((p, n))
    Lr, Lc = _graph_of(Y), _graph_of(Y.T)
    om_r, om_c = np.sort(rng.choice(p, 14, replace=False)), np.sort(rng.choice(n, 10, replace=False))
    Xt = Y[np.ix_(om_r, om_c)]
    X, U, k = D.approx_decode_projected(Y, Xt, om_r, om_c, Lr, Lc, 0, tol=1e-12)
    s = np.linalg.svd(Xt, compute_uv=False)[:k]
    c = np.sqrt(n * p / (len(om_r) * len(om_c)))
    V = Y.T @ U @ np.diag(1.0 / s) / c
    np.testing.assert_allclose(X, U @ np.diag(s) @ V.T * c, rtol=0, atol=1e-10 * np.abs(X).max())


def test_decoder3_is_decoder2_of_the_transposed_problem():
    p, n = 26, 22
    rng = np.random.default_rng(10)
    Y = _lowrank(11, p, n, 3) + 0.01 * rng.standard_normal((p, n))
    Lr, Lc = _graph_of(Y), _graph_of(Y.T)
    om_r, om_c = np.sort(rng.choice(p, 12, replace=False)), np.sort(rng.choice(n, 11, replace=False))
    Xt = Y[np.ix_(om_r, om_c)]
    X3, _, k3 = D.approx_decode_projected(Y, Xt, om_r, om_c, Lr, Lc, 1, tol=1e-12)
    X2t, _, k2 = D.approx_decode_projected(Y.T, Xt.T, om_c, om_r, Lc, Lr, 0, tol=1e-12)
    assert k2 == k3
    np.testing.assert_allclose(X3, X2t.T, rtol=0, atol=1e-9 * np.abs(X3).max())


# ------------------------------------------------------ clustering decoder
def _blobs(seed, sizes, dim, sep=20.0):
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((len(sizes), dim)) * sep
    pts, lab = [], []
    for c, s in enumerate(sizes):
        pts.append(centres[c] + rng.standard_normal((s, dim)))
        lab += [c] * s
    perm = rng.permutation(sum(sizes))
    return np.concatenate(pts)[perm], np.array(lab)[perm]


def _same_partition(a, b):
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def test_kmeans_finds_well_separated_blobs():
    P, truth = _blobs(1, [30, 25, 40], 6)
    labels, C, steps, obj = D.kmeans_columns(P.T, 3, seed=2)
    assert _same_partition(labels, truth)


def test_kmeans_ends_at_lloyds_fixed_point_with_non_increasing_objective():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((60, 4))  # no cluster structure: a real local search
    labels, C, steps, obj = D.kmeans_columns(P.T, 5, seed=4)
    assert all(b <= a + 1e-12 for a, b in zip(obj, obj[1:]))
    for i in range(len(P)):
        d = ((C - P[i]) ** 2).sum(axis=1)
        assert d[labels[i]] <= d.min() + 1e-12
    for c in range(5):
        if (labels == c).any():
            np.testing.assert_allclose(C[c], P[labels == c].mean(axis=0), atol=1e-12)


def test_cluster_decoder_labels_whole_components():
    """L_c with three components, each with sampled nodes of one cluster:
    the harmonic extension is constant on a component, so every node takes
    its component's label."""
    rng = np.random.default_rng(5)
    sizes = [12, 9, 15]
    n = sum(sizes)
    W = np.zeros((n, n))
    start = 0
    comp = np.zeros(n, int)
    for c, s in enumerate(sizes):
        idx = np.arange(start, start + s)
        comp[idx] = c
        for a in range(s):                       # a path plus chords inside the component
            if a + 1 < s:
                W[idx[a], idx[a + 1]] = W[idx[a + 1], idx[a]] = rng.uniform(0.5, 1)
        for _ in range(s):
            a, b = rng.choice(idx, 2, replace=False)
            W[a, b] = W[b, a] = rng.uniform(0.5, 1)
        start += s
    Lc = O.laplacian_from_weights(sp.csr_matrix(W))
    om_c = np.sort(np.concatenate([np.arange(0, 12, 3), np.arange(12, 21, 3), np.arange(21, 36, 3)]))
    # sampled columns of X~: three far-apart blobs, one per component
    centres = np.array([[10.0, 0, 0], [0, 10.0, 0], [0, 0, 10.0]])
    Xt = (centres[comp[om_c]] + 0.1 * rng.standard_normal((len(om_c), 3))).T
    labels, C, lab_t = D.cluster_decode(Xt, om_c, n, Lc, 3, seed=1, tol=1e-12)
    np.testing.assert_array_equal(labels[om_c], lab_t)
    for c in range(3):
        assert len(set(labels[comp == c].tolist())) == 1
    assert _same_partition(labels, comp)
