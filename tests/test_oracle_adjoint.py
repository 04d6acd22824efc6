"""Pins for the FP64 adjoint oracle: every reverse-mode piece against
central finite differences of the forward oracle (FP64, small h, where the
map is smooth), and the whole held-out loss gradient against finite
differences in gamma_r, gamma_c, Y~ and the edge weights of all four graphs.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle as O
from oracle import cpca_adjoint as A


def _sym_direction(W, rng):
    """A random symmetric perturbation on W's off-diagonal pattern."""
    C = sp.triu(sp.csr_matrix(W), k=1).tocoo()
    d = rng.standard_normal(C.nnz)
    E = sp.csr_matrix((d, (C.row, C.col)), shape=W.shape)
    return E + E.T


def _edge_dot(Wbar, E):
    """sum over undirected edges of dloss/dw_e * E_e (both entries hold each)."""
    return 0.5 * float(sp.csr_matrix(Wbar).multiply(E).sum())


def _pattern_dot(Lbar, E):
    return float(sp.csr_matrix(Lbar).multiply(E).sum())


@pytest.fixture(scope="module")
def small():
    Y, _, _ = gen.make_instance(7, 48, 40, 3, 3, 0.05)
    Y = Y.astype(np.float64)
    p, n = Y.shape
    om_r, om_c = O.sample_indices(3, p, 24, 0), O.sample_indices(3, n, 20, 1)
    Yt = Y[np.ix_(om_r, om_c)]
    _, Wr, *_ = O.knn_graph(Y, 4)
    _, Wc, *_ = O.knn_graph(Y.T, 4)
    _, Wrt, *_ = O.knn_graph(Yt, 4)
    _, Wct, *_ = O.knn_graph(Yt.T, 4)
    rng = np.random.default_rng(11)
    inside = np.zeros((p, n), dtype=bool)
    inside[np.ix_(om_r, om_c)] = True
    cand = np.argwhere(~inside)
    pick = cand[rng.choice(len(cand), 60, replace=False)]
    return dict(Y=Y, om_r=om_r, om_c=om_c, Yt=Yt, Wr=Wr, Wc=Wc, Wrt=Wrt, Wct=Wct,
                rows=pick[:, 0], cols=pick[:, 1])


@pytest.mark.parametrize("lap", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
def test_laplacian_weight_vjp(small, lap):
    rng = np.random.default_rng(1)
    W = small["Wr"]
    L = O.laplacian_from_weights(W, lap)
    Lbar = A.pattern_outer(L, rng.standard_normal((L.shape[0], 1)),
                           rng.standard_normal((L.shape[0], 1)))
    g = A.laplacian_weight_vjp(W, Lbar, lap)
    for _ in range(3):
        E = _sym_direction(W, rng)
        h = 1e-6
        fd = (_pattern_dot(Lbar, O.laplacian_from_weights(W + h * E, lap))
              - _pattern_dot(Lbar, O.laplacian_from_weights(W - h * E, lap))) / (2 * h)
        assert _edge_dot(g, E) == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_power_norm_vjp(small):
    rng = np.random.default_rng(2)
    L = O.laplacian_from_weights(small["Wrt"])
    g = A.power_norm_vjp(L, 1.0, 60, 0, 2)
    for _ in range(3):
        E = _sym_direction(L, rng) + sp.diags(rng.standard_normal(L.shape[0]))
        h = 1e-6
        fd = (O.power_norm(L + h * E, 60, 0, 2) - O.power_norm(L - h * E, 60, 0, 2)) / (2 * h)
        assert _pattern_dot(g, E) == pytest.approx(fd, rel=1e-6)


def test_fista_step_vjp():
    gr, gc, nr, nc = 0.7, 1.9, 1.3, 1.6
    out = A.fista_step_vjp(gr, gc, nr, nc, 1.0)
    h = 1e-7
    args = [gr, gc, nr, nc]
    for i in range(4):
        up, dn = list(args), list(args)
        up[i] += h
        dn[i] -= h
        fd = (O.fista_step(*up) - O.fista_step(*dn)) / (2 * h)
        assert out[i] == pytest.approx(fd, rel=1e-7)


def test_frpcag_fista_vjp(small):
    rng = np.random.default_rng(3)
    Yt = small["Yt"]
    Lr = O.laplacian_from_weights(small["Wrt"])
    Lc = O.laplacian_from_weights(small["Wct"])
    gr, gc, J = 0.8, 1.3, 40
    lam = O.fista_step(gr, gc, O.power_norm(Lr), O.power_norm(Lc))
    B = rng.standard_normal(Yt.shape)
    out = A.frpcag_fista_vjp(Yt, Lr, Lc, gr, gc, lam, J, B)

    def f(Yt_=Yt, Lr_=Lr, Lc_=Lc, gr_=gr, gc_=gc, lam_=lam):
        S, _ = O.frpcag_fista(Yt_, Lr_, Lc_, gr_, gc_, lam_, J)
        return float(np.sum(B * S))

    h = 1e-7
    D = rng.standard_normal(Yt.shape)
    fd = (f(Yt_=Yt + h * D) - f(Yt_=Yt - h * D)) / (2 * h)
    assert np.sum(out["Yt"] * D) == pytest.approx(fd, rel=1e-6)
    for key, kw in (("gamma_r", "gr_"), ("gamma_c", "gc_"), ("lam", "lam_")):
        base = {"gr_": gr, "gc_": gc, "lam_": lam}[kw]
        fd = (f(**{kw: base + h}) - f(**{kw: base - h})) / (2 * h)
        assert out[key] == pytest.approx(fd, rel=1e-6)
    for key, L, kw in (("Lr", Lr, "Lr_"), ("Lc", Lc, "Lc_")):
        E = _sym_direction(L, rng)
        fd = (f(**{kw: L + h * E}) - f(**{kw: L - h * E})) / (2 * h)
        assert _pattern_dot(out[key], E) == pytest.approx(fd, rel=1e-6)


def test_frpcag_fista_vjp_gamma_zero_is_identity(small):
    """gamma = 0: S_J = Y~ whatever lambda, so dS/dY~ = I and nothing else."""
    Yt = small["Yt"]
    Lr = O.laplacian_from_weights(small["Wrt"])
    Lc = O.laplacian_from_weights(small["Wct"])
    B = np.random.default_rng(4).standard_normal(Yt.shape)
    out = A.frpcag_fista_vjp(Yt, Lr, Lc, 0.0, 0.0, 1.0, 25, B)
    assert np.array_equal(out["Yt"], B)
    assert out["gamma_r"] == 0.0 and out["gamma_c"] == 0.0


def _aligned_topk(A_, k, ref_U):
    U, s, Vh = np.linalg.svd(A_, full_matrices=False)
    sg = np.sign(np.sum(U[:, :k] * ref_U, axis=0))
    return U[:, :k] * sg, s[:k], Vh[:k].T * sg


def test_svd_topk_vjp():
    rng = np.random.default_rng(5)
    for m, n in ((30, 18), (14, 25)):
        A_ = rng.standard_normal((m, 4)) @ rng.standard_normal((4, n)) * 3 \
            + 0.1 * rng.standard_normal((m, n))
        k = 4
        U0, s0, V0 = _aligned_topk(A_, k, np.linalg.svd(A_)[0][:, :k])
        Ub, sb, Vb = (rng.standard_normal(U0.shape), rng.standard_normal(k),
                      rng.standard_normal(V0.shape))
        g = A.svd_topk_vjp(A_, k, Ub, sb, Vb)

        def f(M):
            U, s, V = _aligned_topk(M, k, U0)
            return np.sum(Ub * U) + np.sum(sb * s) + np.sum(Vb * V)

        D = rng.standard_normal(A_.shape)
        h = 1e-6
        fd = (f(A_ + h * D) - f(A_ - h * D)) / (2 * h)
        assert np.sum(g * D) == pytest.approx(fd, rel=1e-6)


def test_approx_decode_vjp(small):
    rng = np.random.default_rng(6)
    Y = small["Y"]
    p, n = Y.shape
    Lr = O.laplacian_from_weights(small["Wr"])
    Lc = O.laplacian_from_weights(small["Wc"])
    Xt = O.frpcag_fista(small["Yt"], O.laplacian_from_weights(small["Wrt"]),
                        O.laplacian_from_weights(small["Wct"]), 1.0, 1.0, 0.2, 60)[0]
    k = 3
    rows, cols = small["rows"], small["cols"]
    g = rng.standard_normal(len(rows))
    out = A.approx_decode_vjp(Xt, small["om_r"], small["om_c"], p, n, Lr, Lc, k, rows, cols, g)

    def f(Xt_=Xt, Lr_=Lr, Lc_=Lc):
        d = A.approx_decode_exact(Xt_, small["om_r"], small["om_c"], p, n, Lr_, Lc_, k)
        return float(np.sum(g * np.einsum("ec,c,ec->e", d["U"][rows], d["sigma"], d["V"][cols])))

    h = 1e-6
    D = rng.standard_normal(Xt.shape)
    fd = (f(Xt_=Xt + h * D) - f(Xt_=Xt - h * D)) / (2 * h)
    assert np.sum(out["Xt"] * D) == pytest.approx(fd, rel=1e-6)
    for key, L, kw in (("Lr", Lr, "Lr_"), ("Lc", Lc, "Lc_")):
        E = _sym_direction(L, rng)
        fd = (f(**{kw: L + h * E}) - f(**{kw: L - h * E})) / (2 * h)
        assert _pattern_dot(out[key], E) == pytest.approx(fd, rel=1e-6)


def test_decode_exact_matches_pcg_decoder(small):
    """The exact-solve decoder used for derivatives is the PCG decoder at a
    tight tolerance."""
    Y = small["Y"]
    p, n = Y.shape
    Lr = O.laplacian_from_weights(small["Wr"])
    Lc = O.laplacian_from_weights(small["Wc"])
    Xt = small["Yt"]
    dp = O.approx_decode(Xt, small["om_r"], small["om_c"], p, n, Lr, Lc, tol=1e-13)
    de = A.approx_decode_exact(Xt, small["om_r"], small["om_c"], p, n, Lr, Lc, dp["k"])
    X = (de["U"] * de["sigma"]) @ de["V"].T
    assert np.allclose(X, dp["X"], rtol=0, atol=1e-10 * np.abs(dp["X"]).max())


def test_cpca_loss_grad(small):
    rng = np.random.default_rng(8)
    s = small
    args = dict(omega_r=s["om_r"], omega_c=s["om_c"], J=30, k=3, rows=s["rows"],
                cols=s["cols"], power_iters=60)
    W = dict(Wr=s["Wr"], Wc=s["Wc"], Wrt=s["Wrt"], Wct=s["Wct"])
    gr, gc = 0.9, 1.2
    G = A.cpca_loss_grad(s["Y"], gamma_r=gr, gamma_c=gc, **W, **args)
    L0, _ = A.cpca_loss(s["Y"], gamma_r=gr, gamma_c=gc, **W, **args)
    assert G["loss"] == pytest.approx(L0, rel=1e-12)

    def f(Y=s["Y"], gr_=gr, gc_=gc, **Wo):
        Ws = dict(W, **Wo)
        return A.cpca_loss(Y, gamma_r=gr_, gamma_c=gc_, **Ws, **args)[0]

    h = 1e-6
    assert G["gamma_r"] == pytest.approx((f(gr_=gr + h) - f(gr_=gr - h)) / (2 * h), rel=1e-5)
    assert G["gamma_c"] == pytest.approx((f(gc_=gc + h) - f(gc_=gc - h)) / (2 * h), rel=1e-5)
    D = np.zeros_like(s["Y"])
    D[np.ix_(s["om_r"], s["om_c"])] = rng.standard_normal(s["Yt"].shape)
    fd = (f(Y=s["Y"] + h * D) - f(Y=s["Y"] - h * D)) / (2 * h)
    assert np.sum(G["Yt"] * D[np.ix_(s["om_r"], s["om_c"])]) == pytest.approx(fd, rel=1e-5)
    for key in ("Wr", "Wc", "Wrt", "Wct"):
        E = _sym_direction(W[key], rng)
        fd = (f(**{key: W[key] + h * E}) - f(**{key: W[key] - h * E})) / (2 * h)
        assert _edge_dot(G[key], E) == pytest.approx(fd, rel=1e-5), key
