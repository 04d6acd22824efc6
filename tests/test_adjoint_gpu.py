"""Reverse-mode derivatives on the GPU against the FP64 adjoint oracle
(which is itself pinned by finite differences in test_oracle_adjoint.py)."""
import numpy as np
import pytest

import gen
import oracle as O
from oracle import cpca_adjoint as A
from tests._util import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


@pytest.fixture(scope="module")
def inst(M):
    """Ragged 130 x 100 sampled matrix (5 x 4 tiles) with K = 6 graphs."""
    Y, _, _ = gen.make_instance(21, 130, 100, 4, 4, 0.05)
    Yt = Y.astype(np.float64)
    Lr, Wr, *_ = O.knn_graph(Yt, 6)
    Lc, Wc, *_ = O.knn_graph(Yt.T, 6)
    return dict(Yt=Yt, Lr=Lr, Lc=Lc, Wr=Wr, Wc=Wc,
                gLr=M.Csr.from_scipy(Lr, weight=Wr), gLc=M.Csr.from_scipy(Lc, weight=Wc))


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_fista_backward_given_step(M, inst):
    J, gr, gc = 60, 0.8, 1.3
    lam = O.fista_step(gr, gc, O.power_norm(inst["Lr"]), O.power_norm(inst["Lc"]))
    B = np.random.default_rng(1).standard_normal(inst["Yt"].shape)
    ref = A.frpcag_fista_vjp(inst["Yt"], inst["Lr"], inst["Lc"], gr, gc, lam, J, B)
    out = M.cpca_frpcag_backward(_dev(inst["Yt"]), inst["gLr"], inst["gLc"], _dev(B),
                                 gamma_r=gr, gamma_c=gc, step=lam, max_iter=J, ckpt_every=7)
    assert rel_fro(out["dYt"].cpu().numpy(), ref["Yt"]) < GRAD_TOL
    info = out["info"]
    assert _rel(info.dgamma_r, ref["gamma_r"]) < GRAD_TOL
    assert _rel(info.dgamma_c, ref["gamma_c"]) < GRAD_TOL
    # dloss/dlambda is a sum whose terms cancel about 10^4-fold (the output
    # barely depends on the step once FISTA converges): rounding the oracle's
    # own FP64 trajectory to FP32 moves it by about 0.5%. It reaches the named
    # gradients only through lambda's small share of them (dgamma above, dL).
    assert _rel(info.dlambda, ref["lam"]) < 2e-2
    for key, L in (("dLr", "gLr"), ("dLc", "gLc")):
        got = inst[L].pattern_scipy(out[key]).toarray()
        want = ref[key[1:]].toarray()
        assert rel_fro(got, want) < GRAD_TOL


def test_fista_backward_through_power_iterations_and_weights(M, inst):
    J, gr, gc, T = 50, 1.1, 0.6, 200
    Lr, Lc = inst["Lr"], inst["Lc"]
    nr, nc = O.power_norm(Lr, T, 0, 2), O.power_norm(Lc, T, 0, 3)
    lam = O.fista_step(gr, gc, nr, nc)
    B = np.random.default_rng(2).standard_normal(inst["Yt"].shape)
    fb = A.frpcag_fista_vjp(inst["Yt"], Lr, Lc, gr, gc, lam, J, B)
    dgr, dgc, dnr, dnc = A.fista_step_vjp(gr, gc, nr, nc, fb["lam"])
    Lr_b = fb["Lr"] + A.power_norm_vjp(Lr, dnr, T, 0, 2)
    Lc_b = fb["Lc"] + A.power_norm_vjp(Lc, dnc, T, 0, 3)
    out = M.cpca_frpcag_backward(_dev(inst["Yt"]), inst["gLr"], inst["gLc"], _dev(B),
                                 gamma_r=gr, gamma_c=gc, max_iter=J, power_iters=T,
                                 want_dw=True)
    info = out["info"]
    assert _rel(info.norm_r, nr) < 1e-6 and _rel(info.norm_c, nc) < 1e-6
    assert _rel(info.dgamma_r, fb["gamma_r"] + dgr) < GRAD_TOL
    assert _rel(info.dgamma_c, fb["gamma_c"] + dgc) < GRAD_TOL
    assert rel_fro(out["dYt"].cpu().numpy(), fb["Yt"]) < GRAD_TOL
    for key, L, ref in (("dLr", "gLr", Lr_b), ("dLc", "gLc", Lc_b)):
        assert rel_fro(inst[L].pattern_scipy(out[key]).toarray(), ref.toarray()) < GRAD_TOL
    for key, L, W, ref in (("dwr", "gLr", "Wr", Lr_b), ("dwc", "gLc", "Wc", Lc_b)):
        want = A.laplacian_weight_vjp(inst[W], ref).toarray()
        assert rel_fro(inst[L].pattern_scipy(out[key]).toarray(), want) < GRAD_TOL


def test_fista_backward_checkpoint_spacing_is_exact(M, inst):
    """Recomputing segments reproduces the trajectory exactly: dY~ does not
    depend on the checkpoint spacing (a given step: the power iterations'
    FP64 atomic sums are not bitwise repeatable). dL and the scalars agree to
    rounding (per-segment FP32 partial sums, FP64 atomics)."""
    J = 23
    B = _dev(np.random.default_rng(3).standard_normal(inst["Yt"].shape))
    Yt = _dev(inst["Yt"])
    outs = [M.cpca_frpcag_backward(Yt, inst["gLr"], inst["gLc"], B, gamma_r=1.0, gamma_c=1.0,
                                   step=0.15, max_iter=J, ckpt_every=c) for c in (1, 5, 20, J)]
    for o in outs[1:]:
        assert torch.equal(o["dYt"], outs[0]["dYt"])
        for key in ("dLr", "dLc"):
            assert rel_fro(o[key].cpu().numpy(), outs[0][key].cpu().numpy()) < 1e-6
        assert _rel(o["info"].dgamma_r, outs[0]["info"].dgamma_r) < 1e-9


def test_fista_backward_gamma_zero_is_identity(M, inst):
    B = _dev(np.random.default_rng(4).standard_normal(inst["Yt"].shape))
    out = M.cpca_frpcag_backward(_dev(inst["Yt"]), inst["gLr"], inst["gLc"], B, gamma_r=0.0,
                                 gamma_c=0.0, max_iter=15)
    assert torch.equal(out["dYt"], B)
    assert out["info"].dgamma_r == 0.0 or abs(out["info"].dgamma_r) < 1e-30


@pytest.mark.parametrize("p,n,rr,rc", [(260, 200, 130, 100), (200, 260, 100, 130)])
def test_decode_backward_matches_oracle(M, p, n, rr, rc):
    """Both orientations of the SVD adjoint (rr >= rc uses X~, else X~^T)."""
    Y, _, _ = gen.make_instance(31, p, n, 4, 4, 0.05)
    Y = Y.astype(np.float64)
    om_r, om_c = O.sample_indices(5, p, rr, 0), O.sample_indices(5, n, rc, 1)
    Yt = Y[np.ix_(om_r, om_c)]
    Lr, Wr, *_ = O.knn_graph(Y, 6)
    Lc, Wc, *_ = O.knn_graph(Y.T, 6)
    Lrt, *_ = O.knn_graph(Yt, 6)
    Lct, *_ = O.knn_graph(Yt.T, 6)
    Xt = O.frpcag_fista(Yt, Lrt, Lct, 1.0, 1.0, 0.15, 150)[0].astype(np.float32).astype(np.float64)
    k = O.svd_rank(Xt)[3]
    rng = np.random.default_rng(7)
    inside = np.zeros((p, n), dtype=bool)
    inside[np.ix_(om_r, om_c)] = True
    cand = np.argwhere(~inside)
    pick = cand[rng.choice(len(cand), 400, replace=False)]
    g = rng.standard_normal(400).astype(np.float32)
    ref = A.approx_decode_vjp(Xt, om_r, om_c, p, n, Lr, Lc, k, pick[:, 0], pick[:, 1],
                              g.astype(np.float64))
    gLr, gLc = M.Csr.from_scipy(Lr, weight=Wr), M.Csr.from_scipy(Lc, weight=Wc)
    ti = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device="cuda")
    out = M.cpca_decode_backward(_dev(Xt), ti(om_r), ti(om_c), p, n, gLr, gLc, k,
                                 ti(pick[:, 0]), ti(pick[:, 1]), _dev(g), want_dw=True)
    assert rel_fro(out["dXt"].cpu().numpy(), ref["Xt"]) < GRAD_TOL
    assert rel_fro(gLr.pattern_scipy(out["dLr"]).toarray(), ref["Lr"].toarray()) < GRAD_TOL
    assert rel_fro(gLc.pattern_scipy(out["dLc"]).toarray(), ref["Lc"].toarray()) < GRAD_TOL
    for key, G, W, Lb in (("dwr", gLr, Wr, ref["Lr"]), ("dwc", gLc, Wc, ref["Lc"])):
        want = A.laplacian_weight_vjp(W, Lb).toarray()
        assert rel_fro(G.pattern_scipy(out[key]).toarray(), want) < GRAD_TOL


def test_autograd_pipeline_gradient_matches_oracle(M):
    """Held-out loss 1/2 sum (X_e - Y_e)^2 of FISTA (lambda by power
    iteration) + decoder, differentiated by torch.autograd through the
    library's adjoints, against the FP64 oracle gradient: gamma_r, gamma_c,
    Y~ and the edge weights of all four graphs."""
    from paper_1602_02070_gb300 import autograd as AG
    p, n, rr, rc, J, T = 180, 150, 90, 75, 40, 60
    Y, _, _ = gen.make_instance(41, p, n, 3, 3, 0.05)
    Y = Y.astype(np.float64)
    om_r, om_c = O.sample_indices(9, p, rr, 0), O.sample_indices(9, n, rc, 1)
    Yt = Y[np.ix_(om_r, om_c)]
    _, Wr, *_ = O.knn_graph(Y, 5)
    _, Wc, *_ = O.knn_graph(Y.T, 5)
    _, Wrt, *_ = O.knn_graph(Yt, 5)
    _, Wct, *_ = O.knn_graph(Yt.T, 5)
    rng = np.random.default_rng(12)
    inside = np.zeros((p, n), dtype=bool)
    inside[np.ix_(om_r, om_c)] = True
    cand = np.argwhere(~inside)
    pick = cand[rng.choice(len(cand), 300, replace=False)]
    gr, gc = 0.9, 1.2
    # k from the oracle's own forward
    Lrt_o, Lct_o = O.laplacian_from_weights(Wrt), O.laplacian_from_weights(Wct)
    lam = O.fista_step(gr, gc, O.power_norm(Lrt_o, T, 0, 2), O.power_norm(Lct_o, T, 0, 3))
    k = O.svd_rank(O.frpcag_fista(Yt, Lrt_o, Lct_o, gr, gc, lam, J)[0])[3]
    G = A.cpca_loss_grad(Y, Wr, Wc, Wrt, Wct, om_r, om_c, gr, gc, J, k, pick[:, 0], pick[:, 1],
                         power_iters=T)

    pats = {key: M.Csr.from_scipy(O.laplacian_from_weights(W), weight=W)
            for key, W in (("Wr", Wr), ("Wc", Wc), ("Wrt", Wrt), ("Wct", Wct))}
    w = {key: P.weight.clone().requires_grad_(True) for key, P in pats.items()}
    Yt_t = _dev(Yt).requires_grad_(True)
    g_r = torch.tensor(gr, dtype=torch.float64, device="cuda", requires_grad=True)
    g_c = torch.tensor(gc, dtype=torch.float64, device="cuda", requires_grad=True)
    L = {key: AG.laplacian(pats[key].rowptr, pats[key].col, w[key]) for key in pats}
    Xt = AG.frpcag(Yt_t, g_r, g_c, L["Wrt"], L["Wct"], pats["Wrt"], pats["Wct"], max_iter=J,
                   power_iters=T, ckpt_every=7)
    ti = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device="cuda")
    vals = AG.decode_entries(Xt, L["Wr"], L["Wc"], pats["Wr"], pats["Wc"], ti(om_r), ti(om_c), p, n,
                             ti(pick[:, 0]), ti(pick[:, 1]), M.decode_params(k_override=k))
    target = torch.as_tensor(Y[pick[:, 0], pick[:, 1]], dtype=torch.float32, device="cuda")
    loss = 0.5 * ((vals.double() - target.double()) ** 2).sum()
    loss.backward()
    assert _rel(loss.item(), G["loss"]) < GRAD_TOL
    assert _rel(g_r.grad.item(), G["gamma_r"]) < GRAD_TOL
    assert _rel(g_c.grad.item(), G["gamma_c"]) < GRAD_TOL
    assert rel_fro(Yt_t.grad.cpu().numpy(), G["Yt"]) < GRAD_TOL
    for key in ("Wr", "Wc", "Wrt", "Wct"):
        got = pats[key].pattern_scipy(w[key].grad).toarray()
        assert rel_fro(got, G[key].toarray()) < GRAD_TOL, key


def test_forward_tape_and_resume(M, inst):
    """The taped forward equals the plain solve; the resumed backward equals
    the self-contained one."""
    Yt = _dev(inst["Yt"])
    prm = M.frpcag_params(gamma_r=0.7, gamma_c=1.4, max_iter=45)
    X0, _ = M.cpca_frpcag_solve(Yt, inst["gLr"], inst["gLc"], prm)
    X1, ws, ginfo = M.capi.cpca_frpcag_forward_tape(Yt, inst["gLr"], inst["gLc"], prm, 10)
    assert rel_fro(X1.cpu().numpy(), X0.cpu().numpy()) < 1e-6
    B = _dev(np.random.default_rng(5).standard_normal(inst["Yt"].shape))
    r0 = M.cpca_frpcag_backward(Yt, inst["gLr"], inst["gLc"], B, prm, ckpt_every=10)
    r1 = M.cpca_frpcag_backward(Yt, inst["gLr"], inst["gLc"], B, prm, ckpt_every=10, ws=ws, resume=True)
    assert rel_fro(r1["dYt"].cpu().numpy(), r0["dYt"].cpu().numpy()) < 1e-5
    assert _rel(r1["info"].dgamma_r, r0["info"].dgamma_r) < 1e-5
    assert _rel(ginfo.lambda_, r0["info"].lambda_) < 1e-7


def test_decode_backward_resume_matches(M):
    p, n, rr, rc = 240, 180, 120, 90
    Y, _, _ = gen.make_instance(33, p, n, 4, 4, 0.05)
    Yd = torch.as_tensor(Y, device="cuda")
    Lr, _, _ = M.cpca_knn_graph(Yd, 6)
    Lc, _, _ = M.cpca_knn_graph(Yd, 6, transposed=True)
    om_r, om_c, Yt = M.cpca_sample(2, p, n, rr, rc, Yd)
    Xt = Yt.contiguous()
    prm = M.decode_params()
    ws = M.capi.decode_backward_workspace(Xt, p, n, Lr, Lc, prm)
    dec = M.cpca_decode(Xt, om_r, om_c, p, n, Lr, Lc, prm, want_X=False, ws=ws)
    rng = np.random.default_rng(3)
    hr = torch.as_tensor(rng.integers(0, p, 500).astype(np.int32), device="cuda")
    hc = torch.as_tensor(rng.integers(0, n, 500).astype(np.int32), device="cuda")
    g = torch.as_tensor(rng.standard_normal(500).astype(np.float32), device="cuda")
    r1 = M.cpca_decode_backward(Xt, om_r, om_c, p, n, Lr, Lc, dec["k"], hr, hc, g, prm, ws=ws, resume=True)
    r0 = M.cpca_decode_backward(Xt, om_r, om_c, p, n, Lr, Lc, dec["k"], hr, hc, g, prm)
    assert rel_fro(r1["dXt"].cpu().numpy(), r0["dXt"].cpu().numpy()) < 1e-6
    assert rel_fro(r1["dLr"].cpu().numpy(), r0["dLr"].cpu().numpy()) < 1e-6
    with pytest.raises(M.CpcaError):
        M.cpca_decode_backward(Xt, om_r, om_c, p, n, Lr, Lc, dec["k"] + 1, hr, hc, g, prm, ws=ws,
                               resume=True)
