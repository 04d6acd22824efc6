"""Batched FRPCAG (many uneven instances and gamma values in one launch):
equal to per-instance solves and to the FP64 oracle, per-instance stopping,
the launch-width autotuner, and replay from a captured CUDA graph."""
import numpy as np
import pytest

import gen
import oracle as O
from oracle.cpca_fista_c import frpcag_fista_c
from tests._oracle_knn import oracle_knn_graph
from tests._util import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FISTA_TOL = 1e-4


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _small_batch(M, shapes, seed=0):
    """Instances built on the host: Y~ from the seeded generator, graphs and
    lambda from the oracle (so the oracle can check every instance)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (rr, rc) in enumerate(shapes):
        Y, _, _ = gen.make_instance(seed + i, rr, rc, 3, 3, 0.05)
        Yt = Y.astype(np.float64)
        Lr, *_ = O.knn_graph(Yt, min(6, rr - 1))
        Lc, *_ = O.knn_graph(Yt.T, min(6, rc - 1))
        gr, gc = float(10 ** rng.uniform(-1, 1)), float(10 ** rng.uniform(-1, 1))
        lam = O.fista_step(gr, gc, O.power_norm(Lr), O.power_norm(Lc))
        out.append(dict(Yt_np=Yt, Lr_np=Lr, Lc_np=Lc, gamma_r=gr, gamma_c=gc, step=lam,
                        Yt=_dev(Yt), Lr=M.Csr.from_scipy(Lr), Lc=M.Csr.from_scipy(Lc)))
    return out


SHAPES = [(40, 33), (97, 250), (64, 64), (150, 71), (33, 200), (256, 128)]


def test_batched_matches_individual_and_oracle(M):
    probs = _small_batch(M, SHAPES)
    J = 120
    B = M.Batch(probs)
    Xs, infos = B.solve(M.frpcag_params(max_iter=J), want_info=True)
    for q, X, info in zip(probs, Xs, infos):
        Xi, ii = M.cpca_frpcag_solve(q["Yt"], q["Lr"], q["Lc"], gamma_r=q["gamma_r"],
                                     gamma_c=q["gamma_c"], step=q["step"], max_iter=J)
        assert torch.equal(X, Xi)  # same arithmetic, same order per entry
        assert info.iters == ii.iters == J
        assert info.objective == pytest.approx(ii.objective, rel=1e-12)
        Xo, _ = O.frpcag_fista(q["Yt_np"], q["Lr_np"], q["Lc_np"], q["gamma_r"], q["gamma_c"],
                               q["step"], J)
        assert rel_fro(X.cpu().numpy(), Xo) < FISTA_TOL


def test_batched_power_iteration_per_instance(M):
    probs = _small_batch(M, SHAPES[:3], seed=5)
    for q in probs:
        q.pop("step")
    B = M.Batch(probs)
    _, infos = B.solve(M.frpcag_params(max_iter=5, power_iters=200), want_info=True)
    for q, info in zip(probs, infos):
        assert info.norm_r == pytest.approx(O.power_norm(q["Lr_np"], 200, 0, 2), rel=1e-6)
        assert info.norm_c == pytest.approx(O.power_norm(q["Lc_np"], 200, 0, 3), rel=1e-6)
        lam = O.fista_step(q["gamma_r"], q["gamma_c"], info.norm_r, info.norm_c)
        assert info.step == pytest.approx(lam, rel=1e-12)


def test_batched_stopping_per_instance(M):
    probs = _small_batch(M, SHAPES[:4], seed=9)
    B = M.Batch(probs)
    Xs, infos = B.solve(M.frpcag_params(max_iter=3000, eps=1e-8), want_info=True)
    for q, X, info in zip(probs, Xs, infos):
        Xo, oi = O.frpcag_fista(q["Yt_np"], q["Lr_np"], q["Lc_np"], q["gamma_r"], q["gamma_c"],
                                q["step"], 3000, eps=1e-8)
        assert abs(info.iters - oi["iters"]) <= 2
        assert rel_fro(X.cpu().numpy(), Xo) < 1e-3
    assert len({i.iters for i in infos}) > 1  # instances really stop on their own


def test_autotuner_and_graph_replay(M):
    probs = _small_batch(M, SHAPES, seed=3)
    B = M.Batch(probs)
    blocks, ms = B.tune()
    assert blocks > 0 and ms > 0
    prm = M.frpcag_params(max_iter=60, blocks=blocks)
    X0 = [x.clone() for x in B.solve(prm)[0]]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.solve(prm)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    for x in B.X:
        x.zero_()
    with torch.cuda.graph(g):
        B.solve(prm)
    for x in B.X:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(B.X, X0):
        assert torch.equal(a, b)


def test_batched_workload_64_instances(M):
    """The 64-instance workload (sizes p ~ U[500, 8000], n ~ U[200, 5000],
    1/4 sampling, K = 10 graphs, gamma pairs over an 8 x 8 log grid, J = 300)
    in one batched launch: a seeded subset of six instances is built by the
    oracle (its own sampling of the generator's Y and its own graphs) and
    checked against the oracle's C restatement of Algorithm 1; every 7th
    instance equals its separate solve exactly."""
    specs = gen.batched_instances(64)
    J = specs[0]["J"]
    subset = set(np.random.default_rng(17).choice(len(specs), size=6, replace=False).tolist())
    probs, refs = [], {}
    for i, sp_ in enumerate(specs):
        Y = gen.make_instance_torch(sp_["seed"], sp_["p"], sp_["n"], sp_["r"], sp_["C"], sp_["frac"])
        rr, rc = M.rho_of(sp_["p"], sp_["fr"]), M.rho_of(sp_["n"], sp_["fc"])
        if i in subset:
            om_r = O.sample_indices(sp_["seed"], sp_["p"], rr, 0)
            om_c = O.sample_indices(sp_["seed"], sp_["n"], rc, 1)
            Yt32 = Y.cpu().numpy()[np.ix_(om_r, om_c)]
            Lr_o, *_ = oracle_knn_graph(Yt32, sp_["K"])
            Lc_o, *_ = oracle_knn_graph(Yt32.T, sp_["K"])
            refs[i] = (Yt32.astype(np.float64), Lr_o, Lc_o)
            probs.append(dict(Yt=_dev(Yt32), Lr=M.Csr.from_scipy(Lr_o), Lc=M.Csr.from_scipy(Lc_o),
                              gamma_r=sp_["gamma_r"], gamma_c=sp_["gamma_c"]))
        else:
            _, _, Yt = M.cpca_sample(sp_["seed"], sp_["p"], sp_["n"], rr, rc, Y)
            Lr, _, _ = M.cpca_knn_graph(Yt, sp_["K"])
            Lc, _, _ = M.cpca_knn_graph(Yt, sp_["K"], transposed=True)
            probs.append(dict(Yt=Yt, Lr=Lr, Lc=Lc, gamma_r=sp_["gamma_r"], gamma_c=sp_["gamma_c"]))
        del Y
    B = M.Batch(probs)
    Xs, infos = B.solve(M.frpcag_params(max_iter=J), want_info=True)
    for i, (Yt_o, Lr_o, Lc_o) in sorted(refs.items()):
        q, info = probs[i], infos[i]
        nr, nc = O.power_norm(Lr_o, 200, 0, 2), O.power_norm(Lc_o, 200, 0, 3)
        assert info.norm_r == pytest.approx(nr, rel=1e-6)
        assert info.norm_c == pytest.approx(nc, rel=1e-6)
        lam = O.fista_step(q["gamma_r"], q["gamma_c"], nr, nc)
        Xo, _ = frpcag_fista_c(Yt_o, Lr_o, Lc_o, q["gamma_r"], q["gamma_c"], lam, J)
        assert info.iters == J
        assert rel_fro(Xs[i].cpu().numpy(), Xo) < FISTA_TOL
    for q, X, info in list(zip(probs, Xs, infos))[::7]:
        # the batch's power iterations run grid-wide, a single solve's in one
        # thread-block cluster: the same per-row and per-warp arithmetic, so
        # the same lambda bit for bit, then the same FISTA entry by entry
        Xi, ii = M.cpca_frpcag_solve(q["Yt"], q["Lr"], q["Lc"], gamma_r=q["gamma_r"],
                                     gamma_c=q["gamma_c"], max_iter=J)
        assert info.norm_r > 0 and info.norm_c > 0
        assert (info.norm_r, info.norm_c, info.step) == (ii.norm_r, ii.norm_c, ii.step)
        assert torch.equal(X, Xi)
