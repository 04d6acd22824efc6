"""Full-size parity, in the launch configuration the benchmark times.

10304 x 1000 (rank 10, 10 clusters, 5% gross errors, K = 10, 1/4 x 1/4
sampling, 300 FISTA iterations): every step against the FP64 oracle element
by element, each step fed the oracle's own inputs, then the whole pipeline
end to end. Every check runs unconditionally.

20000 x 100000 (8 GB on the device; rank 20, 50 clusters, 2% gross errors,
1/10 x 1/10 sampling): sampled kNN queries of the full graphs, every query
of the sampled matrix's graphs, FISTA for the full 300 iterations on the
oracle's graphs against the oracle's C restatement of Algorithm 1, and the
decoder at full size (same p, n, sampled sets and X~) on graphs the oracle
builds itself (kNN graphs of seeded 20-dimensional latent points of the
workload's model: the decoder takes any Laplacian, and these are cheap for
the oracle to search) against oracle.approx_decode at sampled entries of X;
then properties of the pipeline's own decoder that hold at any size.

kNN sets must agree exactly: the library settles every FP32 ordering its
error bound cannot decide in FP64, so a difference could only come from a
gap far below the 1e-6 relative that the contract allows.
"""
import numpy as np
import pytest

import gen
import oracle as O
from oracle.cpca_fista_c import frpcag_fista_c, knn_c
from tests._oracle_knn import oracle_knn_graph
from tests._util import knn_sets_match, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FISTA_TOL = 1e-4


def d2_rtol(dim):
    """Worst-case relative error of the FP32 exact squared distance: each of
    32 lanes sums about dim/32 squares in order, then a 5-level tree."""
    return (dim / 32 + 8) * 2.0 ** -24


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _check_lists(gi, gd, oi, od, K, dim):
    """GPU kNN lists against the oracle's K+1 nearest: the same sets (near
    ties below 1e-6 relative are the only allowed difference, and none
    occurs), the same distances to FP32 rounding."""
    gi = gi.cpu().numpy()
    gd = gd.cpu().numpy().astype(np.float64)
    assert knn_sets_match(gi, gd, oi[:, :K], od, K, rel_gap=1e-6) == []
    same = np.array([set(a.tolist()) == set(b.tolist()) for a, b in zip(gi, oi[:, :K])])
    assert same.all(), f"{int((~same).sum())} queries differ"
    assert np.allclose(np.sort(gd, axis=1), od[:, :K], rtol=d2_rtol(dim), atol=0)


def _check_graph(G, L):
    Gs = G.to_scipy()
    assert np.array_equal(Gs.indptr, L.indptr) and np.array_equal(Gs.indices, L.indices)
    assert np.allclose(Gs.data, L.data, rtol=1e-5, atol=1e-7)


def test_c1_every_step_and_end_to_end(M):
    cfg = gen.CONFIGS["bench_10304x1000"]
    p, n, K, J = cfg["p"], cfg["n"], cfg["K"], cfg["J"]
    Y, _, _ = gen.make_instance(0, p, n, cfg["r"], cfg["C"], cfg["frac"])
    Yd = Y.astype(np.float64)
    Ydev = torch.as_tensor(Y, device="cuda")
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])

    # step 1: graphs of the rows and columns of Y
    Lr_o, _, ir_o, dr_o = oracle_knn_graph(Y, K)
    Lc_o, _, ic_o, dc_o = oracle_knn_graph(Y.T, K)
    Lr, kr, dr = M.cpca_knn_graph(Ydev, K, want_knn=True)
    Lc, kc, dc = M.cpca_knn_graph(Ydev, K, transposed=True, want_knn=True)
    _check_lists(kr, dr, ir_o, dr_o, K, n)
    _check_lists(kc, dc, ic_o, dc_o, K, p)
    _check_graph(Lr, Lr_o)
    _check_graph(Lc, Lc_o)

    # steps 2-3: sampling, bit-exact
    om_r, om_c, Yt = M.cpca_sample(0, p, n, rr, rc, Ydev)
    om_r_o, om_c_o = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    assert np.array_equal(om_r.cpu().numpy(), om_r_o)
    assert np.array_equal(om_c.cpu().numpy(), om_c_o)
    Yt_o = O.sample_matrix(Yd, om_r_o, om_c_o)
    assert np.array_equal(Yt.cpu().numpy(), Yt_o.astype(np.float32))

    # step 4: graphs of the sampled matrix
    Lrt_o, _, irt, drt = oracle_knn_graph(Yt_o.astype(np.float32), K)
    Lct_o, _, ict, dct = oracle_knn_graph(Yt_o.T.astype(np.float32), K)
    Lrt, krt, drt_g = M.cpca_knn_graph(Yt, K, want_knn=True)
    Lct, kct, dct_g = M.cpca_knn_graph(Yt, K, transposed=True, want_knn=True)
    _check_lists(krt, drt_g, irt, drt, K, rc)
    _check_lists(kct, dct_g, ict, dct, K, rr)
    _check_graph(Lrt, Lrt_o)
    _check_graph(Lct, Lct_o)

    # step 5: power iterations and FISTA on the oracle's graphs
    nr, nc = O.power_norm(Lrt_o, 200, 0, 2), O.power_norm(Lct_o, 200, 0, 3)
    lam = O.fista_step(1.0, 1.0, nr, nc)
    Xt_o, _ = O.frpcag_fista(Yt_o, Lrt_o, Lct_o, 1.0, 1.0, lam, J)
    Xt, info = M.cpca_frpcag_solve(Yt, M.Csr.from_scipy(Lrt_o), M.Csr.from_scipy(Lct_o),
                                   gamma_r=1.0, gamma_c=1.0, max_iter=J)
    assert info.norm_r == pytest.approx(nr, rel=1e-6)
    assert info.norm_c == pytest.approx(nc, rel=1e-6)
    assert info.iters == J
    assert rel_fro(Xt.cpu().numpy(), Xt_o) < FISTA_TOL

    # step 6: decoder on the oracle's X~ (rounded to FP32, the kernel's input) and graphs
    Xt_in = Xt_o.astype(np.float32)
    dec_o = O.approx_decode(Xt_in.astype(np.float64), om_r_o, om_c_o, p, n, Lr_o, Lc_o,
                            tol=cfg["cg_tol"])
    dec = M.cpca_decode(torch.as_tensor(Xt_in, device="cuda"), om_r, om_c, p, n,
                        M.Csr.from_scipy(Lr_o), M.Csr.from_scipy(Lc_o), cg_tol=cfg["cg_tol"])
    assert dec["k"] == dec_o["k"]
    assert np.allclose(dec["sigma"].cpu().numpy(), dec_o["sigma"], rtol=1e-5)
    assert rel_fro(dec["X"].cpu().numpy(), dec_o["X"]) < FISTA_TOL

    # the whole pipeline, as timed (its graphs equal the oracle's, checked above)
    out = M.cpca_pipeline(Ydev, K=K, fr=cfg["fr"], fc=cfg["fc"], seed=0, J=J, cg_tol=cfg["cg_tol"])
    dec_e = O.approx_decode(Xt_o, om_r_o, om_c_o, p, n, Lr_o, Lc_o, tol=cfg["cg_tol"])
    assert out["k"] == dec_e["k"]
    assert rel_fro(out["Xt"].cpu().numpy(), Xt_o) < FISTA_TOL
    assert rel_fro(out["X"].cpu().numpy(), dec_e["X"]) < FISTA_TOL


def test_c2_full_size(M):
    cfg = gen.CONFIGS["large_20000x100000"]
    p, n, K, J = cfg["p"], cfg["n"], cfg["K"], cfg["J"]
    Y = gen.make_instance_torch(0, p, n, cfg["r"], cfg["C"], cfg["frac"], device="cuda")
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    rng = np.random.default_rng(1)

    # full graphs (tensor-core candidates + exact recheck): sampled queries
    Lr, kr, dr = M.cpca_knn_graph(Y, K, want_knn=True)
    Lc, kc, dc = M.cpca_knn_graph(Y, K, transposed=True, want_knn=True)
    Yh = Y.cpu().numpy()
    for P, kk, dd, npts, dim in ((Yh, kr, dr, p, n), (None, kc, dc, n, p)):
        P = np.ascontiguousarray(Yh.T) if P is None else P
        qs = np.sort(rng.choice(npts, size=48, replace=False))
        oi, od = knn_c(P, K + 1, queries=qs)
        qt = torch.as_tensor(qs, device="cuda")
        _check_lists(kk[qt], dd[qt], oi, od, K, dim)
        del P

    # Laplacians: symmetric, L_n D^{1/2} 1 = 0, on sampled rows
    for G in (Lr, Lc):
        rp, cols = G.rowptr.cpu().numpy(), G.col.cpu().numpy()
        vals, w = G.val.cpu().numpy(), G.weight.cpu().numpy().astype(np.float64)
        deg = np.add.reduceat(w, rp[:-1])
        for i in rng.choice(G.n, size=64, replace=False):
            seg = slice(rp[i], rp[i + 1])
            assert np.all(np.diff(cols[seg]) > 0)
            for j, v in zip(cols[seg], vals[seg]):
                jc = cols[rp[j]:rp[j + 1]]
                t = np.searchsorted(jc, i)
                assert jc[t] == i and vals[rp[j] + t] == v
            assert abs(np.dot(vals[seg], np.sqrt(deg[cols[seg]]))) < 1e-5 * np.sqrt(deg[i])

    # sampling (bit-exact), graphs of the sampled matrix (all queries)
    om_r, om_c, Yt = M.cpca_sample(0, p, n, rr, rc, Y)
    om_r_o, om_c_o = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    assert np.array_equal(om_r.cpu().numpy(), om_r_o)
    assert np.array_equal(om_c.cpu().numpy(), om_c_o)
    Yt32 = Yh[np.ix_(om_r_o, om_c_o)]
    del Yh
    assert np.array_equal(Yt.cpu().numpy(), Yt32)
    Lrt_o, _, irt, drt = oracle_knn_graph(Yt32, K)
    Lct_o, _, ict, dct = oracle_knn_graph(Yt32.T, K)
    Lrt, krt, drt_g = M.cpca_knn_graph(Yt, K, want_knn=True)
    Lct, kct, dct_g = M.cpca_knn_graph(Yt, K, transposed=True, want_knn=True)
    _check_lists(krt, drt_g, irt, drt, K, rc)
    _check_lists(kct, dct_g, ict, dct, K, rr)
    _check_graph(Lrt, Lrt_o)
    _check_graph(Lct, Lct_o)

    # FISTA on the oracle's graphs, all J iterations, in the benchmark's launch
    Yt_o = Yt32.astype(np.float64)
    nr, nc = O.power_norm(Lrt_o, 200, 0, 2), O.power_norm(Lct_o, 200, 0, 3)
    lam = O.fista_step(1.0, 1.0, nr, nc)
    Xt_o, oinfo = frpcag_fista_c(Yt_o, Lrt_o, Lct_o, 1.0, 1.0, lam, J)
    assert oinfo["iters"] == J
    Xt, info = M.cpca_frpcag_solve(Yt, M.Csr.from_scipy(Lrt_o), M.Csr.from_scipy(Lct_o),
                                   gamma_r=1.0, gamma_c=1.0, max_iter=J)
    assert info.norm_r == pytest.approx(nr, rel=1e-6)
    assert info.norm_c == pytest.approx(nc, rel=1e-6)
    assert info.iters == J
    assert rel_fro(Xt.cpu().numpy(), Xt_o) < FISTA_TOL
    del Y

    # decoder at full size against the oracle: the oracle's X~ (rounded to
    # FP32, the kernel's input), the sampled sets, and graphs of seeded
    # latent points built by the oracle (rows: one cloud; columns: the
    # workload's 50 clusters)
    Lr_l, *_ = oracle_knn_graph(gen.latent_points(11, p, 20, 1), K)
    Lc_l, *_ = oracle_knn_graph(gen.latent_points(12, n, 20, cfg["C"]), K)
    Xt_in = Xt_o.astype(np.float32)
    dec_o = O.approx_decode(Xt_in.astype(np.float64), om_r_o, om_c_o, p, n, Lr_l, Lc_l,
                            tol=cfg["cg_tol"], want_X=False)
    dec_l = M.cpca_decode(torch.as_tensor(Xt_in, device="cuda"), om_r, om_c, p, n,
                          M.Csr.from_scipy(Lr_l), M.Csr.from_scipy(Lc_l), cg_tol=cfg["cg_tol"])
    k = dec_o["k"]
    assert dec_l["k"] == k
    assert np.allclose(dec_l["sigma"].cpu().numpy(), dec_o["sigma"], rtol=1e-5)
    ii, jj = rng.integers(0, p, 1 << 16), rng.integers(0, n, 1 << 16)
    x_o = np.einsum("ek,k,ek->e", dec_o["U"][ii], dec_o["sigma"], dec_o["V"][jj])
    x_g = dec_l["X"][torch.as_tensor(ii, device="cuda"), torch.as_tensor(jj, device="cuda")]
    assert rel_fro(x_g.double().cpu().numpy(), x_o) < FISTA_TOL
    del dec_l
    torch.cuda.empty_cache()

    # the pipeline's own decoder (its FISTA output, its full graphs):
    # properties that hold at any size
    Xt_full, _ = M.cpca_frpcag_solve(Yt, Lrt, Lct, gamma_r=1.0, gamma_c=1.0, max_iter=J)
    dec = M.cpca_decode(Xt_full, om_r, om_c, p, n, Lr, Lc, cg_tol=cfg["cg_tol"])
    k, info = dec["k"], dec["info"]
    s_np = np.linalg.svd(Xt_full.double().cpu().numpy(), compute_uv=False)
    assert k == int(np.sum(s_np / s_np[0] >= 0.1))
    assert np.allclose(np.array(info.s_tilde[:k]), s_np[:k], rtol=1e-5)
    sig = dec["sigma"].cpu().numpy()
    assert np.allclose(sig, np.sqrt(p * n / (rr * rc)) * np.array(info.s_tilde[:k]), rtol=1e-12)
    assert info.cg_res_u <= cfg["cg_tol"] and info.cg_res_v <= cfg["cg_tol"]
    for F, G, om in ((dec["U"], Lr, om_r_o), (dec["V"], Lc, om_c_o)):
        F = F.double().cpu().numpy()
        assert np.allclose(np.linalg.norm(F, axis=0), 1.0, atol=1e-5)
        # the sampled rows keep orthogonal columns (they are scaled SVD vectors)
        Gm = F[om].T @ F[om]
        dg = np.sqrt(np.diag(Gm))
        assert np.abs(Gm - np.diag(np.diag(Gm))).max() <= 1e-5 * dg.max() ** 2
        # Lemma 1: (L F)(a, :) = 0 on the unsampled rows a, to the CG
        # tolerance plus the rounding of F to FP32 (|L| |F| times a few ulps)
        Ls = G.to_scipy()
        mask = np.ones(Ls.shape[0], dtype=bool)
        mask[om] = False
        La = Ls[mask]
        res = np.linalg.norm(La @ F, axis=0)
        rhs = np.linalg.norm(La[:, om] @ F[om], axis=0)
        rnd = np.linalg.norm(abs(La) @ np.abs(F), axis=0) * 64 * 2.0 ** -24
        assert np.all(res <= 2 * cfg["cg_tol"] * rhs + rnd)
    U, V = dec["U"].double().cpu().numpy(), dec["V"].double().cpu().numpy()
    ii, jj = rng.integers(0, p, 4096), rng.integers(0, n, 4096)
    terms = U[ii] * sig * V[jj]
    got = dec["X"][torch.as_tensor(ii, device="cuda"), torch.as_tensor(jj, device="cuda")]
    err = np.abs(got.double().cpu().numpy() - terms.sum(axis=1))
    assert np.all(err <= 1e-5 * np.abs(terms).sum(axis=1) + 1e-30)
