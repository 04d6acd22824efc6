"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, from the spec contract): FISTA and decoded
matrices within 1e-4 relative Frobenius error after a fixed iteration count,
converged objectives within 1e-5 relative; sampling indices and kNN
neighbour sets bit-exact (kNN sets may differ only where the K-th and
(K+1)-th exact distances are within 1e-6 relative); FP32 squared distances
and Laplacian values within 2e-6 / 1e-5 relative of FP64.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle as O
from tests._util import knn_sets_match, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FISTA_TOL = 1e-4
DECODE_TOL = 1e-4
OBJ_TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("seed,p,n,rr,rc", [(0, 256, 512, 128, 256), (7, 10304, 1000, 2576, 250),
                                            (3, 37, 53, 1, 53), (11, 100000, 5, 9973, 2)])
def test_sample_bit_exact(M, seed, p, n, rr, rc):
    om_r, om_c, _ = M.cpca_sample(seed, p, n, rr, rc)
    assert np.array_equal(om_r.cpu().numpy(), O.sample_indices(seed, p, rr, 0))
    assert np.array_equal(om_c.cpu().numpy(), O.sample_indices(seed, n, rc, 1))


def test_gather_exact(M):
    Y, _, _ = gen.make_instance(1, 97, 131, 3, 3, 0.05)
    om_r, om_c, Yt = M.cpca_sample(5, 97, 131, 31, 45, _dev(Y))
    r, c = om_r.cpu().numpy(), om_c.cpu().numpy()
    assert np.array_equal(Yt.cpu().numpy(), Y[np.ix_(r, c)])


# ----------------------------------------------------------------------- kNN
def _oracle_sorted_d2(P, queries):
    P = np.asarray(P, dtype=np.float64)
    out = []
    for i in queries:
        d = np.einsum("ij,ij->i", P - P[i], P - P[i])
        d[i] = np.inf
        out.append(np.sort(d))
    return out


@pytest.mark.parametrize("shape,transposed,K", [((256, 512), False, 10), ((256, 512), True, 10),
                                                ((129, 37), False, 7), ((300, 70), True, 10),
                                                ((66, 9), False, 32)])
def test_knn_lists_and_graph(M, shape, transposed, K):
    Y, _, _ = gen.make_instance(2, shape[0], shape[1], 4, 3, 0.05)
    P = Y.T if transposed else Y
    Lg, gi, gd = M.cpca_knn_graph(_dev(Y), K, M.LAP_NORMALIZED, transposed=transposed, want_knn=True)
    oi, od = O.knn_bruteforce(P, K)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    full = _oracle_sorted_d2(P, range(P.shape[0]))
    assert knn_sets_match(gi, gd, oi, full, K, rel_gap=1e-6) == []
    # Undecided FP32 orderings are settled in FP64, so the sets agree exactly
    # (a difference could only come from a gap below FP64 summation-order
    # rounding, ~1e-13 relative, which these seeded inputs do not have).
    same = np.all(np.sort(gi, 1) == np.sort(oi, 1), axis=1)
    assert same.all()
    assert np.allclose(gd, od, rtol=2e-6, atol=0)
    # graph on the oracle's rules, from the oracle's kNN lists
    L, W = O.laplacian_from_knn(oi, od, P.shape[0], O.sigma2_mean(od), O.LAP_NORMALIZED)
    assert Lg.sigma2 == pytest.approx(O.sigma2_mean(od), rel=1e-6)
    Gs = Lg.to_scipy()
    assert np.array_equal(Gs.indptr, L.indptr) and np.array_equal(Gs.indices, L.indices)
    assert np.allclose(Gs.data, L.data, rtol=1e-5, atol=1e-7)
    Wg = sp.csr_matrix((Lg.weight.double().cpu().numpy(), Gs.indices, Gs.indptr), shape=Gs.shape)
    assert abs(Wg - W).max() < 1e-6
    assert abs(Gs - Gs.T).max() == 0.0  # exactly symmetric


@pytest.mark.parametrize("shape,transposed,K", [((300, 40000), False, 10), ((33001, 260), True, 10),
                                                ((150, 34000), False, 20)])
def test_knn_chunked_accumulation_high_dimension(M, shape, transposed, K):
    """Points in more than 32768 dimensions: the tensor-core ranking adds its
    products in accumulation chunks of 4096 dimensions (a ragged last chunk
    for 33001), and the certificate uses the chunked bound. The lists are
    the exact ones (the oracle's C search) and the graph follows from them
    by the oracle's rules."""
    from tests._oracle_knn import oracle_knn_graph
    Y, _, _ = gen.make_instance(4, shape[0], shape[1], 4, 3, 0.05)
    P = np.ascontiguousarray(Y.T if transposed else Y)
    Lg, gi, gd = M.cpca_knn_graph(_dev(Y), K, M.LAP_NORMALIZED, transposed=transposed, want_knn=True)
    d = P.shape[1]
    chunks = -(-(-(-d // 64)) // 64)  # k-steps of 64 dimensions, 64 k-steps per chunk
    assert M.knn_last_err_rel() == pytest.approx(2.0**-10 + 2.0**-22 + (4096 + 8 + chunks) * 2.0**-23, rel=1e-6)
    assert M.knn_last_uncertified() == 0
    L, _, oi, od = oracle_knn_graph(P, K)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert knn_sets_match(gi, gd, oi[:, :K], od, K, rel_gap=1e-6) == []
    assert np.all(np.sort(gi, 1) == np.sort(oi[:, :K], 1))
    assert np.allclose(gd, od[:, :K], rtol=2e-6, atol=0)
    Gs = Lg.to_scipy()
    assert np.array_equal(Gs.indptr, L.indptr) and np.array_equal(Gs.indices, L.indices)
    assert np.allclose(Gs.data, L.data, rtol=1e-5, atol=1e-7)


def test_knn_combinatorial_zero_row_sums(M):
    Y, _, _ = gen.make_instance(3, 200, 60, 4, 3, 0.05)
    Lg, _, _ = M.cpca_knn_graph(_dev(Y), 10, M.LAP_COMBINATORIAL)
    Ls = Lg.to_scipy()
    assert np.abs(np.asarray(Ls.sum(1))).max() < 1e-5 * np.abs(Ls.diagonal()).max()


# --------------------------------------------------------------------- FISTA
def _compressed(seed=0, p=256, n=512, r=5, C=4, fr=0.5, fc=0.5, K=10):
    Y, _, _ = gen.make_instance(seed, p, n, r, C, 0.05)
    rr, rc = max(1, int(p * fr + 0.5)), max(1, int(n * fc + 0.5))
    om_r, om_c = O.sample_indices(seed, p, rr, 0), O.sample_indices(seed, n, rc, 1)
    Yt = Y.astype(np.float64)[np.ix_(om_r, om_c)]
    Lr, *_ = O.knn_graph(Yt, K)
    Lc, *_ = O.knn_graph(Yt.T, K)
    return Y, Yt, Lr, Lc, om_r, om_c


@pytest.fixture(scope="module")
def c0():
    return _compressed()


def test_power_norms_match(M, c0):
    _, Yt, Lr, Lc, *_ = c0
    X, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                  gamma_r=1.0, gamma_c=1.0, max_iter=0, power_iters=200)
    assert info.norm_r == pytest.approx(O.power_norm(Lr, 200, 0, 2), rel=1e-6)
    assert info.norm_c == pytest.approx(O.power_norm(Lc, 200, 0, 3), rel=1e-6)
    lam = O.fista_step(1.0, 1.0, info.norm_r, info.norm_c)
    assert info.step == pytest.approx(lam, rel=1e-12)
    assert np.array_equal(X.cpu().numpy(), Yt.astype(np.float32))


@pytest.mark.parametrize("gr,gc,J", [(1.0, 1.0, 200), (0.3, 2.0, 57), (5.0, 0.1, 300)])
def test_fista_fixed_iterations(M, c0, gr, gc, J):
    _, Yt, Lr, Lc, *_ = c0
    lam = O.fista_step(gr, gc, O.power_norm(Lr), O.power_norm(Lc))
    Xo, _ = O.frpcag_fista(Yt, Lr, Lc, gr, gc, lam, J)
    Xg, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                   gamma_r=gr, gamma_c=gc, step=lam, max_iter=J)
    assert info.iters == J
    assert rel_fro(Xg.cpu().numpy(), Xo) < FISTA_TOL
    Fo = O.frpcag_objective(Xo, Yt, Lr, Lc, gr, gc)
    assert info.objective == pytest.approx(Fo, rel=1e-5)


def test_fista_gamma_zero_is_data(M, c0):
    _, Yt, Lr, Lc, *_ = c0
    Xg, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                   gamma_r=0.0, gamma_c=0.0, max_iter=40)
    assert info.step == 1.0
    assert np.array_equal(Xg.cpu().numpy(), Yt.astype(np.float32))


def test_fista_converged_objective(M):
    _, Yt, Lr, Lc, *_ = _compressed(seed=4, p=60, n=90, fr=0.5, fc=0.5, K=5)
    lam = O.fista_step(1, 1, O.power_norm(Lr), O.power_norm(Lc))
    Xo, _ = O.frpcag_fista(Yt, Lr, Lc, 1.0, 1.0, lam, 20000)
    Fo = O.frpcag_objective(Xo, Yt, Lr, Lc, 1.0, 1.0)
    Xg, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                   gamma_r=1.0, gamma_c=1.0, step=lam, max_iter=20000)
    assert abs(info.objective - Fo) / Fo < OBJ_TOL


@pytest.mark.parametrize("shape,eps,J", [((301, 3003), 0.0, 150), ((301, 3003), 1e-7, 3000),
                                         ((300, 14003), 0.0, 60)])
def test_fista_striped_launch_equals_cooperative(M, shape, eps, J):
    """A problem too large for the resident launch (301 x 3003: ragged row
    boxes, a ragged last stripe and padded leading dimensions; 300 x 14003,
    large enough to be processed in the column graph's locality order)
    takes the striped per-iteration launch by default; forcing a launch
    width takes the cooperative streaming kernel. Same arithmetic in the
    same order: the same iterates bit for bit (and, with the stopping rule,
    the same stop up to the FP64 order of the statistics)."""
    Y, _, _ = gen.make_instance(31, shape[0], shape[1], 6, 5 if shape[1] < 10000 else 40, 0.05)
    Lr = _graph_c(Y, 8)
    Lc = _graph_c(np.ascontiguousarray(Y.T), 8)
    Yd, Lrd, Lcd = _dev(Y), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc)
    M.profile_enable(True, "fista_")
    Xs, i_s = M.cpca_frpcag_solve(Yd, Lrd, Lcd, gamma_r=0.7, gamma_c=1.3, max_iter=J, eps=eps)
    prof = M.profile_read()
    M.profile_enable(False, "")
    assert "fista_stripe" in prof
    Xc, i_c = M.cpca_frpcag_solve(Yd, Lrd, Lcd, gamma_r=0.7, gamma_c=1.3, max_iter=J, eps=eps,
                                  blocks=2 * 152)
    if eps == 0:
        assert i_s.iters == i_c.iters == J
        assert torch.equal(Xs, Xc)
        lam = O.fista_step(0.7, 1.3, O.power_norm(Lr), O.power_norm(Lc, 200, 0, 3))
        Xo, _ = O.frpcag_fista(Y.astype(np.float64), Lr, Lc, 0.7, 1.3, lam, J)
        assert rel_fro(Xs.cpu().numpy(), Xo) < FISTA_TOL
    else:
        assert abs(i_s.iters - i_c.iters) <= 1 and i_s.iters < J
        assert rel_fro(Xs.cpu().numpy(), Xc.cpu().numpy()) < 1e-5


def _graph_c(P, K):
    from tests._oracle_knn import oracle_knn_graph
    return oracle_knn_graph(P, K)[0]


def _kkt(X, Yt, Lr, Lc, gr, gc):
    """l1 optimality residuals of X (FP64 products): |G + sgn(X - Y~)| where
    X != Y~ and (|G| - 1)_+ where X == Y~, G = 2 (gr Lr X + gc X Lc)."""
    G = 2.0 * (gr * (Lr @ X) + gc * (Lc @ X.T).T)
    on = X != Yt
    return (np.max(np.abs(G[on] + np.sign(X - Yt)[on]), initial=0.0),
            np.max(np.maximum(np.abs(G[~on]) - 1.0, 0.0), initial=0.0), on.mean())


@pytest.mark.parametrize("which", ["small", "10304x1000"])
def test_fista_kkt_with_library_step(M, which):
    """lambda from the library's own 200 power iterations (step <= 0; the
    estimate sits up to 0.7% below |L|_2 at the workloads' sizes, so lambda
    can exceed 1/beta slightly): FISTA still reaches the l1 optimality
    conditions of Eq. frpcag_small."""
    if which == "small":
        _, Yt, Lr, Lc, *_ = _compressed(seed=4, p=60, n=90, fr=0.5, fc=0.5, K=5)
        J = 20000
    else:
        cfg = gen.CONFIGS["bench_10304x1000"]
        _, Yt, Lr, Lc, *_ = _compressed(0, cfg["p"], cfg["n"], cfg["r"], cfg["C"], cfg["fr"], cfg["fc"], cfg["K"])
        J = 20000
    Xg, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                   gamma_r=1.0, gamma_c=1.0, max_iter=J)
    assert info.step == pytest.approx(O.fista_step(1.0, 1.0, O.power_norm(Lr), O.power_norm(Lc, 200, 0, 3)),
                                      rel=1e-6)
    X = Xg.double().cpu().numpy()
    r_on, r_off, frac_on = _kkt(X, Yt.astype(np.float32).astype(np.float64), Lr, Lc, 1.0, 1.0)
    assert 0.0 < frac_on < 1.0
    assert r_on < 1e-3 and r_off < 1e-3


def test_fista_stopping_rule_matches(M, c0):
    _, Yt, Lr, Lc, *_ = c0
    lam = O.fista_step(1, 1, O.power_norm(Lr), O.power_norm(Lc))
    Xo, oi = O.frpcag_fista(Yt, Lr, Lc, 1.0, 1.0, lam, 5000, eps=1e-7)
    Xg, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                   gamma_r=1.0, gamma_c=1.0, step=lam, max_iter=5000, eps=1e-7)
    assert abs(info.iters - oi["iters"]) <= 2
    assert rel_fro(Xg.cpu().numpy(), Xo) < 1e-3


@pytest.mark.parametrize("rr,rc", [(1, 7), (5, 1), (33, 65), (97, 250), (300, 1001)])
def test_fista_ragged_shapes(M, rr, rc):
    rng = np.random.default_rng(rr * 1000 + rc)
    Yt = rng.standard_normal((rr, rc))
    Lr = O.knn_graph(Yt, min(4, rr - 1))[0] if rr > 2 else sp.csr_matrix(np.zeros((rr, rr)) + 0 * np.eye(rr))
    Lc = O.knn_graph(Yt.T, min(4, rc - 1))[0] if rc > 2 else sp.csr_matrix(np.zeros((rc, rc)) + 0 * np.eye(rc))
    Lr = sp.csr_matrix(Lr + sp.csr_matrix((np.zeros(rr), (np.arange(rr), np.arange(rr))), shape=(rr, rr)))
    Lc = sp.csr_matrix(Lc + sp.csr_matrix((np.zeros(rc), (np.arange(rc), np.arange(rc))), shape=(rc, rc)))
    lam = O.fista_step(0.7, 1.3, O.power_norm(Lr), O.power_norm(Lc))
    Xo, _ = O.frpcag_fista(Yt, Lr, Lc, 0.7, 1.3, lam, 60)
    Xg, _ = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                gamma_r=0.7, gamma_c=1.3, step=lam, max_iter=60)
    assert rel_fro(Xg.cpu().numpy(), Xo) < FISTA_TOL


# -------------------------------------------------------------------- decode
@pytest.fixture(scope="module")
def c0_decode(c0):
    Y, Yt, Lr_t, Lc_t, om_r, om_c = c0
    Lr, *_ = O.knn_graph(Y, 10)
    Lc, *_ = O.knn_graph(Y.T, 10)
    lam = O.fista_step(1, 1, O.power_norm(Lr_t), O.power_norm(Lc_t))
    Xt, _ = O.frpcag_fista(Yt, Lr_t, Lc_t, 1.0, 1.0, lam, 200)
    return Y, Xt, Lr, Lc, om_r, om_c


def test_decode_matches_oracle(M, c0_decode):
    Y, Xt, Lr, Lc, om_r, om_c = c0_decode
    p, n = Y.shape
    do = O.approx_decode(Xt, om_r, om_c, p, n, Lr, Lc, tol=1e-6)
    dg = M.cpca_decode(_dev(Xt), torch.as_tensor(om_r, dtype=torch.int32, device="cuda"),
                       torch.as_tensor(om_c, dtype=torch.int32, device="cuda"), p, n,
                       M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc), cg_tol=1e-6)
    assert dg["k"] == do["k"]
    s = np.array(dg["info"].s_tilde[:dg["k"]])
    assert np.allclose(s, do["s_tilde"][:do["k"]], rtol=1e-5)
    assert rel_fro(dg["X"].cpu().numpy(), do["X"]) < DECODE_TOL
    assert np.allclose(dg["sigma"].cpu().numpy(), do["sigma"], rtol=1e-5)


def test_decode_into_pinned_host_output(M, c0_decode):
    """X written by the output kernel straight into page-locked host memory
    equals the device-resident X bit for bit (same kernel, same arithmetic);
    a pageable host buffer is refused before any launch."""
    Y, Xt, Lr, Lc, om_r, om_c = c0_decode
    p, n = Y.shape
    args = (_dev(Xt), torch.as_tensor(om_r, dtype=torch.int32, device="cuda"),
            torch.as_tensor(om_c, dtype=torch.int32, device="cuda"), p, n,
            M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc))
    dd = M.cpca_decode(*args, cg_tol=1e-6)
    Xh = torch.full((p, n), float("nan"), dtype=torch.float32).pin_memory()
    dh = M.cpca_decode(*args, cg_tol=1e-6, out=Xh)
    assert dh["X"] is Xh and dh["k"] == dd["k"]
    assert torch.equal(Xh, dd["X"].cpu())
    with pytest.raises(ValueError):
        M.cpca_decode(*args, cg_tol=1e-6, out=torch.empty(p, n, dtype=torch.float32))


def test_decode_full_sampling_and_override(M):
    rng = np.random.default_rng(9)
    Xt = rng.standard_normal((40, 3)) @ np.diag([10.0, 5.0, 2.0]) @ rng.standard_normal((3, 50))
    Lr, *_ = O.knn_graph(rng.standard_normal((40, 3)), 4)
    Lc, *_ = O.knn_graph(rng.standard_normal((50, 3)), 4)
    om_r, om_c = np.arange(40), np.arange(50)
    do = O.approx_decode(Xt, om_r, om_c, 40, 50, Lr, Lc)
    dg = M.cpca_decode(_dev(Xt), torch.arange(40, dtype=torch.int32, device="cuda"),
                       torch.arange(50, dtype=torch.int32, device="cuda"), 40, 50,
                       M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc))
    assert dg["k"] == do["k"] == 3
    assert rel_fro(dg["X"].cpu().numpy(), do["X"]) < DECODE_TOL
    do2 = O.approx_decode(Xt, om_r, om_c, 40, 50, Lr, Lc, k_override=2)
    dg2 = M.cpca_decode(_dev(Xt), torch.arange(40, dtype=torch.int32, device="cuda"),
                        torch.arange(50, dtype=torch.int32, device="cuda"), 40, 50,
                        M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc), k_override=2)
    assert dg2["k"] == 2 and rel_fro(dg2["X"].cpu().numpy(), do2["X"]) < DECODE_TOL


def test_decode_singular_component_reported(M):
    # two components; the second has no sampled node -> L_aa singular
    rng = np.random.default_rng(14)
    P = np.vstack([rng.standard_normal((20, 2)), 100.0 + rng.standard_normal((20, 2))])
    L, *_ = O.knn_graph(P, 4, O.LAP_COMBINATORIAL)
    Lc, *_ = O.knn_graph(rng.standard_normal((12, 2)), 3)
    Xt = rng.standard_normal((5, 12))
    om_r = torch.tensor([0, 3, 7, 9, 12], dtype=torch.int32, device="cuda")
    om_c = torch.arange(12, dtype=torch.int32, device="cuda")
    Xt[:, :] = np.outer(np.ones(5), rng.standard_normal(12))
    with pytest.raises(M.CpcaError) as e:
        M.cpca_decode(_dev(Xt), om_r, om_c, 40, 12, M.Csr.from_scipy(L), M.Csr.from_scipy(Lc),
                      cg_max_iter=400)
    assert e.value.status in (M.CPCA_ERR_SINGULAR, M.CPCA_ERR_NOT_CONVERGED)


# ------------------------------------------------------------------ pipeline
def test_pipeline_c0_end_to_end(M):
    cfg = gen.CONFIGS["small_256x512"]
    Y, _, _ = gen.make_instance(0, cfg["p"], cfg["n"], cfg["r"], cfg["C"], cfg["frac"])
    rr, rc = M.rho_of(cfg["p"], cfg["fr"]), M.rho_of(cfg["n"], cfg["fc"])
    out = M.cpca_pipeline(_dev(Y), K=cfg["K"], fr=cfg["fr"], fc=cfg["fc"], seed=0, J=cfg["J"])
    ref = O.cpca(Y, cfg["K"], rr, rc, 0, cfg["J"], 1.0, 1.0)
    assert np.array_equal(out["omega_r"].cpu().numpy(), ref["omega_r"])
    assert np.array_equal(out["omega_c"].cpu().numpy(), ref["omega_c"])
    assert rel_fro(out["Xt"].cpu().numpy(), ref["Xt"]) < FISTA_TOL
    assert out["k"] == ref["k"]
    assert rel_fro(out["X"].cpu().numpy(), ref["X"]) < DECODE_TOL


# ---------------------------------------------------------- warm start
@pytest.mark.parametrize("case", ["resident", "striped", "striped_reordered", "beyond_mu_table"])
def test_fista_warm_start_resumes_bit_for_bit(M, case):
    """Checkpoint and resume of Algorithm 1: J1 iterations (exporting
    S_{J1-1}) followed by J2 resumed iterations equal one run of J1 + J2,
    bit for bit, in the resident launch, the striped launch, and across the
    end of the momentum table (t_j continued on the host)."""
    if case in ("striped", "striped_reordered"):
        shape = (301, 3003) if case == "striped" else (300, 14003)
        Y, _, _ = gen.make_instance(32, shape[0], shape[1], 6, 40, 0.05)
        Lr, Lc = _graph_c(Y, 8), _graph_c(np.ascontiguousarray(Y.T), 8)
        Yt = Y.astype(np.float64)
        J1, J2 = 40, 35
    else:
        _, Yt, Lr, Lc, *_ = _compressed(seed=6, p=120, n=200, fr=0.5, fc=0.5, K=6)
        J1, J2 = (70, 55) if case == "resident" else (8190, 5)
    Yd, Lrd, Lcd = _dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc)
    kw = dict(gamma_r=0.9, gamma_c=1.1)
    full, info = M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=J1 + J2, **kw)
    X = torch.empty_like(full)
    prev = torch.empty_like(full)
    _, i1 = M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=J1, out=X, prev_out=prev, **kw)
    prev2 = torch.empty_like(full)
    X2, i2 = M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=J2, out=X, start_iter=J1, start_prev=prev,
                                 prev_out=prev2, **kw)
    assert i1.iters == J1 and i2.iters == J2 and i1.step == info.step == i2.step
    assert torch.equal(X2, full)
    # the exported pair resumes again: one more iteration equals J1 + J2 + 1
    full1, _ = M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=J1 + J2 + 1, **kw)
    X3, _ = M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=1, out=X2.clone(), start_iter=J1 + J2,
                                start_prev=prev2, **kw)
    assert torch.equal(X3, full1)


def test_fista_warm_start_argument_errors(M):
    _, Yt, Lr, Lc, *_ = _compressed(seed=6, p=40, n=60, fr=0.5, fc=0.5, K=4)
    Yd, Lrd, Lcd = _dev(Yt), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc)
    with pytest.raises(M.CpcaError) as e:
        M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=5, start_iter=3)  # no S_{j0-1}
    assert e.value.status == M.CPCA_ERR_INVALID_ARG
    with pytest.raises(M.CpcaError) as e:
        M.cpca_frpcag_solve(Yd, Lrd, Lcd, max_iter=5, eps=1e-6, prev_out=torch.empty_like(Yd))
    assert e.value.status == M.CPCA_ERR_INVALID_ARG
