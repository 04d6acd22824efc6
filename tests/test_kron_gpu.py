"""Kron-reduced compressed Laplacians (Sec. IV-A) through the C ABI against
the FP64 oracle, and FISTA on them.

Bars (written here). The reduction: relative Frobenius error <= 1e-5 and
every entry within 1e-5 of the largest diagonal entry. Each column comes
from a Jacobi PCG run to relative residual 1e-6 in FP32 (the same solver
as the decoder); an FP32 emulation of that solver on these graphs lands at
about 1e-7, so the bars leave two orders of magnitude for rounding order.
Entries with no path through unsampled nodes are exactly 0 on both sides
(the PCG iterates never leave the support of their right-hand side), and
the result is exactly symmetric (it is symmetrised). FISTA fed the
oracle's reduced Laplacians: relative Frobenius 1e-4 after J iterations
(the bar of the sparse graphs), norms within 1e-6; at 10304 x 1000 each
side runs on its own reductions (they differ by ~1e-7), so the norms are
held to 1e-5 there. The dense contraction kernel and the gather kernel
agree to 1e-5 (FP32 sums in different orders).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import gen
import oracle as O
from oracle import cpca_kron as KR
from tests._oracle_knn import oracle_knn_graph
from tests._util import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KRON_TOL = 1e-5
FISTA_TOL = 1e-4


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a, dt=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda")


def _reachable_pairs(L, omega):
    """[a, b] True when kept nodes omega[a] != omega[b] are joined by an edge
    or by a path through unsampled nodes only (breadth-first search)."""
    L = sp.csr_matrix(L)
    N = L.shape[0]
    sampled = np.zeros(N, dtype=bool)
    sampled[omega] = True
    pos = -np.ones(N, dtype=np.int64)
    pos[omega] = np.arange(len(omega))
    out = np.zeros((len(omega), len(omega)), dtype=bool)
    for a, s in enumerate(omega):
        seen = np.zeros(N, dtype=bool)
        seen[s] = True
        stack = [int(s)]
        while stack:
            u = stack.pop()
            for e in range(L.indptr[u], L.indptr[u + 1]):
                v = L.indices[e]
                if v == u or L.data[e] == 0:
                    continue
                if sampled[v]:
                    out[a, pos[v]] = True
                elif not seen[v]:
                    seen[v] = True
                    stack.append(int(v))
    np.fill_diagonal(out, False)
    return out


def _check_reduction(res, Lo, L, omega):
    Lt = res["Lt"].cpu().numpy().astype(np.float64)
    assert rel_fro(Lt, Lo) < KRON_TOL
    assert np.abs(Lt - Lo).max() <= KRON_TOL * np.abs(np.diag(Lo)).max()
    assert np.array_equal(Lt, Lt.T)
    reach = _reachable_pairs(L, omega)
    off = ~np.eye(len(omega), dtype=bool)
    assert np.all(Lt[off & ~reach] == 0.0)
    if res["csr"] is not None:
        C = res["csr"].to_scipy().toarray()
        assert np.array_equal(C, Lt)


@pytest.mark.parametrize("lap_type", [O.LAP_NORMALIZED, O.LAP_COMBINATORIAL])
@pytest.mark.parametrize("N,dim,rho", [(300, 450, 77), (260, 120, 130), (90, 64, 20)])
def test_kron_matches_oracle(M, lap_type, N, dim, rho):
    """Chunks of 48 columns with a ragged last chunk (77 = 48 + 29,
    130 = 48 + 48 + 34) and a single short chunk (20)."""
    Y, _, _ = gen.make_instance(11, N, dim, 5, 4, 0.05)
    L, *_ = O.knn_graph(Y, 10, lap_type)
    om = O.sample_indices(11, N, rho, 0)
    Lo = KR.kron_reduce(L, om)
    res = M.cpca_kron_reduce(M.Csr.from_scipy(L), _dev(om, np.int32), tol=1e-6)
    assert res["info"].chunks == (rho + 47) // 48
    assert res["info"].cg_res <= 1e-6
    _check_reduction(res, Lo, L, om)


def test_kron_sparse_graph_with_exact_zeros(M):
    """A sparse graph (K = 2) where many kept pairs are not joined through
    unsampled nodes: those entries are exactly zero."""
    Y, _, _ = gen.make_instance(12, 200, 40, 3, 5, 0.0)
    L, *_ = O.knn_graph(Y, 2)
    ncomp, comp = csg.connected_components(L - sp.diags(L.diagonal()), directed=False)
    om = np.unique(np.concatenate([[np.flatnonzero(comp == c)[0] for c in range(ncomp)],
                                   O.sample_indices(12, 200, 60, 0)]))
    Lo = KR.kron_reduce(L, om)
    res = M.cpca_kron_reduce(M.Csr.from_scipy(L), _dev(om, np.int32), want_csr=False)
    assert res["csr"] is None
    _check_reduction(res, Lo, L, om)
    assert np.count_nonzero(res["Lt"].cpu().numpy()) < 0.5 * len(om) ** 2


def test_kron_full_sampling_returns_L(M):
    Y, _, _ = gen.make_instance(13, 120, 50, 3, 3, 0.05)
    L, *_ = O.knn_graph(Y, 6)
    res = M.cpca_kron_reduce(M.Csr.from_scipy(L), _dev(np.arange(120), np.int32))
    assert np.array_equal(res["Lt"].cpu().numpy(), L.toarray().astype(np.float32))


def test_kron_component_without_sample_is_singular(M):
    W = np.zeros((20, 20))
    for i in range(9):
        W[i, i + 1] = W[i + 1, i] = 1.0
    for i in range(10, 19):
        W[i, i + 1] = W[i + 1, i] = 0.5
    L = O.laplacian_from_weights(sp.csr_matrix(W), O.LAP_NORMALIZED)
    res = M.cpca_kron_reduce(M.Csr.from_scipy(L), _dev([1, 4, 8], np.int32), check_status=False)
    assert res["status"] == M.CPCA_ERR_SINGULAR


def test_kron_rejects_unsorted_omega(M):
    Y, _, _ = gen.make_instance(14, 64, 32, 3, 3, 0.05)
    L, *_ = O.knn_graph(Y, 6)
    for bad in ([5, 3, 9], [2, 2, 7], [1, 4, 64]):
        with pytest.raises(M.CpcaError) as e:
            M.cpca_kron_reduce(M.Csr.from_scipy(L), _dev(bad, np.int32))
        assert e.value.status == M.CPCA_ERR_INVALID_ARG


def test_fista_on_kron_graphs_matches_oracle(M):
    """256 x 512 (rank 5, 4 clusters, 5% gross errors), 1/2 x 1/2 sampling,
    J = 200: FISTA on the oracle's Kron-reduced Laplacians (dense CSR)."""
    cfg = gen.CONFIGS["small_256x512"]
    p, n, J = cfg["p"], cfg["n"], cfg["J"]
    Y, _, _ = gen.make_instance(0, p, n, cfg["r"], cfg["C"], cfg["frac"])
    Lr, *_ = O.knn_graph(Y, cfg["K"])
    Lc, *_ = O.knn_graph(Y.T, cfg["K"])
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    om_r, om_c = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    Yt = O.sample_matrix(Y.astype(np.float64), om_r, om_c)
    Lrt, Lct = KR.kron_reduce(Lr, om_r), KR.kron_reduce(Lc, om_c)
    nr, nc = O.power_norm(Lrt, 200, 0, 2), O.power_norm(Lct, 200, 0, 3)
    Xo, _ = O.frpcag_fista(Yt, Lrt, Lct, 1.0, 1.0, O.fista_step(1.0, 1.0, nr, nc), J)
    X, info = M.cpca_frpcag_solve(_dev(Yt), M.Csr.from_scipy(KR.kron_reduce_csr(Lr, om_r)),
                                  M.Csr.from_scipy(KR.kron_reduce_csr(Lc, om_c)), gamma_r=1.0, gamma_c=1.0,
                                  max_iter=J)
    assert info.norm_r == pytest.approx(nr, rel=1e-6)
    assert info.norm_c == pytest.approx(nc, rel=1e-6)
    assert rel_fro(X.cpu().numpy(), Xo) < FISTA_TOL


@pytest.mark.parametrize("N,dim,rr,rc,gr,gc", [(300, 260, 77, 45, 1.0, 1.0), (256, 512, 128, 256, 0.0, 2.0),
                                                (256, 512, 128, 256, 0.5, 0.0)])
def test_dense_fista_path_matches_gather_path_and_oracle(M, N, dim, rr, rc, gr, gc):
    """Dense Laplacians (every entry stored, row-major) take the dense
    contraction kernel, one launch per iteration; an explicit launch width
    keeps the gather kernel. Both against each other and the oracle, with a
    ragged tile edge (77 x 45) and either gamma zero."""
    Y, _, _ = gen.make_instance(21, N, dim, 4, 3, 0.05)
    Lr, *_ = O.knn_graph(Y, 10)
    Lc, *_ = O.knn_graph(Y.T, 10)
    om_r, om_c = O.sample_indices(21, N, rr, 0), O.sample_indices(21, dim, rc, 1)
    Yt = O.sample_matrix(Y.astype(np.float64), om_r, om_c)
    Lrt, Lct = KR.kron_reduce(Lr, om_r), KR.kron_reduce(Lc, om_c)
    nr, nc = O.power_norm(Lrt, 200, 0, 2), O.power_norm(Lct, 200, 0, 3)
    J = 150
    Xo, _ = O.frpcag_fista(Yt, Lrt, Lct, gr, gc, O.fista_step(gr, gc, nr, nc), J)
    Gr = M.Csr.from_scipy(KR.kron_reduce_csr(Lr, om_r))
    Gc = M.Csr.from_scipy(KR.kron_reduce_csr(Lc, om_c))
    M.profile_enable(True, "fista_")
    Xd, infod = M.cpca_frpcag_solve(_dev(Yt), Gr, Gc, gamma_r=gr, gamma_c=gc, max_iter=J)
    torch.cuda.synchronize()
    used = M.profile_read()
    M.profile_enable(False, "")
    assert "fista_dense" in used and "fista_persistent" not in used
    Xg, infog = M.cpca_frpcag_solve(_dev(Yt), Gr, Gc, gamma_r=gr, gamma_c=gc, max_iter=J, blocks=152)
    assert infod.iters == infog.iters == J
    assert infod.step == infog.step
    assert rel_fro(Xd.cpu().numpy(), Xg.cpu().numpy()) < 1e-5
    assert rel_fro(Xd.cpu().numpy(), Xo) < FISTA_TOL
    assert infod.rel_change > 0 and infod.rel_change == pytest.approx(infog.rel_change, rel=0.5)
    assert infod.objective == pytest.approx(infog.objective, rel=1e-5)


def test_kron_full_size_and_fista(M):
    """10304 x 1000 (rank 10, 10 clusters, 1/4 x 1/4 sampling): the oracle's
    full graphs of Y's rows (10304 nodes) and columns (1000 nodes) reduced
    onto the sampled 2576 rows and 250 columns, then 30 FISTA iterations on
    the reduced Laplacians (dense CSR, 6.6 M entries for the rows)."""
    cfg = gen.CONFIGS["bench_10304x1000"]
    p, n, K = cfg["p"], cfg["n"], cfg["K"]
    Y, _, _ = gen.make_instance(0, p, n, cfg["r"], cfg["C"], cfg["frac"])
    Yd = Y.astype(np.float64)
    Lr, _, _, _ = oracle_knn_graph(Y, K)
    Lc, _, _, _ = oracle_knn_graph(Y.T, K)
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    om_r, om_c = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    Lrt_o, Lct_o = KR.kron_reduce(Lr, om_r), KR.kron_reduce(Lc, om_c)
    rr_res = M.cpca_kron_reduce(M.Csr.from_scipy(Lr), _dev(om_r, np.int32))
    rc_res = M.cpca_kron_reduce(M.Csr.from_scipy(Lc), _dev(om_c, np.int32))
    for res, Lo, L, om in ((rr_res, Lrt_o, Lr, om_r), (rc_res, Lct_o, Lc, om_c)):
        Lt = res["Lt"].cpu().numpy().astype(np.float64)
        assert rel_fro(Lt, Lo) < KRON_TOL
        assert np.abs(Lt - Lo).max() <= KRON_TOL * np.abs(np.diag(Lo)).max()
        assert np.array_equal(Lt, Lt.T)
    J = 30
    Yt = O.sample_matrix(Yd, om_r, om_c)
    nr, nc = O.power_norm(Lrt_o, 200, 0, 2), O.power_norm(Lct_o, 200, 0, 3)
    Xo, _ = O.frpcag_fista(Yt, Lrt_o, Lct_o, 1.0, 1.0, O.fista_step(1.0, 1.0, nr, nc), J)
    X, info = M.cpca_frpcag_solve(_dev(Yt), rr_res["csr"], rc_res["csr"], gamma_r=1.0, gamma_c=1.0, max_iter=J)
    assert info.norm_r == pytest.approx(nr, rel=1e-5)
    assert info.norm_c == pytest.approx(nc, rel=1e-5)
    assert rel_fro(X.cpu().numpy(), Xo) < FISTA_TOL
