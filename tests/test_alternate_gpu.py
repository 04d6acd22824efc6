"""Alternate decoder (Sec. V-B, Eq. alternatedecoder): CUDA PCG through the
C ABI against the FP64 oracle's exact solve.

Tolerances (written here): the PCG stops at relative residual 1e-6 in FP32
vectors with FP64 dot products; the decoded X must match the exact
minimiser within 1e-4 relative Frobenius error (the benchmark spec's bound for
decoded matrices), and its FP64 residual in the normal equations, evaluated
on the CPU from the definition, must be below 1e-5 |B| (the solver's
1e-6 plus FP32 rounding of X and of the recursively updated residual).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle as O
from oracle import cpca_decoders as D
from tests._util import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DECODE_TOL = 1e-4
RES_TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a, dt=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda")


def _residual(X, Xt, om_r, om_c, Lr, Lc, gr, gc):
    """|D_r X D_c + gc X Lc + gr Lr X - M_r^T Xt M_c^T|_F / |B|_F in FP64."""
    X = np.asarray(X, dtype=np.float64)
    p, n = X.shape
    mr = np.zeros(p, bool)
    mr[om_r] = True
    mc = np.zeros(n, bool)
    mc[om_c] = True
    B = np.zeros((p, n))
    B[np.ix_(om_r, om_c)] = Xt
    AX = np.where(np.outer(mr, mc), X, 0.0) + gc * np.asarray(sp.csr_matrix(Lc).T @ X.T).T \
        + gr * np.asarray(sp.csr_matrix(Lr) @ X)
    return float(np.linalg.norm(AX - B) / np.linalg.norm(B))


def _instance(seed, p, n, rr, rc, K=10):
    Y, _, _ = gen.make_instance(seed, p, n, 5, 4, 0.05)
    Lr, *_ = O.knn_graph(Y, K)
    Lc, *_ = O.knn_graph(Y.T, K)
    om_r = O.sample_indices(seed, p, rr, 0)
    om_c = O.sample_indices(seed, n, rc, 1)
    Xt = Y[np.ix_(om_r, om_c)]
    return Y, Lr, Lc, om_r, om_c, Xt


@pytest.mark.parametrize("p,n,rr,rc,gr,gc", [(200, 300, 100, 150, 1.0, 1.0), (96, 301, 40, 77, 0.5, 2.0),
                                            (256, 512, 128, 256, 1.0, 1.0)])
def test_alternate_decoder_matches_oracle(M, p, n, rr, rc, gr, gc):
    Y, Lr, Lc, om_r, om_c, Xt = _instance(3, p, n, rr, rc)
    X, info, _ = M.cpca_alternate_decode(_dev(Xt), _dev(om_r, np.int32), _dev(om_c, np.int32), p, n,
                                         M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                         M.alt_params(gamma_r=gr, gamma_c=gc, tol=1e-6, max_iter=5000))
    assert info.converged and info.rel_res <= 1e-6
    Xo = D.alternate_decode(Xt, om_r, om_c, p, n, Lr, Lc, gr, gc, tol=1e-12)
    Xg = X.cpu().numpy()
    assert rel_fro(Xg, Xo) < DECODE_TOL
    assert _residual(Xg, Xt, om_r, om_c, Lr, Lc, gr, gc) < RES_TOL


def test_full_sampling_without_regularisation_returns_the_samples(M):
    """A = I: one iteration with alpha = 1 exactly, X = Xt bit for bit."""
    p, n = 70, 45
    rng = np.random.default_rng(1)
    Y, Lr, Lc, _, _, _ = _instance(5, p, n, p, n)
    Xt = rng.standard_normal((p, n)).astype(np.float32)
    X, info, _ = M.cpca_alternate_decode(_dev(Xt), _dev(np.arange(p), np.int32), _dev(np.arange(n), np.int32),
                                         p, n, M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc),
                                         M.alt_params(gamma_r=0.0, gamma_c=0.0))
    assert info.iters == 1
    assert np.array_equal(X.cpu().numpy(), Xt)


def test_repeated_sample_index_is_rejected(M):
    p, n = 64, 40
    Y, Lr, Lc, om_r, om_c, Xt = _instance(2, p, n, 20, 10)
    bad = om_r.copy()
    bad[3] = bad[2]
    with pytest.raises(M.CpcaError) as e:
        M.cpca_alternate_decode(_dev(Xt), _dev(bad, np.int32), _dev(om_c, np.int32), p, n,
                                M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc))
    assert e.value.status == M.CPCA_ERR_INVALID_ARG


def test_alternate_decoder_full_size_residual(M):
    """10304 x 1000 (rank 10, 10 clusters, 1/4 x 1/4 sampling), graphs from
    the CUDA kNN: the FP64 residual of the returned X, from the definition."""
    cfg = gen.CONFIGS["bench_10304x1000"]
    p, n = cfg["p"], cfg["n"]
    Yd = gen.make_instance_torch(0, p, n, cfg["r"], cfg["C"], cfg["frac"], device="cuda")
    Lr, _, _ = M.cpca_knn_graph(Yd, cfg["K"])
    Lc, _, _ = M.cpca_knn_graph(Yd, cfg["K"], transposed=True)
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    om_r, om_c, Yt = M.cpca_sample(0, p, n, rr, rc, Yd)
    X, info, _ = M.cpca_alternate_decode(Yt, om_r, om_c, p, n, Lr, Lc,
                                         M.alt_params(gamma_r=1.0, gamma_c=1.0, tol=1e-6, max_iter=20000))
    assert info.converged
    sc = lambda L: sp.csr_matrix((L.val.cpu().numpy().astype(np.float64), L.col.cpu().numpy(),
                                  L.rowptr.cpu().numpy()), shape=(L.n, L.n))
    res = _residual(X.cpu().numpy(), Yt.cpu().numpy(), om_r.cpu().numpy(), om_c.cpu().numpy(), sc(Lr), sc(Lc),
                    1.0, 1.0)
    assert res < RES_TOL
