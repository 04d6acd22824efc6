"""Clustering decoder (Sec. V-D, Algorithm 3) through the C ABI against the
FP64 oracle.

Bars (written here): the k-means labels of X~'s columns are bit-exact (both
sides take the same Lloyd path from the same seeded centres; the data are
clustered, so no assignment is near a tie); the decoded labels are equal
wherever the oracle's two largest row entries differ by more than 1e-4
(the PCG stops at relative residual 1e-6; a closer margin may flip in FP32),
and elsewhere the GPU's label is one of the tied candidates.
"""
import numpy as np
import pytest

import gen
import oracle as O
from oracle import cpca_decoders as D
from tests._oracle_knn import oracle_knn_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-4


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a, dt=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda")


def _check_labels(lab_g, C_o):
    top2 = np.sort(C_o, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > MARGIN
    lab_o = np.argmax(C_o, axis=1)
    assert np.array_equal(lab_g[clear], lab_o[clear])
    for i in np.flatnonzero(~clear):
        assert C_o[i, lab_g[i]] >= top2[i, 1] - MARGIN


@pytest.mark.parametrize("p,n,C,rr,rc,frac", [(256, 512, 4, 128, 256, 0.0), (300, 450, 6, 100, 150, 0.02)])
def test_cluster_decoder_matches_oracle(M, p, n, C, rr, rc, frac):
    Y, _, _ = gen.make_instance(6, p, n, 5, C, frac)
    Lc, *_ = O.knn_graph(Y.T, 10)
    om_r = O.sample_indices(6, p, rr, 0)
    om_c = O.sample_indices(6, n, rc, 1)
    Xt = Y[np.ix_(om_r, om_c)]
    out = M.cpca_cluster_decode(_dev(Xt), _dev(om_c, np.int32), n, M.Csr.from_scipy(Lc), C, seed=3)
    lab_o, C_o, labt_o = D.cluster_decode(Xt, om_c, n, Lc, C, seed=3, tol=1e-10)
    assert np.array_equal(out["labels_t"].cpu().numpy(), labt_o)
    _check_labels(out["labels"].cpu().numpy(), C_o)


def test_cluster_decoder_full_size(M):
    """10304 x 1000 (10 clusters of columns), X~ 2576 x 250, k = 10: the
    oracle's column graph (1000 nodes) and sampled matrix feed both sides."""
    cfg = gen.CONFIGS["bench_10304x1000"]
    p, n = cfg["p"], cfg["n"]
    Y, _, _ = gen.make_instance(0, p, n, cfg["r"], cfg["C"], cfg["frac"])
    Lc, _, _, _ = oracle_knn_graph(Y.T, cfg["K"])
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    om_r, om_c = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    Xt = O.sample_matrix(Y.astype(np.float64), om_r, om_c)
    out = M.cpca_cluster_decode(_dev(Xt), _dev(om_c, np.int32), n, M.Csr.from_scipy(Lc), cfg["C"], seed=1)
    lab_o, C_o, labt_o = D.cluster_decode(Xt, om_c, n, Lc, cfg["C"], seed=1, tol=1e-10)
    assert np.array_equal(out["labels_t"].cpu().numpy(), labt_o)
    _check_labels(out["labels"].cpu().numpy(), C_o)
