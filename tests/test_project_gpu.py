"""Approximate decoders 2 and 3 (appendix, "Other Approximate Decoders"):
the CUDA decoder's upsampled basis and the projection X = U U^T Y or
X = Y V V^T through the C ABI, against the FP64 oracle.

Tolerances (written here): the decoded X within 1e-4 relative Frobenius
error of the oracle's (the benchmark spec's bound for decoded matrices; both
sides run PCG to 1e-6); the projection alone, given the same basis, within
1e-5 of its FP64 value (FP32 sums over p or n terms).
"""
import numpy as np
import pytest

import gen
import oracle as O
from oracle import cpca_decoders as D
from tests._util import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _dev(a, dt=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda")


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("p,n,rr,rc", [(200, 300, 100, 150), (130, 77, 65, 40)])
def test_projected_decoder_matches_oracle(M, side, p, n, rr, rc):
    Y, _, _ = gen.make_instance(4, p, n, 5, 4, 0.05)
    Lr, *_ = O.knn_graph(Y, 10)
    Lc, *_ = O.knn_graph(Y.T, 10)
    om_r = O.sample_indices(4, p, rr, 0)
    om_c = O.sample_indices(4, n, rc, 1)
    Xt = Y[np.ix_(om_r, om_c)]
    dec = M.cpca_decode(_dev(Xt), _dev(om_r, np.int32), _dev(om_c, np.int32), p, n, M.Csr.from_scipy(Lr),
                        M.Csr.from_scipy(Lc), M.decode_params(), want_X=False)
    k = dec["k"]
    basis = dec["U"] if side == 0 else dec["V"]
    X = M.cpca_subspace_project(side, basis, k, _dev(Y)).cpu().numpy()
    Xo, Bo, ko = D.approx_decode_projected(Y, Xt, om_r, om_c, Lr, Lc, side, k_override=k)
    assert rel_fro(X, Xo) < 1e-4


@pytest.mark.parametrize("side", [0, 1])
def test_projection_full_size_against_fp64(M, side):
    """10304 x 1000: the projection kernels given a basis, against FP64."""
    cfg = gen.CONFIGS["bench_10304x1000"]
    p, n = cfg["p"], cfg["n"]
    Yd = gen.make_instance_torch(0, p, n, cfg["r"], cfg["C"], cfg["frac"], device="cuda")
    rng = np.random.default_rng(side)
    k, ldb = 9, 24
    B = rng.standard_normal(((p if side == 0 else n), ldb)).astype(np.float32)
    B[:, :k] /= np.linalg.norm(B[:, :k], axis=0)
    X = M.cpca_subspace_project(side, _dev(B), k, Yd).cpu().numpy()
    Y = Yd.cpu().numpy().astype(np.float64)
    Bk = B[:, :k].astype(np.float64)
    Xo = Bk @ (Bk.T @ Y) if side == 0 else (Y @ Bk) @ Bk.T
    assert rel_fro(X, Xo) < 1e-5


def test_projection_rank_zero_gives_zeros(M):
    Y = torch.randn(40, 30, device="cuda")
    X = M.cpca_subspace_project(0, torch.ones(40, 4, device="cuda"), 0, Y)
    assert torch.count_nonzero(X).item() == 0
