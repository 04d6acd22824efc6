"""The allocation-free FISTA entry point (for callers that cannot allocate
device memory, e.g. a plugin whose host owns the whole memory pool): through
the C ABI, two calls in a row, each equal to cpca_frpcag_solve with a
caller workspace. Kept in a file collected last."""
import ctypes as C

import numpy as np
import pytest

import gen
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4  # the FISTA parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


def _problem(M, seed, rr, rc):
    Y, _, _ = gen.make_instance(seed, rr, rc, 4, 3, 0.05)
    Yt = Y.astype(np.float64)
    Lr, *_ = O.knn_graph(Yt, 8)
    Lc, *_ = O.knn_graph(Yt.T, 8)
    return (torch.as_tensor(Y, device="cuda"), M.Csr.from_scipy(Lr), M.Csr.from_scipy(Lc))


def test_noalloc_matches_workspace_solve_twice(M):
    L = M.lib()
    for seed, (rr, rc) in ((1, (300, 130)), (2, (257, 77))):
        Yt, Lr, Lc = _problem(M, seed, rr, rc)
        prm = M.frpcag_params(gamma_r=0.8, gamma_c=1.7, max_iter=150)
        ref, rinfo = M.cpca_frpcag_solve(Yt, Lr, Lc, prm)
        X = torch.full((rr, rc), float("nan"), device="cuda")
        info = M.capi.cpca_solve_info()
        lr, lc = Lr.c(), Lc.c()
        st = L.cpca_frpcag_solve_noalloc(C.c_void_p(Yt.data_ptr()), rr, rc, Yt.stride(0),
                                         C.byref(lr), C.byref(lc), C.byref(prm),
                                         C.c_void_p(X.data_ptr()), X.stride(0), C.byref(info),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == M.CPCA_OK, L.cpca_last_error()
        err = float(torch.linalg.norm(X - ref) / torch.linalg.norm(ref))
        assert err <= TOL
        assert info.iters == rinfo.iters == 150
        assert info.step == pytest.approx(rinfo.step, rel=1e-6)


def test_noalloc_rejects_oversized_problem(M):
    L = M.lib()
    rr, rc = 4096, 1024  # needs more scratch than the built-in array
    dummy = C.c_void_p(16)
    lr = M.capi.cpca_csr(rr, 0, 16, None, None)
    lc = M.capi.cpca_csr(rc, 0, 16, None, None)
    prm = M.frpcag_params(max_iter=1)
    st = L.cpca_frpcag_solve_noalloc(dummy, rr, rc, rc, C.byref(lr), C.byref(lc), C.byref(prm),
                                     dummy, rc, None, None)
    assert st == M.CPCA_ERR_WORKSPACE
    assert b"scratch" in L.cpca_last_error()
