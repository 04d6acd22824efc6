"""Failure paths, exercised without any GPU fault.

A grid-barrier wait that runs out (poll limit 1, set through the library's
test hook or CPCA_FAULT=timeout) makes every block leave its loops; the call
reports CPCA_ERR_TIMEOUT and the context stays usable: the same solve then
gives its normal result. CPCA_FAULT=nan makes a solve with info report
CPCA_ERR_NONFINITE. CPCA_FAULT=alloc fails the binding's workspace
allocation before any launch (a CPU test).
"""
import os

import numpy as np
import pytest

import gen
import oracle as O

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_02070_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def problem(M):
    Y, _, _ = gen.make_instance(0, 256, 512, 5, 4, 0.05)
    Yt = Y.astype(np.float64)[np.ix_(O.sample_indices(0, 256, 128, 0), O.sample_indices(0, 512, 256, 1))]
    Lr, *_ = O.knn_graph(Yt, 10)
    Lc, *_ = O.knn_graph(Yt.T, 10)
    return (torch.as_tensor(Yt.astype(np.float32), device="cuda"), M.Csr.from_scipy(Lr),
            M.Csr.from_scipy(Lc))


@pytest.mark.gpu
def test_barrier_timeout_is_reported_and_recovered(M, problem):
    Yt, Lr, Lc = problem
    X0, _ = M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=200)
    ws = torch.empty(M.lib().cpca_frpcag_workspace_size(*Yt.shape), dtype=torch.uint8, device="cuda")
    M.debug_set_barrier_spin_limit(1)
    try:
        with pytest.raises(M.CpcaError) as e:
            M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=200, ws=ws)
        assert e.value.status == M.CPCA_ERR_TIMEOUT
        # without info the call is asynchronous; the flag waits in ws
        M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=200, want_info=False, ws=ws)
        with pytest.raises(M.CpcaError) as e:
            M.cpca_frpcag_status(ws)
        assert e.value.status == M.CPCA_ERR_TIMEOUT
    finally:
        M.debug_set_barrier_spin_limit(0)
    X1, info = M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=200, ws=ws)
    M.cpca_frpcag_status(ws)
    assert info.iters == 200 and torch.equal(X0, X1)


@pytest.mark.gpu
def test_fault_env_timeout_and_nan(M, problem, monkeypatch):
    Yt, Lr, Lc = problem
    monkeypatch.setenv("CPCA_FAULT", "timeout")
    with pytest.raises(M.CpcaError) as e:
        M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=100)
    assert e.value.status == M.CPCA_ERR_TIMEOUT
    monkeypatch.setenv("CPCA_FAULT", "nan")
    with pytest.raises(M.CpcaError) as e:
        M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=100)
    assert e.value.status == M.CPCA_ERR_NONFINITE
    monkeypatch.delenv("CPCA_FAULT")
    _, info = M.cpca_frpcag_solve(Yt, Lr, Lc, max_iter=100)
    assert np.isfinite(info.objective)


@pytest.mark.gpu
def test_decoder_barrier_timeout(M):
    Y, _, _ = gen.make_instance(1, 200, 300, 4, 3, 0.05)
    p, n = Y.shape
    om_r, om_c = O.sample_indices(0, p, 100, 0), O.sample_indices(0, n, 150, 1)
    Lr, *_ = O.knn_graph(Y.astype(np.float64), 8)
    Lc, *_ = O.knn_graph(Y.T.astype(np.float64), 8)
    Xt = torch.as_tensor(Y[np.ix_(om_r, om_c)], device="cuda")
    args = (Xt, torch.as_tensor(om_r, dtype=torch.int32, device="cuda"),
            torch.as_tensor(om_c, dtype=torch.int32, device="cuda"), p, n, M.Csr.from_scipy(Lr),
            M.Csr.from_scipy(Lc))
    ref = M.cpca_decode(*args)
    M.debug_set_barrier_spin_limit(1)
    try:
        with pytest.raises(M.CpcaError) as e:
            M.cpca_decode(*args)
        assert e.value.status == M.CPCA_ERR_TIMEOUT
    finally:
        M.debug_set_barrier_spin_limit(0)
    again = M.cpca_decode(*args)
    assert again["k"] == ref["k"] and torch.equal(again["X"], ref["X"])


def test_fault_env_alloc_fails_before_any_launch(monkeypatch):
    """Host only: the binding's workspace allocation fails as an
    out-of-memory would, with CPCA_ERR_WORKSPACE, before anything runs."""
    from paper_1602_02070_gb300 import capi
    monkeypatch.setenv("CPCA_FAULT", "alloc")
    with pytest.raises(capi.CpcaError) as e:
        capi._workspace(1 << 20, "cpu")
    assert e.value.status == capi.CPCA_ERR_WORKSPACE
    monkeypatch.delenv("CPCA_FAULT")
    assert capi._workspace(1 << 10, "cpu").numel() == 1 << 10
