"""The C ABI library loads and exports every function include/cpca.h
declares; argument errors are reported on the host (no GPU needed)."""
import ctypes as C

import pytest

from tests._util import header_functions


@pytest.fixture(scope="module")
def capi():
    from paper_1602_02070_gb300 import capi as m
    m.lib()
    return m


def test_exports_every_declared_function(capi):
    L = capi.lib()
    declared = header_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(L, name), name
    assert set(capi.exported_names()) <= set(declared)
    assert set(declared) <= set(capi.exported_names())


def test_version_and_counter(capi):
    assert capi.lib().cpca_version() >= 100
    assert capi.lib().cpca_launch_count() >= 0


def test_invalid_arguments_rejected_on_host(capi):
    L = capi.lib()
    om = C.c_void_p(16)
    st = L.cpca_sample(0, 10, 10, 11, 5, None, 0, om, om, None, 0, None)
    assert st == capi.CPCA_ERR_INVALID_ARG
    assert b"rho" in L.cpca_last_error()
    st = L.cpca_knn_graph(C.c_void_p(16), 100, 8, 8, 0, 40, 0, -1.0, om, om, om, None, 100000,
                          None, None, None, None, None, 0, None)
    assert st == capi.CPCA_ERR_INVALID_ARG and b"K" in L.cpca_last_error()
    prm = capi.frpcag_params(max_iter=-1)
    lr = capi.cpca_csr(4, 4, 16, 16, 16)
    st = L.cpca_frpcag_solve(C.c_void_p(16), 4, 4, 4, C.byref(lr), C.byref(lr), C.byref(prm),
                             C.c_void_p(16), 4, None, C.c_void_p(16), 1 << 20, None)
    assert st == capi.CPCA_ERR_INVALID_ARG
    dprm = capi.decode_params(kmax=64)
    st = L.cpca_decode(C.c_void_p(16), 2, 2, 2, om, om, 4, 4, C.byref(lr), C.byref(lr),
                       C.byref(dprm), None, 4, None, None, None, None, None, C.c_void_p(16), 1 << 20, None)
    assert st == capi.CPCA_ERR_INVALID_ARG and b"kmax" in L.cpca_last_error()


def test_workspace_queries_are_host_only(capi):
    L = capi.lib()
    assert L.cpca_frpcag_workspace_size(2576, 250) >= 2 * 2576 * 250 * 4
    assert L.cpca_decode_workspace_size(10304, 1000, 2576, 250, 32, 170000, 17000) > 0
    assert L.cpca_decode_workspace_size(10, 10, 5, 5, 64, 30, 30) == 0


def test_kron_reduce_arguments_checked_on_host(capi):
    L = capi.lib()
    lap = capi.cpca_csr(10, 30, 16, 16, 16)
    p = C.c_void_p(16)
    st = L.cpca_kron_reduce(C.byref(lap), p, 11, 1e-6, 0, p, 11, None, None, None, None, p, 1 << 20, None)
    assert st == capi.CPCA_ERR_INVALID_ARG and b"rho" in L.cpca_last_error()
    st = L.cpca_kron_reduce(C.byref(lap), p, 4, 1e-6, 0, p, 4, p, None, None, None, p, 1 << 20, None)
    assert st == capi.CPCA_ERR_INVALID_ARG and b"together" in L.cpca_last_error()
    st = L.cpca_kron_reduce(C.byref(lap), p, 4, 1e-6, 0, p, 3, None, None, None, None, p, 1 << 20, None)
    assert st == capi.CPCA_ERR_INVALID_ARG
    st = L.cpca_kron_reduce(C.byref(lap), p, 4, 1e-6, 0, p, 4, None, None, None, None, p, 16, None)
    assert st == capi.CPCA_ERR_WORKSPACE
    assert L.cpca_kron_reduce_workspace_size(10304, 2576, 180000) > 0
    assert L.cpca_kron_reduce_workspace_size(10, 11, 30) == 0


def test_binding_argument_counts_match_header(capi):
    """Every ctypes signature in the binding has as many arguments as the
    declaration in include/cpca.h (an ABI drift check, no GPU needed)."""
    import os
    import re
    from tests._util import ROOT
    txt = open(os.path.join(ROOT, "include", "cpca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    decl = {}
    for m in re.finditer(r"\b(cpca_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
        args = m.group(2).strip()
        decl[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    sigs = {name: len(args) for name, _, args in capi._SIGS}
    assert set(sigs) == set(decl)
    for name, n in sigs.items():
        assert decl[name] == n, (name, decl[name], n)


def test_pipeline_rejects_unknown_graph_kind_before_any_launch(capi):
    import paper_1602_02070_gb300 as M
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        M.cpca_pipeline(torch.zeros(8, 8), graphs="dense")
