"""ctypes loader for the oracle's C part: oracle/fista_c.c (Algorithm 1)
and oracle/knn_c.c (the exact kNN search of Sec. I).

TEST INFRASTRUCTURE ONLY (see the package docstring). ``build()`` compiles
liboracle.so next to this file with gcc (FP64, no floating-point
contraction, OpenMP). ``frpcag_fista_c`` has the signature and return value
of :func:`oracle.frpcag_fista`, ``knn_c`` those of
:func:`oracle.knn_bruteforce`; both are pinned against the numpy functions
in ``tests/test_oracle_fista_c.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "fista_c.c"), os.path.join(HERE, "knn_c.c")]
LIB = os.path.join(HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp, IEEE FP64: no contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, SRCS)):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", *SRCS, "-o", LIB, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle C build failed:\n" + r.stdout + r.stderr)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        f = L.oracle_frpcag_fista
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                      C.c_int, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        g = L.oracle_knn
        g.restype = C.c_int
        g.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                      C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def _csr(L):
    L = sp.csr_matrix(L)
    return (np.ascontiguousarray(L.indptr, dtype=np.int64), np.ascontiguousarray(L.indices, dtype=np.int32),
            np.ascontiguousarray(L.data, dtype=np.float64))


def frpcag_fista_c(Yt, Lr, Lc, gamma_r: float, gamma_c: float, lam: float, J: int, eps: float = 0.0,
                   threads: int = 0):
    """Algorithm 1 as :func:`oracle.frpcag_fista`, in C on ``threads`` OpenMP
    threads (0: all). Returns (S, {"iters", "rel_change"})."""
    Y = np.ascontiguousarray(Yt, dtype=np.float64)
    rr, rc = Y.shape
    r, c = _csr(Lr), _csr(Lc)
    S = np.empty_like(Y)
    it = C.c_int(0)
    rel = C.c_double(0.0)
    p = lambda a: a.ctypes.data  # noqa: E731
    st = _load().oracle_frpcag_fista(rr, rc, p(Y), p(r[0]), p(r[1]), p(r[2]), p(c[0]), p(c[1]), p(c[2]),
                                     float(gamma_r), float(gamma_c), float(lam), int(J), float(eps),
                                     int(threads), p(S), C.byref(it), C.byref(rel))
    if st != 0:
        raise MemoryError("oracle_frpcag_fista: out of host memory")
    return S, {"iters": int(it.value), "rel_change": float(rel.value)}


def knn_c(P, K: int, queries=None, threads: int = 0):
    """The K nearest neighbours of the query rows of P (float32 points,
    row-major) as :func:`oracle.knn_bruteforce`: FP64 direct sums, the point
    itself excluded, ties by (d^2, j). Returns (idx int64 [Q, K], d2 float64
    [Q, K])."""
    P = np.asarray(P)
    if P.dtype != np.float32:
        raise TypeError("knn_c takes float32 points (converted to FP64 per coordinate)")
    if P.ndim != 2 or P.strides[1] != 4:
        P = np.ascontiguousarray(P)
    N, d = P.shape
    ld = P.strides[0] // 4
    qs = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = N if qs is None else len(qs)
    idx = np.empty((nq, K), dtype=np.int64)
    d2 = np.empty((nq, K))
    st = _load().oracle_knn(P.ctypes.data, N, d, ld, int(K), None if qs is None else qs.ctypes.data, nq,
                            int(threads), idx.ctypes.data, d2.ctypes.data)
    if st != 0:
        raise ValueError("oracle_knn: bad K or query index")
    return idx, d2
