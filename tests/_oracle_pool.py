"""Runs the oracle's per-query kNN search in a spawn-started process pool.

The point set is written once to a .npy file that every worker maps
read-only, so it is not pickled per task. No method arithmetic here: each
task is one call of the oracle's own search.
"""
import multiprocessing as mp
import os
import tempfile

import numpy as np

import oracle as O

_cache = {}


def _load(path):
    P = _cache.get(path)
    if P is None:
        _cache.clear()
        P = _cache[path] = np.load(path, mmap_mode="r")
    return P


def _bruteforce_task(args):
    path, K, qs = args
    return O.knn_bruteforce(_load(path), K, queries=qs)


class OraclePool:
    def __init__(self, procs=None):
        self.procs = procs or max(2, min(16, os.cpu_count() or 2))
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.dir = tempfile.mkdtemp(prefix="oracle_pool_")
        self.seq = 0

    def knn(self, P, K, queries=None):
        """knn_bruteforce(P, K, queries) split over the pool."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        self.seq += 1
        path = os.path.join(self.dir, f"P{self.seq}.npy")
        np.save(path, P)
        qs = np.arange(P.shape[0]) if queries is None else np.asarray(queries)
        parts = self.pool.map(_bruteforce_task,
                              [(path, K, c) for c in np.array_split(qs, 4 * self.procs) if len(c)])
        os.remove(path)
        return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))

    def knn_graph(self, P, K):
        """The oracle's knn_graph (normalised Laplacian, mean sigma^2) with
        the search done in the pool. The search keeps K + 1 neighbours so
        that callers can tell near ties at the K-th place; the graph uses
        the first K. Returns (L, W, idx [N, K+1], d2 [N, K+1])."""
        idx, d2 = self.knn(P, K + 1)
        L, W = O.laplacian_from_knn(idx[:, :K], d2[:, :K], P.shape[0], O.sigma2_mean(d2[:, :K]))
        return L, W, idx, d2

    def close(self):
        self.pool.close()
        self.pool.join()
        os.rmdir(self.dir)
