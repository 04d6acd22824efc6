"""Helpers shared by the parity tests (no method arithmetic here)."""
import re
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def header_functions():
    """Names of the functions declared in include/cpca.h."""
    txt = open(os.path.join(ROOT, "include", "cpca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cpca_[a-z0-9_]+)\s*\(", txt)))


def knn_sets_match(gi, gd, oi, od_full_sorted, K, rel_gap=1e-6):
    """Neighbour sets equal except where the K-th and (K+1)-th exact
    distances are within rel_gap (relative): then only the strictly closer
    neighbours must agree. Returns the list of mismatching queries."""
    bad = []
    for q in range(len(gi)):
        g, o = set(gi[q].tolist()), set(oi[q].tolist())
        if g == o:
            continue
        dk, dk1 = od_full_sorted[q][K - 1], od_full_sorted[q][K]
        if abs(dk1 - dk) < rel_gap * max(dk, 1e-300):
            continue
        bad.append(q)
    return bad
