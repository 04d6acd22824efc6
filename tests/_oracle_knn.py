"""The oracle's kNN graph at sizes where the numpy search is too slow.

No method arithmetic here: the search is the oracle's C restatement of the
exact kNN definition (oracle/knn_c.c, pinned against oracle.knn_bruteforce)
run on every host core, and the graph is oracle.laplacian_from_knn on its
lists, exactly as oracle.knn_graph composes them.
"""
import numpy as np

import oracle as O
from oracle.cpca_fista_c import knn_c


def oracle_knn_graph(P, K, lap_type=O.LAP_NORMALIZED):
    """(L, W, idx [N, K+1], d2 [N, K+1]) for the rows of P (FP32 values):
    the K + 1 nearest are kept so that callers can tell near ties at the
    K-th place; the graph uses the first K."""
    P32 = np.ascontiguousarray(P, dtype=np.float32)
    if not np.array_equal(P32, P):
        raise ValueError("oracle_knn_graph takes FP32-representable points")
    idx, d2 = knn_c(P32, K + 1)
    L, W = O.laplacian_from_knn(idx[:, :K], d2[:, :K], P32.shape[0], O.sigma2_mean(d2[:, :K]), lap_type)
    return L, W, idx, d2
