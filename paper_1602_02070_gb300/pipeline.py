"""End-to-end compressive PCA (Table "tab:cpca", steps 1-6) through the C ABI.

Sequencing and buffer marshalling only; each step is one libcpca call.
"""
from __future__ import annotations

import math

import torch

from . import capi


def rho_of(N: int, frac: float) -> int:
    """Number of sampled rows/columns: floor(N * frac + 1/2), at least 1."""
    return max(1, int(math.floor(N * frac + 0.5)))


def cpca_pipeline(Y: torch.Tensor, K: int = 10, fr: float = 0.25, fc: float = 0.25, seed: int = 0,
                  J: int = 300, gamma_r: float = 1.0, gamma_c: float = 1.0,
                  lap_type: int = capi.LAP_NORMALIZED, cg_tol: float = 1e-6,
                  power_iters: int = 200, power_seed: int = 0, rank_ratio: float = 0.1,
                  delta: float = 0.0, kmax: int = 24, svd_iters: int = 6, marks=None,
                  want_X: bool = True, check_status: bool = True, graphs: str = "knn",
                  kron_tol: float = 1e-6, out: torch.Tensor | None = None):
    """Steps 1-6 on a dense device matrix Y (p x n, FP32, row-major).

    1. kNN graphs L_r (rows of Y) and L_c (columns of Y);
    2-3. sampling Omega_r, Omega_c and Y~ = M_r Y M_c;
    4. graphs of Y~'s rows and columns: new kNN graphs (``graphs="knn"``,
       the experiments' choice) or the Kron reductions of L_r and L_c onto
       Omega_r and Omega_c (``graphs="kron"``, Sec. IV-A; dense);
    5. FRPCAG by FISTA on Y~ (J iterations, lambda by power iteration);
    6. approximate decoder (Algorithm 2) to X (p x n).
    ``marks``: optional callable(name) invoked between steps (timing hooks).
    ``out``: optional p x n float32 output - a device tensor, or a pinned
    host tensor that the decoder's output kernel writes directly over the
    CPU-GPU link (no device copy of X and no separate transfer).
    """
    if graphs not in ("knn", "kron"):
        raise ValueError("graphs must be 'knn' or 'kron'")
    mark = marks or (lambda name: None)
    p, n = Y.shape
    rr, rc = rho_of(p, fr), rho_of(n, fc)
    mark("start")
    cert = {}  # per graph: (queries brute-forced, queries left uncertified)

    def knn(pts, name, transposed):
        G, _, _ = capi.cpca_knn_graph(pts, K, lap_type, transposed=transposed)
        cert[name] = (capi.knn_last_bruteforce(), capi.knn_last_uncertified())
        return G

    Lr = knn(Y, "Lr", False)
    Lc = knn(Y, "Lc", True)
    mark("graphs")
    om_r, om_c, Yt = capi.cpca_sample(seed, p, n, rr, rc, Y)
    if graphs == "knn":
        Lrt = knn(Yt, "Lrt", False)
        Lct = knn(Yt, "Lct", True)
    else:
        Lrt = capi.cpca_kron_reduce(Lr, om_r, tol=kron_tol)["csr"]
        Lct = capi.cpca_kron_reduce(Lc, om_c, tol=kron_tol)["csr"]
    mark("sample")
    prm = capi.frpcag_params(gamma_r, gamma_c, -1.0, J, 0.0, power_iters, power_seed)
    fws = capi._workspace(capi.lib().cpca_frpcag_workspace_size(*Yt.shape), Y.device)
    Xt, finfo = capi.cpca_frpcag_solve(Yt, Lrt, Lct, prm, want_info=False, ws=fws)
    mark("fista")
    dprm = capi.decode_params(rank_ratio, 0, kmax, delta, cg_tol, 0, svd_iters, 0)
    dec = capi.cpca_decode(Xt, om_r, om_c, p, n, Lr, Lc, dprm, want_X=want_X, out=out,
                           check_status=check_status)
    # the info-less FISTA solve reports a barrier timeout through its
    # workspace (the decoder has synchronised the stream already)
    if check_status:
        capi.cpca_frpcag_status(fws)
    mark("decode")
    dec.update({"Xt": Xt, "Yt": Yt, "omega_r": om_r, "omega_c": om_c, "Lr": Lr, "Lc": Lc,
                "Lrt": Lrt, "Lct": Lct, "knn_certification": cert})
    return dec
