"""Plain FP64 restatement of the CPCA hot path (test infrastructure only).

Steps, in the order of the complete CPCA algorithm (Table "tab:cpca"):
  1. kNN graphs and Laplacians between rows and columns (Sec. I, graph
     construction paragraph; Sec. VII-A "Graph Construction").
  2-3. Uniform row/column sampling without replacement, Y~ = M_r Y M_c
     (Sec. III, Eq. Mc).
  4. Graphs of the sampled matrix by kNN on Y~ (Sec. VII-A, "can also be
     constructed using FLANN").
  5. FRPCAG on Y~ by FISTA (Sec. IV-B, Eq. frpcag_small, Algorithm 1).
  6. Approximate decoder by subspace upsampling (Sec. V-C, Lemma 1,
     Eq. Uupsample, Algorithm 2).

Readings where the paper is silent or garbled are stated in each docstring.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "splitmix64_outputs", "uniform01", "sample_indices", "sample_matrix",
    "knn_bruteforce", "knn_query_blocked", "sigma2_mean", "laplacian_from_knn", "laplacian_from_weights",
    "knn_graph",
    "power_norm", "fista_step", "frpcag_fista", "frpcag_objective",
    "svd_rank", "pcg", "upsample_subspace", "approx_decode", "cpca",
    "LAP_NORMALIZED", "LAP_COMBINATORIAL", "GOLDEN_GAMMA",
]

LAP_NORMALIZED = 0
LAP_COMBINATORIAL = 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64, Steele, Lea & Flood, OOPSLA 2014)
# ---------------------------------------------------------------------------
def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_outputs(seed: int, stream: int, count: int) -> list[int]:
    """Outputs 1..count of SplitMix64 started at
    state0 = seed XOR (GOLDEN_GAMMA * (stream + 1) mod 2^64).

    Output i is mix64(state0 + i * GOLDEN_GAMMA), i = 1..count (the state
    is advanced by the golden gamma before each output). Pure Python ints.
    """
    s0 = (seed ^ ((GOLDEN_GAMMA * (stream + 1)) & _M64)) & _M64
    return [_mix64((s0 + i * GOLDEN_GAMMA) & _M64) for i in range(1, count + 1)]


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Top 53 bits of each SplitMix64 output scaled to [0, 1)."""
    return np.array([(k >> 11) * 2.0 ** -53 for k in splitmix64_outputs(seed, stream, count)])


# ---------------------------------------------------------------------------
# Sampling (Sec. III, Eq. Mc)
# ---------------------------------------------------------------------------
def sample_indices(seed: int, N: int, rho: int, stream: int) -> np.ndarray:
    """Omega: rho indices of [0, N) drawn uniformly without replacement.

    Eq. Mc only asks for uniform sampling without replacement. Reading: each
    index i gets the key k_i = SplitMix64 output i+1 of ``stream`` (0 = rows,
    1 = columns); Omega is the rho indices with the smallest (k_i, i), returned
    in ascending index order. Keeping the rho smallest of N i.i.d. keys gives
    every rho-subset the same probability.
    """
    if not (0 <= rho <= N):
        raise ValueError("rho out of range")
    keys = splitmix64_outputs(seed, stream, N)
    order = sorted(range(N), key=lambda i: (keys[i], i))
    return np.array(sorted(order[:rho]), dtype=np.int64)


def sample_matrix(Y: np.ndarray, omega_r: np.ndarray, omega_c: np.ndarray) -> np.ndarray:
    """Y~ = M_r Y M_c with M_r, M_c of Eq. Mc: rows omega_r, columns omega_c.

    Sec. III writes Y~ in R^{rho_c x rho_r}; M_r Y M_c is rho_r x rho_c (as
    Sec. IV states), which is the shape used here.
    """
    p, n = Y.shape
    Mr = np.zeros((len(omega_r), p))
    Mr[np.arange(len(omega_r)), omega_r] = 1.0
    Mc = np.zeros((n, len(omega_c)))
    Mc[omega_c, np.arange(len(omega_c))] = 1.0
    return Mr @ np.asarray(Y, dtype=np.float64) @ Mc


# ---------------------------------------------------------------------------
# Graphs (Sec. I, graph construction; Sec. VII-A)
# ---------------------------------------------------------------------------
def knn_bruteforce(P: np.ndarray, K: int, queries=None):
    """Exact K nearest neighbours by Euclidean distance (Sec. I).

    Squared distances are summed directly as sum_t (y_it - y_jt)^2 over the
    coordinates, never through |a|^2 + |b|^2 - 2ab. The point itself is
    excluded. Ties (paper silent) are broken by (d^2, j) ascending.
    Returns (idx int64 [Q, K], d2 float64 [Q, K]) for the query rows.
    """
    P = np.asarray(P, dtype=np.float64)
    N = P.shape[0]
    if not (1 <= K < N):
        raise ValueError("need 1 <= K < N")
    qs = np.arange(N) if queries is None else np.asarray(queries)
    idx = np.empty((len(qs), K), dtype=np.int64)
    d2o = np.empty((len(qs), K))
    ar = np.arange(N)
    for t, i in enumerate(qs):
        diff = P - P[i]
        d2 = np.einsum("ij,ij->i", diff, diff)
        d2[i] = np.inf
        order = np.lexsort((ar, d2))[:K]
        idx[t] = order
        d2o[t] = d2[order]
    return idx, d2o


def knn_query_blocked(P, i: int, K: int, block: int = 256):
    """The K + 1 nearest neighbours of one point i (Sec. I), for point sets
    too large to difference in one piece: the candidates are visited in
    blocks of ``block`` points, each converted to FP64 and differenced
    coordinate by coordinate as in knn_bruteforce. Same exclusion of i and
    the same (d^2, j) tie order. Returns (idx int64 [K+1], d2 float64 [K+1]).
    """
    N = P.shape[0]
    if not (1 <= K < N - 1):
        raise ValueError("need 1 <= K < N - 1")
    q = np.asarray(P[i], dtype=np.float64)
    d2 = np.empty(N)
    for j0 in range(0, N, block):
        B = np.asarray(P[j0:j0 + block], dtype=np.float64)
        diff = B - q
        d2[j0:j0 + B.shape[0]] = np.einsum("ij,ij->i", diff, diff)
    d2[i] = np.inf
    order = np.lexsort((np.arange(N), d2))[:K + 1]
    return order.astype(np.int64), d2[order]


def sigma2_mean(d2: np.ndarray) -> float:
    """Gaussian kernel width: the mean of the N*K directed kNN squared
    distances. Sec. VII-A says "average distance of the K-nearest neighbors";
    the squared-distance mean is the reading used for sigma^2."""
    return float(np.mean(d2))


def laplacian_from_knn(idx: np.ndarray, d2: np.ndarray, N: int, sigma2: float,
                       lap_type: int = LAP_NORMALIZED):
    """Weights and Laplacian of Sec. I.

    W_ij = exp(-|y_i - y_j|^2 / sigma^2) if j is among the K nearest
    neighbours of i or vice versa, else 0 (no self loops); D_ii = sum_j W_ij;
    combinatorial L = D - W, normalised L_n = D^{-1/2} (D - W) D^{-1/2}.
    A node with D_ii = 0 uses D^{-1/2}_ii = 0 (its row and column of L_n
    vanish). Returns (L, W) as scipy CSR float64 matrices with sorted
    indices; L stores its diagonal explicitly.
    """
    edges = {}
    for i in range(idx.shape[0]):
        for k in range(idx.shape[1]):
            j = int(idx[i, k])
            a, b = (i, j) if i < j else (j, i)
            edges[(a, b)] = float(d2[i, k])
    rows, cols, vals = [], [], []
    for (a, b), dd in edges.items():
        w = math.exp(-dd / sigma2)
        rows += [a, b]
        cols += [b, a]
        vals += [w, w]
    W = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    W.sort_indices()
    return laplacian_from_weights(W, lap_type), W


def laplacian_from_weights(W, lap_type: int = LAP_NORMALIZED):
    """The Laplacian of Sec. I as a function of a symmetric weight matrix W
    (no self loops): combinatorial L = D - W or normalised
    L_n = D^{-1/2} (D - W) D^{-1/2}, D_ii = sum_j W_ij, with D^{-1/2}_ii = 0
    where D_ii = 0. Returns L as a scipy CSR float64 matrix with sorted
    indices and an explicit diagonal."""
    W = sp.csr_matrix(W)
    N = W.shape[0]
    deg = np.asarray(W.sum(axis=1)).ravel()
    if lap_type == LAP_COMBINATORIAL:
        L = sp.diags(deg) - W
    elif lap_type == LAP_NORMALIZED:
        # entrywise D^{-1/2} (D - W) D^{-1/2}: diagonal D_ii / D_ii = 1,
        # off-diagonal -W_ij / sqrt(D_ii D_jj) (the same value for ij and ji)
        Wc = W.tocoo()
        off = -Wc.data / np.sqrt(deg[Wc.row] * deg[Wc.col])
        L = sp.csr_matrix((off, (Wc.row, Wc.col)), shape=(N, N)) + sp.diags((deg > 0).astype(float))
    else:
        raise ValueError("lap_type")
    L = sp.csr_matrix(L)
    # keep the diagonal as an explicit entry even where it is zero
    L = L + sp.csr_matrix((np.full(N, 0.0), (np.arange(N), np.arange(N))), shape=(N, N))
    L = sp.csr_matrix(L)
    L.sort_indices()
    return L


def knn_graph(P: np.ndarray, K: int, lap_type: int = LAP_NORMALIZED, sigma2=None):
    """kNN -> sigma^2 -> symmetric Gaussian weights -> Laplacian (Sec. I).

    ``sigma2`` <= 0 or None selects the mean squared kNN distance.
    Returns (L, W, idx, d2, sigma2).
    """
    idx, d2 = knn_bruteforce(P, K)
    s2 = sigma2_mean(d2) if (sigma2 is None or sigma2 <= 0) else float(sigma2)
    L, W = laplacian_from_knn(idx, d2, P.shape[0], s2, lap_type)
    return L, W, idx, d2, s2


# ---------------------------------------------------------------------------
# Step size (Sec. IV-B: lambda = 1/beta', beta' = 2 g_c |L_c|_2 + 2 g_r |L_r|_2)
# ---------------------------------------------------------------------------
def power_norm(L, iters: int = 200, seed: int = 0, stream: int = 2) -> float:
    """Largest eigenvalue of a symmetric PSD matrix by power iteration.

    Start vector v0_i = u_i - 1/2 with u the SplitMix64 uniforms of
    (seed, stream). ``iters`` normalised products v <- L v / |L v|, then the
    Rayleigh quotient v^T L v / v^T v.
    """
    N = L.shape[0]
    v = uniform01(seed, stream, N) - 0.5
    v /= np.linalg.norm(v)
    for _ in range(iters):
        w = L @ v
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(v @ (L @ v) / (v @ v))


def fista_step(gamma_r: float, gamma_c: float, norm_r: float, norm_c: float) -> float:
    """lambda = 1/beta' with beta' = 2 gamma_c |L_c|_2 + 2 gamma_r |L_r|_2
    (Sec. IV-B). With beta' = 0 the smooth part vanishes and lambda = 1
    (any lambda gives the same iterates, which stay at Y~)."""
    beta = 2.0 * gamma_c * norm_c + 2.0 * gamma_r * norm_r
    return 1.0 / beta if beta > 0 else 1.0


# ---------------------------------------------------------------------------
# FRPCAG by FISTA (Sec. IV-B, Eq. frpcag_small, Algorithm 1)
# ---------------------------------------------------------------------------
def frpcag_objective(X, Yt, Lr, Lc, gamma_r, gamma_c) -> float:
    """phi(Y~ - X) + gamma_c tr(X L_c X^T) + gamma_r tr(X^T L_r X), phi = l1."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.abs(Yt - X).sum()
                 + gamma_c * np.sum((X @ Lc) * X)
                 + gamma_r * np.sum(X * (Lr @ X)))


def frpcag_fista(Yt, Lr, Lc, gamma_r: float, gamma_c: float, lam: float,
                 J: int, eps: float = 0.0):
    """Algorithm 1 for Eq. frpcag_small with phi = l1.

    Z_1 = S_0 = Y~, t_1 = 1; for j = 1..J:
      S_j = prox_{lam h}(Z_j - lam grad g(Z_j)),
        grad g(Z) = 2 (gamma_c Z L_c + gamma_r L_r Z),
        prox_{lam h}(V) = Y~ + sgn(V - Y~) max(|V - Y~| - lam, 0);
      t_{j+1} = (1 + sqrt(1 + 4 t_j^2)) / 2;
      Z_{j+1} = S_j + ((t_j - 1) / t_{j+1}) (S_j - S_{j-1});
      stop if |Z_{j+1} - Z_j|_F^2 < eps |Z_j|_F^2 (only when eps > 0).
    The algorithm's output line names an undefined "U_{j+1}"; reading: the
    output is the last prox output S_j. Returns (S, info dict).
    """
    Yt = np.asarray(Yt, dtype=np.float64)
    Z = Yt.copy()
    S_prev = Yt.copy()
    S = Yt.copy()
    t = 1.0
    rel = float("nan")
    it = 0
    for j in range(1, J + 1):
        G = 2.0 * (gamma_c * (Z @ Lc) + gamma_r * (Lr @ Z))
        V = Z - lam * G
        R = V - Yt
        S = Yt + np.sign(R) * np.maximum(np.abs(R) - lam, 0.0)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        Z_next = S + ((t - 1.0) / t_next) * (S - S_prev)
        dz = float(np.sum((Z_next - Z) ** 2))
        nz = float(np.sum(Z ** 2))
        rel = dz / nz if nz > 0 else 0.0
        it = j
        if eps > 0 and dz < eps * nz:
            break
        S_prev, Z, t = S, Z_next, t_next
    return S, {"iters": it, "rel_change": rel}


# ---------------------------------------------------------------------------
# Approximate decoder (Sec. V-C, Lemma 1, Eq. Uupsample, Algorithm 2)
# ---------------------------------------------------------------------------
def svd_rank(Xt, ratio: float = 0.1):
    """Step 1-2 of Algorithm 2: SVD of X~ and the rank k.

    Step 2 reads "find k such that S_kk/S_11 < 0.1" while Sec. V-C says k is
    the number of singular values above a threshold. Reading: k is the number
    of singular values with s_i / s_1 >= ratio. Returns (U~, s, V~ rows, k).
    """
    Ut, s, Vh = np.linalg.svd(np.asarray(Xt, dtype=np.float64), full_matrices=False)
    k = int(np.sum(s / s[0] >= ratio)) if s[0] > 0 else 0
    return Ut, s, Vh, k


def pcg(A, B, tol: float = 1e-6, maxit: int | None = None):
    """Jacobi-preconditioned conjugate gradient, one right-hand side at a
    time (Algorithm 2 step 3 solves every column with PCG; the paper names
    no preconditioner, the reading is diag(A)). x0 = 0; stop when
    |r|_2 <= tol |b|_2 or after maxit iterations (default 10 * rows).
    Returns (X, iterations per column, final relative residuals).
    """
    A = sp.csr_matrix(A)
    m = A.shape[0]
    B = np.asarray(B, dtype=np.float64).reshape(m, -1)
    maxit = 10 * max(m, 1) if maxit is None else maxit
    d = A.diagonal()
    minv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 1.0)
    X = np.zeros_like(B)
    its = np.zeros(B.shape[1], dtype=np.int64)
    res = np.zeros(B.shape[1])
    for c in range(B.shape[1]):
        b = B[:, c]
        nb = np.linalg.norm(b)
        x = np.zeros(m)
        if nb == 0.0:
            continue
        r = b.copy()
        z = minv * r
        pv = z.copy()
        rz = r @ z
        it = 0
        while np.linalg.norm(r) > tol * nb and it < maxit:
            q = A @ pv
            alpha = rz / (pv @ q)
            x += alpha * pv
            r -= alpha * q
            z = minv * r
            rz_new = r @ z
            pv = z + (rz_new / rz) * pv
            rz = rz_new
            it += 1
        X[:, c] = x
        its[c] = it
        res[c] = np.linalg.norm(r) / nb
    return X, its, res


def upsample_subspace(L, omega: np.ndarray, R: np.ndarray, tol: float = 1e-6,
                      maxit: int | None = None):
    """Lemma 1 / Eq. Uupsample: the minimiser of tr(S^T L S) subject to
    S(omega, :) = R has S(a, :) = -L_aa^{-1} L_ab R with a the complement
    of omega (b = omega), solved by PCG. Returns (S, its, res)."""
    L = sp.csr_matrix(L)
    N = L.shape[0]
    mask = np.ones(N, dtype=bool)
    mask[omega] = False
    a = np.nonzero(mask)[0]
    S = np.zeros((N, R.shape[1]))
    S[omega] = R
    if len(a) == 0 or R.shape[1] == 0:
        return S, np.zeros(R.shape[1], dtype=np.int64), np.zeros(R.shape[1])
    Laa = L[a][:, a]
    Lab = L[a][:, omega]
    Sa, its, res = pcg(Laa, -(Lab @ R), tol=tol, maxit=maxit)
    S[a] = Sa
    return S, its, res


def approx_decode(Xt, omega_r, omega_c, p: int, n: int, Lr, Lc,
                  ratio: float = 0.1, delta: float = 0.0, tol: float = 1e-6,
                  k_override: int | None = None, maxit: int | None = None,
                  want_X: bool = True):
    """Algorithm 2 (subspace-upsampling approximate decoder).

    1. SVD of X~; 2. rank k (see svd_rank); 3. upsample every column of
    U~ on L_r and of V~ on L_c (Lemma 1); 4. unit-normalise the columns
    of U and V; 5. Sigma = sqrt(n p / (rho_r rho_c (1 - delta))) Sigma~,
    delta (never given a value) defaults to 0; 6. X = U Sigma V^T.
    Returns dict with X (None when ``want_X`` is false: step 6 is then left
    to the caller, for matrices too large to hold), U, V, sigma, k and CG
    statistics.
    """
    rho_r, rho_c = Xt.shape
    Ut, s, Vh, k = svd_rank(Xt, ratio)
    if k_override is not None:
        k = int(k_override)
    Us, its_u, res_u = upsample_subspace(Lr, omega_r, Ut[:, :k], tol, maxit)
    Vs, its_v, res_v = upsample_subspace(Lc, omega_c, Vh[:k].T, tol, maxit)
    Us = Us / np.linalg.norm(Us, axis=0, keepdims=True)
    Vs = Vs / np.linalg.norm(Vs, axis=0, keepdims=True)
    sig = math.sqrt(n * p / (rho_r * rho_c * (1.0 - delta))) * s[:k]
    X = (Us * sig) @ Vs.T if want_X else None
    return {"X": X, "U": Us, "V": Vs, "sigma": sig, "k": k, "s_tilde": s,
            "cg_iters_u": its_u, "cg_iters_v": its_v, "res_u": res_u, "res_v": res_v}


# ---------------------------------------------------------------------------
# Whole pipeline (Table tab:cpca, steps 1-6)
# ---------------------------------------------------------------------------
def cpca(Y, K: int, rho_r: int, rho_c: int, seed: int, J: int,
         gamma_r: float, gamma_c: float, lap_type: int = LAP_NORMALIZED,
         cg_tol: float = 1e-6, power_iters: int = 200, power_seed: int = 0,
         ratio: float = 0.1, delta: float = 0.0, eps: float = 0.0):
    """Steps 1-6 of the complete CPCA algorithm on a dense Y (p x n)."""
    Y = np.asarray(Y, dtype=np.float64)
    p, n = Y.shape
    Lr, *_ = knn_graph(Y, K, lap_type)
    Lc, *_ = knn_graph(Y.T, K, lap_type)
    om_r = sample_indices(seed, p, rho_r, 0)
    om_c = sample_indices(seed, n, rho_c, 1)
    Yt = Y[np.ix_(om_r, om_c)]
    Lrt, *_ = knn_graph(Yt, K, lap_type)
    Lct, *_ = knn_graph(Yt.T, K, lap_type)
    nr = power_norm(Lrt, power_iters, power_seed, 2)
    nc = power_norm(Lct, power_iters, power_seed, 3)
    lam = fista_step(gamma_r, gamma_c, nr, nc)
    Xt, finfo = frpcag_fista(Yt, Lrt, Lct, gamma_r, gamma_c, lam, J, eps)
    dec = approx_decode(Xt, om_r, om_c, p, n, Lr, Lc, ratio, delta, cg_tol)
    dec.update({"Xt": Xt, "Yt": Yt, "omega_r": om_r, "omega_c": om_c, "lam": lam,
                "norm_r": nr, "norm_c": nc, "fista": finfo,
                "Lr": Lr, "Lc": Lc, "Lrt": Lrt, "Lct": Lct})
    return dec
