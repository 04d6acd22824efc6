"""FP64 reverse-mode derivatives of the CPCA hot path (test infrastructure only).

The paper has no derivatives; what is differentiated, and how, is a
reading of the problem it states:

* The loss is a function of the decoded X (Algorithm 2) at a set of
  entries; its gradient there is an input.
* What varies: gamma_r, gamma_c, the sampled matrix Y~, and the weight w_e
  of every undirected edge of the four graphs (full L_r, L_c used by the
  decoder; compressed L~_r, L~_c used by FISTA). The Laplacians are the
  functions of W of Sec. I, so a weight moves its entry and both degrees.
  kNN selection and the Gaussian kernel are not differentiated (the graphs
  are inputs).
* lambda = 1/beta' (Sec. IV-B) depends on gamma and on the norms |L~|_2,
  which are the outputs of the fixed power iteration (same start vector,
  same count); the derivative is that of the computed estimate, by
  reverse mode through the iterations.
* FISTA (Algorithm 1) runs a fixed J; the prox is differentiated where it
  is smooth (its derivative is the indicator |V - Y~| > lambda).
* The decoder keeps k fixed; the SVD derivative uses the full thin SVD of
  X~ (Townsend, "Differentiating the singular value decomposition", 2016);
  the harmonic extension of Lemma 1 is differentiated through an exact
  sparse solve with L_aa.

Every function stores the whole forward trajectory (no checkpointing):
plain and slow on purpose.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import cpca_oracle as O

__all__ = [
    "pattern_outer", "laplacian_weight_vjp", "power_norm_vjp", "fista_step_vjp",
    "frpcag_fista_vjp", "svd_topk_vjp", "approx_decode_exact", "approx_decode_vjp",
    "cpca_loss", "cpca_loss_grad",
]


def pattern_outer(L, A, B):
    """Sparse matrix on L's pattern with entry (i, j) = sum_c A[i, c] B[j, c]."""
    C = sp.csr_matrix(L, copy=True).tocoo()
    vals = np.einsum("ec,ec->e", np.atleast_2d(A.T).T[C.row], np.atleast_2d(B.T).T[C.col])
    return sp.csr_matrix((vals, (C.row, C.col)), shape=L.shape)


def laplacian_weight_vjp(W, Lbar, lap_type: int = O.LAP_NORMALIZED):
    """Gradient with respect to the undirected edge weights, given Lbar =
    dloss/dL on L's pattern (entries ij and ji separate).

    Normalised: L_ij = -w_ij / sqrt(D_i D_j) (i != j), L_ii constant, so
      dloss/dD_k = -sum_{j != k} (Lbar_kj L_kj + Lbar_jk L_jk) / (2 D_k),
      dloss/dw_ab = -(Lbar_ab + Lbar_ba) / sqrt(D_a D_b) + dD_a + dD_b.
    Combinatorial: L_ij = -w_ij, L_ii = D_i:
      dloss/dw_ab = -(Lbar_ab + Lbar_ba) + Lbar_aa + Lbar_bb.
    Returns a CSR matrix on W's pattern holding dloss/dw_e at both entries
    of each edge.
    """
    W = sp.csr_matrix(W).tocoo()
    Lb = sp.csr_matrix(Lbar)
    N = W.shape[0]
    deg = np.asarray(sp.csr_matrix(W).sum(axis=1)).ravel()
    lb_ij = np.asarray(Lb[W.row, W.col]).ravel()
    lb_ji = np.asarray(Lb[W.col, W.row]).ravel()
    if lap_type == O.LAP_COMBINATORIAL:
        dg = Lb.diagonal()
        g = -(lb_ij + lb_ji) + dg[W.row] + dg[W.col]
    else:
        s = np.sqrt(deg[W.row] * deg[W.col])
        lij = -W.data / s
        # each stored (i, j) with i = row adds Lbar_ij L_ij to D_i and D_j
        contrib = lb_ij * lij
        dD = np.zeros(N)
        np.add.at(dD, W.row, contrib)
        np.add.at(dD, W.col, contrib)
        dD = np.where(deg > 0, -dD / (2.0 * np.where(deg > 0, deg, 1.0)), 0.0)
        g = -(lb_ij + lb_ji) / s + dD[W.row] + dD[W.col]
    return sp.csr_matrix((g, (W.row, W.col)), shape=(N, N))


def power_norm_vjp(L, rho_bar: float, iters: int = 200, seed: int = 0, stream: int = 2):
    """dloss/dL (on L's pattern) of power_norm(L, iters, seed, stream),
    given rho_bar = dloss/drho. Forward: v_0 fixed; w_t = L v_{t-1},
    v_t = w_t / |w_t|; rho = v^T L v / v^T v at v = v_T."""
    L = sp.csr_matrix(L)
    N = L.shape[0]
    v = O.uniform01(seed, stream, N) - 0.5
    v /= np.linalg.norm(v)
    vs, nws = [v], []
    for _ in range(iters):
        w = L @ v
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return sp.csr_matrix(L.shape)
        v = w / nw
        vs.append(v)
        nws.append(nw)
    vT = vs[-1]
    vv = vT @ vT
    Lv = L @ vT
    rho = vT @ Lv / vv
    Lbar = pattern_outer(L, rho_bar * vT[:, None] / vv, vT[:, None])
    vbar = rho_bar * 2.0 * (Lv - rho * vT) / vv
    for t in range(iters, 0, -1):
        vt, nw = vs[t], nws[t - 1]
        wbar = (vbar - vt * (vt @ vbar)) / nw
        Lbar = Lbar + pattern_outer(L, wbar[:, None], vs[t - 1][:, None])
        vbar = L.T @ wbar
    return Lbar


def fista_step_vjp(gamma_r, gamma_c, norm_r, norm_c, lam_bar):
    """Gradients of lambda = 1/(2 gamma_c n_c + 2 gamma_r n_r) with respect
    to (gamma_r, gamma_c, n_r, n_c); zero where beta' = 0 (lambda = 1)."""
    beta = 2.0 * gamma_c * norm_c + 2.0 * gamma_r * norm_r
    if beta <= 0:
        return 0.0, 0.0, 0.0, 0.0
    d = -lam_bar / (beta * beta)
    return 2.0 * norm_r * d, 2.0 * norm_c * d, 2.0 * gamma_r * d, 2.0 * gamma_c * d


def frpcag_fista_vjp(Yt, Lr, Lc, gamma_r, gamma_c, lam, J: int, S_bar):
    """Reverse mode through J iterations of Algorithm 1 (eps = 0).

    Forward, as frpcag_fista: Z_1 = S_0 = Y~;
      V_j = Z_j - 2 lam (gamma_c Z_j L_c + gamma_r L_r Z_j), R_j = V_j - Y~,
      S_j = Y~ + sgn(R_j) max(|R_j| - lam, 0),
      Z_{j+1} = (1 + mu_j) S_j - mu_j S_{j-1}, mu_j = (t_j - 1)/t_{j+1}.
    Returns dict: Yt, gamma_r, gamma_c, lam, Lr, Lc (sparse on the
    patterns), and the number of entries within 1e-9 of a prox kink.
    """
    Yt = np.asarray(Yt, dtype=np.float64)
    Lr, Lc = sp.csr_matrix(Lr), sp.csr_matrix(Lc)
    # forward, keeping every S_j
    S = [Yt.copy()]
    Z = Yt.copy()
    t = 1.0
    mus = [0.0]
    for j in range(1, J + 1):
        V = Z - lam * 2.0 * (gamma_c * (Z @ Lc) + gamma_r * (Lr @ Z))
        R = V - Yt
        S.append(Yt + np.sign(R) * np.maximum(np.abs(R) - lam, 0.0))
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        mus.append((t - 1.0) / t_next)
        Z = (1.0 + mus[j]) * S[j] - mus[j] * S[j - 1]
        t = t_next
    # reverse
    Sb = [np.zeros_like(Yt) for _ in range(J + 1)]
    Sb[J] = np.asarray(S_bar, dtype=np.float64).copy()
    Yb = np.zeros_like(Yt)
    gr_b = gc_b = lam_b = 0.0
    Lr_b = sp.csr_matrix(Lr.shape)
    Lc_b = sp.csr_matrix(Lc.shape)
    near = 0
    for j in range(J, 0, -1):
        Zj = Yt if j == 1 else (1.0 + mus[j - 1]) * S[j - 1] - mus[j - 1] * S[j - 2]
        LrZ = Lr @ Zj
        ZLc = Zj @ Lc
        R = Zj - lam * 2.0 * (gamma_c * ZLc + gamma_r * LrZ) - Yt
        M = np.abs(R) > lam
        near += int(np.sum(np.abs(np.abs(R) - lam) < 1e-9))
        Vb = np.where(M, Sb[j], 0.0)
        Yb += Sb[j] - Vb
        lam_b += float(np.sum(-np.sign(R) * Vb))
        lam_b += float(-np.sum(Vb * 2.0 * (gamma_c * ZLc + gamma_r * LrZ)))
        gr_b += -2.0 * lam * float(np.sum(Vb * LrZ))
        gc_b += -2.0 * lam * float(np.sum(Vb * ZLc))
        Lr_b = Lr_b + pattern_outer(Lr, -2.0 * lam * gamma_r * Vb, Zj)
        Lc_b = Lc_b + pattern_outer(Lc, -2.0 * lam * gamma_c * Zj.T, Vb.T)
        Zb = Vb - 2.0 * lam * (gamma_c * (Vb @ Lc.T) + gamma_r * (Lr.T @ Vb))
        if j == 1:
            Yb += Zb
        else:
            Sb[j - 1] += (1.0 + mus[j - 1]) * Zb
            Sb[j - 2] += -mus[j - 1] * Zb
    Yb += Sb[0]
    return {"Yt": Yb, "gamma_r": gr_b, "gamma_c": gc_b, "lam": lam_b, "Lr": Lr_b,
            "Lc": Lc_b, "near_kinks": near}


def svd_topk_vjp(A, k: int, U_bar, s_bar, V_bar):
    """dloss/dA for a loss of the top-k singular triplets (U_k, s_k, V_k)
    of A, by the full thin SVD and Townsend's formula:
      A_bar = U [ (F o (U^T Ub - Ub^T U)) S + diag(sb) + S (F o (V^T Vb - Vb^T V)) ] V^T
              + (I - U U^T) Ub S^-1 V^T + U S^-1 Vb^T (I - V V^T),
    F_ij = 1/(s_j^2 - s_i^2) (i != j), with Ub, sb, Vb zero beyond k."""
    A = np.asarray(A, dtype=np.float64)
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    V = Vh.T
    r = len(s)
    Ub = np.zeros((A.shape[0], r))
    Vb = np.zeros((A.shape[1], r))
    sb = np.zeros(r)
    Ub[:, :k], Vb[:, :k], sb[:k] = U_bar, V_bar, s_bar
    s2 = s * s
    with np.errstate(divide="ignore"):
        F = 1.0 / (s2[None, :] - s2[:, None])
    np.fill_diagonal(F, 0.0)
    F[k:, k:] = 0.0  # pairs outside the top k meet only zero adjoints
    Ju = U.T @ Ub
    Jv = V.T @ Vb
    inner = (F * (Ju - Ju.T)) * s[None, :] + np.diag(sb) + s[:, None] * (F * (Jv - Jv.T))
    Ab = U @ inner @ V.T
    Ubk_s = Ub[:, :k] / s[:k]
    Vbk_s = Vb[:, :k] / s[:k]
    Ab += (Ubk_s - U @ (U.T @ Ubk_s)) @ V[:, :k].T
    Ab += U[:, :k] @ (Vbk_s - V @ (V.T @ Vbk_s)).T
    return Ab


def _split(L, omega):
    L = sp.csr_matrix(L)
    mask = np.ones(L.shape[0], dtype=bool)
    mask[omega] = False
    a = np.nonzero(mask)[0]
    return L, a


def _extend_exact(L, omega, R):
    """Lemma 1 with an exact sparse solve: S(omega) = R, S(a) = -L_aa^-1 L_ab R."""
    L, a = _split(L, omega)
    S = np.zeros((L.shape[0], R.shape[1]))
    S[omega] = R
    if len(a):
        Laa = sp.csc_matrix(L[a][:, a])
        S[a] = sla.spsolve(Laa, -(L[a][:, omega] @ R)).reshape(len(a), -1)
    return S


def approx_decode_exact(Xt, omega_r, omega_c, p, n, Lr, Lc, k, delta=0.0):
    """Algorithm 2 with a fixed k and exact sparse solves (the limit of
    PCG at zero tolerance). Returns dict of U, V (unit columns), sigma and
    the intermediates the derivative needs."""
    rho_r, rho_c = Xt.shape
    Ut, s, Vh, _ = O.svd_rank(Xt)
    Uh = _extend_exact(Lr, omega_r, Ut[:, :k])
    Vhh = _extend_exact(Lc, omega_c, Vh[:k].T)
    nu, nv = np.linalg.norm(Uh, axis=0), np.linalg.norm(Vhh, axis=0)
    c = math.sqrt(n * p / (rho_r * rho_c * (1.0 - delta)))
    return {"U": Uh / nu, "V": Vhh / nv, "sigma": c * s[:k], "Uh": Uh, "Vh": Vhh,
            "nu": nu, "nv": nv, "c": c, "k": k}


def _extend_vjp(L, omega, Sh, Sbar):
    """Adjoint of S = extension(R) on L: returns (R_bar, L_bar). Rows a:
    Lambda = L_aa^-T Sbar(a); R_bar = Sbar(omega) - L_{a,omega}^T Lambda;
    L_bar(i, j) = -sum_c Lambda_ic S_jc for i in a."""
    L, a = _split(L, omega)
    N, k = Sbar.shape
    Rb = Sbar[omega].copy()
    Lb = sp.csr_matrix(L.shape)
    if len(a):
        Laa = sp.csc_matrix(L[a][:, a]).T
        Lam = sla.spsolve(sp.csc_matrix(Laa), Sbar[a]).reshape(len(a), k)
        Rb -= (L[a][:, omega]).T @ Lam
        LamF = np.zeros((N, k))
        LamF[a] = Lam
        Lb = pattern_outer(L, -LamF, Sh)
    return Rb, Lb


def approx_decode_vjp(Xt, omega_r, omega_c, p, n, Lr, Lc, k, rows, cols, g, delta=0.0):
    """dloss/dXt, dloss/dL_r, dloss/dL_c for a loss of the decoded X at the
    entries (rows[e], cols[e]) with dloss/dX there = g[e] (k fixed, exact
    solves). X = U diag(sigma) V^T, U = Uh / |Uh|, Uh = extension of
    U~_k on L_r, sigma = c s_k; likewise V."""
    d = approx_decode_exact(Xt, omega_r, omega_c, p, n, Lr, Lc, k, delta)
    U, V, sig = d["U"], d["V"], d["sigma"]
    g = np.asarray(g, dtype=np.float64)
    Ub = np.zeros_like(U)
    Vb = np.zeros_like(V)
    np.add.at(Ub, rows, g[:, None] * V[cols] * sig)
    np.add.at(Vb, cols, g[:, None] * U[rows] * sig)
    sig_b = np.einsum("e,ec,ec->c", g, U[rows], V[cols])
    s_b = d["c"] * sig_b
    Uhb = (Ub - U * np.sum(U * Ub, axis=0)) / d["nu"]
    Vhb = (Vb - V * np.sum(V * Vb, axis=0)) / d["nv"]
    Utb, Lr_b = _extend_vjp(Lr, omega_r, d["Uh"], Uhb)
    Vtb, Lc_b = _extend_vjp(Lc, omega_c, d["Vh"], Vhb)
    Xtb = svd_topk_vjp(Xt, k, Utb, s_b, Vtb)
    return {"Xt": Xtb, "Lr": Lr_b, "Lc": Lc_b, "decode": d}


def cpca_loss(Y, Wr, Wc, Wrt, Wct, omega_r, omega_c, gamma_r, gamma_c, J, k,
              rows, cols, lap_type=O.LAP_NORMALIZED, power_iters=200, power_seed=0):
    """Held-out loss 1/2 sum_e (X_e - Y_e)^2 at entries (rows, cols) of the
    pipeline with given graph weights: Y~ = Y(omega_r, omega_c), FISTA on
    the Laplacians of Wrt, Wct with lambda from the power iterations, then
    Algorithm 2 (fixed k, exact solves) on the Laplacians of Wr, Wc.
    Returns (loss, X at the entries)."""
    Y = np.asarray(Y, dtype=np.float64)
    p, n = Y.shape
    Yt = Y[np.ix_(omega_r, omega_c)]
    Lrt = O.laplacian_from_weights(Wrt, lap_type)
    Lct = O.laplacian_from_weights(Wct, lap_type)
    nr = O.power_norm(Lrt, power_iters, power_seed, 2)
    nc = O.power_norm(Lct, power_iters, power_seed, 3)
    lam = O.fista_step(gamma_r, gamma_c, nr, nc)
    Xt, _ = O.frpcag_fista(Yt, Lrt, Lct, gamma_r, gamma_c, lam, J)
    Lr = O.laplacian_from_weights(Wr, lap_type)
    Lc = O.laplacian_from_weights(Wc, lap_type)
    d = approx_decode_exact(Xt, omega_r, omega_c, p, n, Lr, Lc, k)
    Xe = np.einsum("ec,c,ec->e", d["U"][rows], d["sigma"], d["V"][cols])
    return 0.5 * float(np.sum((Xe - Y[rows, cols]) ** 2)), Xe


def cpca_loss_grad(Y, Wr, Wc, Wrt, Wct, omega_r, omega_c, gamma_r, gamma_c, J, k,
                   rows, cols, lap_type=O.LAP_NORMALIZED, power_iters=200, power_seed=0):
    """Gradient of cpca_loss with respect to gamma_r, gamma_c, Y~ and the
    edge weights of the four graphs. Returns dict: loss, gamma_r, gamma_c,
    Yt (rho_r x rho_c), Wr, Wc, Wrt, Wct (CSR on each W's pattern, the edge
    derivative at both entries), and the FISTA kink count."""
    Y = np.asarray(Y, dtype=np.float64)
    p, n = Y.shape
    Yt = Y[np.ix_(omega_r, omega_c)]
    Lrt = O.laplacian_from_weights(Wrt, lap_type)
    Lct = O.laplacian_from_weights(Wct, lap_type)
    nr = O.power_norm(Lrt, power_iters, power_seed, 2)
    nc = O.power_norm(Lct, power_iters, power_seed, 3)
    lam = O.fista_step(gamma_r, gamma_c, nr, nc)
    Xt, _ = O.frpcag_fista(Yt, Lrt, Lct, gamma_r, gamma_c, lam, J)
    Lr = O.laplacian_from_weights(Wr, lap_type)
    Lc = O.laplacian_from_weights(Wc, lap_type)
    d = approx_decode_exact(Xt, omega_r, omega_c, p, n, Lr, Lc, k)
    Xe = np.einsum("ec,c,ec->e", d["U"][rows], d["sigma"], d["V"][cols])
    g = Xe - Y[rows, cols]
    dec = approx_decode_vjp(Xt, omega_r, omega_c, p, n, Lr, Lc, k, rows, cols, g)
    fb = frpcag_fista_vjp(Yt, Lrt, Lct, gamma_r, gamma_c, lam, J, dec["Xt"])
    gr, gc, nr_b, nc_b = fista_step_vjp(gamma_r, gamma_c, nr, nc, fb["lam"])
    Lrt_b = fb["Lr"] + power_norm_vjp(Lrt, nr_b, power_iters, power_seed, 2)
    Lct_b = fb["Lc"] + power_norm_vjp(Lct, nc_b, power_iters, power_seed, 3)
    return {
        "loss": 0.5 * float(np.sum(g * g)),
        "gamma_r": fb["gamma_r"] + gr, "gamma_c": fb["gamma_c"] + gc,
        "Yt": fb["Yt"],
        "Wr": laplacian_weight_vjp(Wr, dec["Lr"], lap_type),
        "Wc": laplacian_weight_vjp(Wc, dec["Lc"], lap_type),
        "Wrt": laplacian_weight_vjp(Wrt, Lrt_b, lap_type),
        "Wct": laplacian_weight_vjp(Wct, Lct_b, lap_type),
        "lam": lam, "Xt": Xt, "near_kinks": fb["near_kinks"], "g": g,
        "Xt_bar": dec["Xt"], "Lr_bar": dec["Lr"], "Lc_bar": dec["Lc"],
        "Lrt_bar": Lrt_b, "Lct_bar": Lct_b, "lam_bar": fb["lam"],
    }
