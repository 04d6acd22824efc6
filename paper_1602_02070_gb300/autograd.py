"""torch.autograd bindings of the library's hand-written adjoints.

Each Function's forward calls the CUDA forward (cpca_laplacian_values,
cpca_frpcag_solve, cpca_decode + cpca_decode_entries) and its backward the
matching reverse-mode entry point (cpca_laplacian_weight_grad,
cpca_frpcag_backward, cpca_decode_backward). Argument marshalling only.

Graphs enter as CSR patterns (row pointers, columns) plus per-entry values;
`laplacian` turns per-entry edge weights into values, so losses can be
differentiated with respect to the weights. The kNN selection that produced
a pattern is not differentiated.
"""
from __future__ import annotations

import torch

from . import capi
from .capi import LAP_NORMALIZED, Csr


class _Laplacian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, rowptr, col, lap_type):
        val = capi.laplacian_values(Csr(rowptr, col, None), w.contiguous(), lap_type)
        ctx.save_for_backward(w, rowptr, col, val)
        ctx.lap_type = lap_type
        return val

    @staticmethod
    def backward(ctx, dval):
        w, rowptr, col, val = ctx.saved_tensors
        dw = capi.laplacian_weight_grad(Csr(rowptr, col, val), w.contiguous(),
                                        dval.double().contiguous(), ctx.lap_type)
        return dw, None, None, None


def laplacian(rowptr: torch.Tensor, col: torch.Tensor, w: torch.Tensor,
              lap_type: int = LAP_NORMALIZED) -> torch.Tensor:
    """Differentiable Laplacian values on the pattern (rowptr, col) from the
    per-entry edge weights w (Sec. I)."""
    return _Laplacian.apply(w, rowptr, col, lap_type)


class _FRPCAG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Yt, gamma_r, gamma_c, Lr_val, Lc_val, Lr_pat, Lc_pat, max_iter, power_iters,
                ckpt_every):
        Lr = Csr(Lr_pat.rowptr, Lr_pat.col, Lr_val.contiguous())
        Lc = Csr(Lc_pat.rowptr, Lc_pat.col, Lc_val.contiguous())
        prm = capi.frpcag_params(float(gamma_r), float(gamma_c), -1.0, int(max_iter), 0.0,
                                 int(power_iters))
        # the forward keeps its tape (power iterates, lambda, checkpoints)
        # for the backward, which then skips recomputing them
        X, ws, _ = capi.cpca_frpcag_forward_tape(Yt, Lr, Lc, prm, int(ckpt_every))
        ctx.save_for_backward(Yt, gamma_r, Lr.val, Lc.val)
        ctx.graphs = (Lr, Lc)
        ctx.prm = prm
        ctx.ckpt_every = int(ckpt_every)
        ctx.tape = ws
        return X

    @staticmethod
    def backward(ctx, dX):
        Yt, gamma_r, _, _ = ctx.saved_tensors
        Lr, Lc = ctx.graphs
        out = capi.cpca_frpcag_backward(Yt, Lr, Lc, dX.contiguous(), ctx.prm, ctx.ckpt_every,
                                        want_dL=True, ws=ctx.tape, resume=True)
        ctx.tape = None
        info = out["info"]
        dgr = torch.tensor(info.dgamma_r, dtype=gamma_r.dtype, device=gamma_r.device)
        dgc = torch.tensor(info.dgamma_c, dtype=gamma_r.dtype, device=gamma_r.device)
        return (out["dYt"], dgr, dgc, out["dLr"].float(), out["dLc"].float(),
                None, None, None, None, None)


def frpcag(Yt: torch.Tensor, gamma_r: torch.Tensor, gamma_c: torch.Tensor, Lr_val: torch.Tensor,
           Lc_val: torch.Tensor, Lr_pat: Csr, Lc_pat: Csr, max_iter: int = 300,
           power_iters: int = 200, ckpt_every: int = 20) -> torch.Tensor:
    """FISTA for FRPCAG (Algorithm 1, fixed max_iter, lambda by power
    iteration) as a differentiable function of Y~, gamma_r, gamma_c (0-d
    tensors) and the Laplacian values; backward = cpca_frpcag_backward with
    checkpoints every ckpt_every iterations."""
    return _FRPCAG.apply(Yt, gamma_r, gamma_c, Lr_val, Lc_val, Lr_pat, Lc_pat, max_iter,
                         power_iters, ckpt_every)


class _DecodeEntries(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Xt, Lr_val, Lc_val, Lr_pat, Lc_pat, omega_r, omega_c, p, n, h_row, h_col,
                dparams):
        Lr = Csr(Lr_pat.rowptr, Lr_pat.col, Lr_val.contiguous())
        Lc = Csr(Lc_pat.rowptr, Lc_pat.col, Lc_val.contiguous())
        # the backward's workspace: the decoder leaves its factors there
        ws = capi.decode_backward_workspace(Xt, p, n, Lr, Lc, dparams)
        dec = capi.cpca_decode(Xt, omega_r, omega_c, p, n, Lr, Lc, dparams, want_X=False, ws=ws)
        vals = capi.decode_entries(dec["U"], dec["V"], dec["sigma"], dec["k"], h_row, h_col)
        ctx.save_for_backward(Xt, Lr.val, Lc.val, omega_r, omega_c, h_row, h_col)
        ctx.graphs = (Lr, Lc)
        ctx.meta = (p, n, dec["k"], dparams)
        ctx.ws = ws
        return vals

    @staticmethod
    def backward(ctx, g):
        Xt, _, _, omega_r, omega_c, h_row, h_col = ctx.saved_tensors
        Lr, Lc = ctx.graphs
        p, n, k, dparams = ctx.meta
        out = capi.cpca_decode_backward(Xt, omega_r, omega_c, p, n, Lr, Lc, k, h_row, h_col,
                                        g.float().contiguous(), dparams, want_dL=True, ws=ctx.ws,
                                        resume=True)
        ctx.ws = None
        return (out["dXt"], out["dLr"].float(), out["dLc"].float()) + (None,) * 9


def decode_entries(Xt: torch.Tensor, Lr_val: torch.Tensor, Lc_val: torch.Tensor, Lr_pat: Csr,
                   Lc_pat: Csr, omega_r: torch.Tensor, omega_c: torch.Tensor, p: int, n: int,
                   h_row: torch.Tensor, h_col: torch.Tensor,
                   dparams: capi.cpca_decode_params | None = None) -> torch.Tensor:
    """Algorithm 2's X at the entries (h_row, h_col), differentiable in X~
    and the full graphs' Laplacian values (rank k fixed by the forward)."""
    return _DecodeEntries.apply(Xt, Lr_val, Lc_val, Lr_pat, Lc_pat, omega_r, omega_c, p, n, h_row,
                                h_col, dparams if dparams is not None else capi.decode_params())
