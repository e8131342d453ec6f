"""torch.autograd.Function over the CUDA SINR kernels and their adjoints.

``compressed_sinr(G, C, alpha, tau, sigma2, dims, precoder="svd", Pt=None)``
returns the SINR [J][K][L] of the groupwise Tucker form on the device; its
backward calls the library's adjoint kernels (``ts_sinr_svd_adjoint`` /
``ts_sinr_mmse_adjoint``), which recompute the per-subcarrier quantities
instead of storing them.  Tensors use the library's device layouts
(``G``: [J*J][p][m][n], ``C``: [J*J][P][p], ``Pt``: [J][n][L], complex64;
``alpha``: [J*J][P] complex64, ``tau``: [J*J][P] float32 seconds,
``sigma2``: [J] float32).  Gradients of complex tensors follow PyTorch's
convention, dl/dRe + i dl/dIm, which is the library's.
"""
from __future__ import annotations

import torch

from . import tuckersinr as ts


class _CompressedSinr(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, C, Pt, alpha, tau, sigma2, dims, precoder):
        coef, keep = ts.make_coef(alpha=alpha, tau=tau)
        J, K, L = dims.J, dims.K, dims.L
        sinr = torch.empty(J, K, L, device=G.device, dtype=torch.float32)
        if precoder == "svd":
            ws = ts.workspace(dims, ts.TS_OP_SINR_SVD, G.device)
            ts.ts_sinr_svd(dims, coef, G, C, sigma2, sinr, None, ws)
        else:
            ws = ts.workspace(dims, ts.TS_OP_SINR_MMSE, G.device)
            ts.ts_sinr_mmse(dims, coef, G, C, Pt, sigma2, sinr, None, ws)
        del keep
        ctx.save_for_backward(G, C, Pt if Pt is not None else G.new_empty(0), alpha, tau, sigma2)
        ctx.dims, ctx.precoder, ctx.has_pt = dims, precoder, Pt is not None
        return sinr

    @staticmethod
    def backward(ctx, dsinr):
        G, C, Pt, alpha, tau, sigma2 = ctx.saved_tensors
        dims = ctx.dims
        coef, keep = ts.make_coef(alpha=alpha, tau=tau)
        dsinr = dsinr.contiguous().float()
        dG = torch.empty_like(G)
        dC = torch.empty_like(C)
        dPt = None
        if ctx.precoder == "svd":
            ws = ts.workspace(dims, ts.TS_OP_SINR_SVD_ADJOINT, G.device)
            ts.ts_sinr_svd_adjoint(dims, coef, G, C, sigma2, dsinr, dG, dC, None, ws)
        else:
            dPt = torch.empty_like(Pt)
            ws = ts.workspace(dims, ts.TS_OP_SINR_MMSE_ADJOINT, G.device)
            ts.ts_sinr_mmse_adjoint(dims, coef, G, C, Pt, sigma2, dsinr, dG, dC, dPt, None, ws)
        del keep
        return dG, dC, (dPt if ctx.has_pt else None), None, None, None, None, None


def compressed_sinr(G, C, alpha, tau, sigma2, dims, precoder="svd", Pt=None):
    """SINR of the compressed form, differentiable in G, C (and Pt)."""
    if precoder not in ("svd", "mmse"):
        raise ValueError(precoder)
    if precoder == "mmse" and Pt is None:
        raise ValueError("the wideband-precoder variant needs Pt")
    return _CompressedSinr.apply(G, C, Pt, alpha, tau, sigma2, dims, precoder)
