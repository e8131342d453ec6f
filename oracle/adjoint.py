"""Gradients of the compressed SINR -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no adjoint; this module differentiates its compressed SINR
(eq. 15, 23-28) so that the CUDA adjoint can be checked.  The forward pass is
restated in float64 / complex128 PyTorch on the CPU and differentiated by
autograd; `central_difference` re-derives single entries from the NumPy
forward in `oracle.sinr`, which shares no code with this module.

Gradient convention for a real loss l of a complex parameter z = x + iy:
grad = dl/dx + i dl/dy.
"""
from __future__ import annotations

import numpy as np
import torch


def _c(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128)


def tucker_sinr_t(G, C, coef, sigma2, L, precoder="svd", Pt=None):
    """Compressed SINR (J, K, L) in torch; same steps as `oracle.sinr.tucker_sinr`."""
    J = G.shape[0]
    w = torch.einsum("ikxP,ikPq->ikxq", torch.conj(coef), C)          # c* C, eq. (15)
    Ht = torch.einsum("ikxq,ikabq->ikxab", w, G)                       # G x_3 (c* C)
    if precoder == "svd":
        V = []
        for k in range(J):
            _, _, Vh = torch.linalg.svd(Ht[k, k], full_matrices=False)  # eq. (7), (23)
            V.append(torch.conj(Vh[:, :L, :]).transpose(1, 2))
    else:
        V = [Pt[k].unsqueeze(0).expand(Ht.shape[2], -1, -1) for k in range(J)]
    out = []
    for i in range(J):
        E = [Ht[i, k] @ V[k] for k in range(J)]                        # eq. (24)
        r = E[0].shape[1]
        eye_r = torch.eye(r, dtype=torch.complex128)
        R = sum(E[k] @ E[k].mH for k in range(J) if k != i) + sigma2[i] * eye_r
        Eii = E[i]
        Lr = torch.linalg.cholesky(R)
        Z = torch.linalg.solve_triangular(Lr, Eii, upper=False)
        eye_l = torch.eye(Eii.shape[2], dtype=torch.complex128)
        F = eye_l + Z.mH @ Z
        Lf_inv = torch.linalg.solve_triangular(torch.linalg.cholesky(F),
                                               eye_l.expand(F.shape[0], -1, -1), upper=False)
        x = torch.sum(torch.abs(Lf_inv) ** 2, dim=1)
        Gm = eye_r + Z @ Z.mH
        Y = torch.linalg.solve_triangular(torch.linalg.cholesky(Gm), Z, upper=False)
        a = torch.sum(torch.abs(Y) ** 2, dim=1)
        out.append(a / x)
    return torch.stack(out)


def tucker_sinr_vjp(G, C, coef, sigma2, L, dsinr, precoder="svd", B=None, Pfull=None):
    """Vector-Jacobian product of the compressed SINR.

    Returns dict with dG, dC (and dB for precoder="mmse", through
    P~_k = B_k^T P_k) of l = sum(dsinr * SINR), plus the SINR itself.
    """
    Gt = _c(G).requires_grad_(True)
    Ct = _c(C).requires_grad_(True)
    ins = [Gt, Ct]
    Pt = None
    if precoder == "mmse":
        Bt = _c(B).requires_grad_(True)
        ins.append(Bt)
        Pt = torch.einsum("kNn,kNl->knl", Bt, _c(Pfull))
    s = tucker_sinr_t(Gt, Ct, _c(coef), torch.as_tensor(np.asarray(sigma2), dtype=torch.float64),
                      L, precoder, Pt)
    loss = torch.sum(torch.as_tensor(np.asarray(dsinr), dtype=torch.float64) * s)
    grads = torch.autograd.grad(loss, ins)
    out = {"sinr": s.detach().numpy(), "dG": grads[0].numpy(), "dC": grads[1].numpy()}
    if precoder == "mmse":
        out["dB"] = grads[2].numpy()
    return out


def central_difference(f, z: np.ndarray, index: tuple, h: float) -> complex:
    """dl/dRe + i dl/dIm of the real scalar f at entry `index` of z, by central differences."""
    def at(delta):
        zz = z.copy()
        zz[index] += delta
        return f(zz)
    d_re = (at(h) - at(-h)) / (2 * h)
    d_im = (at(1j * h) - at(-1j * h)) / (2 * h)
    return complex(d_re, d_im)
