"""Pins of the oracle's SINR gradients (no GPU).

The autograd gradient (oracle.adjoint, torch float64) is checked entry by
entry against central finite differences of the independent NumPy forward
(oracle.sinr), and its forward against that NumPy forward.
"""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import sinr as S


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(rng, r, c):
    Q, _ = np.linalg.qr(_rand(rng, (r, c)))
    return Q


def _system(seed, J=2, N=6, P=3, m=3, n=4, p=2, K=2, L=2):
    rng = np.random.default_rng(seed)
    B = np.stack([_orth(rng, N, n) for _ in range(J)])
    C = np.stack([[_orth(rng, P, p) for _ in range(J)] for _ in range(J)])
    G = _rand(rng, (J, J, m, n, p))
    coef = _rand(rng, (J, J, K, P))
    s2 = rng.uniform(0.2, 1.0, J)
    Pw = np.stack([_orth(rng, N, L) for _ in range(J)])
    dsinr = rng.standard_normal((J, K, L))
    return B, C, G, coef, s2, Pw, dsinr


def test_complex_gradient_convention():
    # l = |z|^2 = x^2 + y^2 -> dl/dx + i dl/dy = 2 z
    import torch
    z = torch.tensor([0.3 - 0.7j], dtype=torch.complex128, requires_grad=True)
    (torch.abs(z) ** 2).sum().backward()
    assert abs(z.grad[0].item() - 2 * (0.3 - 0.7j)) < 1e-14


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_vjp_matches_central_differences(precoder):
    B, C, G, coef, s2, Pw, dsinr = _system(11)
    J, L = G.shape[0], Pw.shape[2]
    out = AD.tucker_sinr_vjp(G, C, coef, s2, L, dsinr, precoder, B, Pw)
    Pt = lambda Bx: np.stack([S.project_precoder(Bx[k], Pw[k]) for k in range(J)])  # noqa: E731
    np.testing.assert_allclose(out["sinr"], S.tucker_sinr(G, C, coef, s2, L, precoder, Pt(B)),
                               rtol=1e-11)

    def loss_G(Gx):
        return float(np.sum(dsinr * S.tucker_sinr(Gx, C, coef, s2, L, precoder, Pt(B))))

    def loss_C(Cx):
        return float(np.sum(dsinr * S.tucker_sinr(G, Cx, coef, s2, L, precoder, Pt(B))))

    def loss_B(Bx):
        return float(np.sum(dsinr * S.tucker_sinr(G, C, coef, s2, L, precoder, Pt(Bx))))

    rng = np.random.default_rng(0)
    checks = [(loss_G, G, out["dG"]), (loss_C, C, out["dC"])]
    if precoder == "mmse":
        checks.append((loss_B, B, out["dB"]))
    for f, z, g in checks:
        scale = np.max(np.abs(g))
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in z.shape)
            fd = AD.central_difference(f, z, idx, 1e-6)
            assert abs(fd - g[idx]) < 1e-6 * scale + 1e-6 * abs(g[idx]), (idx, fd, g[idx])
