"""Dense and compressed (groupwise Tucker) SINR evaluation -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

System (Section 2.2, eq. 1) with one UE per cell, as in the paper's
experiments (Section 4: only the first UE of each other cell interferes, no
intra-cell interference): UE i receives L streams from BS i; every other BS k
interferes with the L streams it sends to its own UE.

Readings of points the paper leaves open:
  * subcarrier model: c_p(kappa) = conj(alpha_p exp(-j 2 pi kappa df tau_p)),
    kappa = 0..K-1, so that eq. (9), H = X x_3 c*, gives
    H(kappa) = sum_p alpha_p exp(-j 2 pi kappa df tau_p) X_p;
  * the matrix form of G x_1 A x_2 B (Section 2.3) is A G B^T, so the
    B_k* of eq. (13), (15) is read as B_k^T; SVD precoders satisfy
    V = conj(B_k) V~ (Section 3.3) and a wideband precoder P_k is carried into
    the compressed domain as P~_k = B_k^T P_k;
  * the precoder of eq. (7) holds the top-L *right* singular vectors (the
    text after eq. 11 says "left"; right is what makes B cancel);
  * the compressed filter of eq. (27) is W~ = Q~^{-1} H~_ii V~_i (its
    printed parentheses are garbled);
  * "MMSE SINR" (sinr_mmse) uses a caller-given wideband precoder; "SVD SINR"
    (sinr_svd) uses eq. (7) on every serving link.

Array shapes: X (J, J, M, N, P); G (J, J, m, n, p); C (J, J, P, p);
coefficients (J, J, K, P); sigma2 (J,); SINR (J, K, L), index (UE i,
subcarrier kappa, stream r).
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------ channel rebuild, a0-a2
def coefficients(alpha: np.ndarray, tau: np.ndarray, K: int, delta_f: float) -> np.ndarray:
    """c(kappa) per path: conj(alpha_p exp(-j 2 pi kappa df tau_p)); shape (..., K, P)."""
    kap = np.arange(K, dtype=np.float64)
    phase = -2.0 * np.pi * kap[:, None] * delta_f * tau[..., None, :]
    return np.conj(alpha[..., None, :] * np.exp(1j * phase))


def dense_channel(Xik: np.ndarray, c: np.ndarray) -> np.ndarray:
    """eq. (9): H(kappa) = X x_3 c(kappa)* = sum_p conj(c_p) X[:, :, p]; (K, M, N)."""
    return np.tensordot(np.conj(c), Xik, axes=([1], [2]))


def projected_coefficients(Cik: np.ndarray, c: np.ndarray) -> np.ndarray:
    """The row vector c* C of eq. (15) for every subcarrier; (K, p)."""
    return np.conj(c) @ Cik


def compressed_channel(Gik: np.ndarray, Cik: np.ndarray, c: np.ndarray) -> np.ndarray:
    """eq. (15): H~(kappa) = G x_3 (c(kappa)* C); (K, m, n)."""
    w = projected_coefficients(Cik, c)
    return np.tensordot(w, Gik, axes=([1], [2]))


# ------------------------------------------------------------- precoders, a3
def svd_precoder(H: np.ndarray, L: int) -> np.ndarray:
    """eq. (7) / eq. (23): top-L right singular vectors of each H(kappa); (K, cols, L)."""
    _, _, Vh = np.linalg.svd(H, full_matrices=False)
    return np.conj(np.swapaxes(Vh[:, :L, :], 1, 2))


def project_precoder(Bk: np.ndarray, Pk: np.ndarray) -> np.ndarray:
    """Wideband precoder carried into the compressed domain: P~ = B^T P (n x L)."""
    return Bk.T @ Pk


# ---------------------------------------------------- covariance and SINR, a4-a6
def effective_channels(Hs: np.ndarray, V: np.ndarray) -> np.ndarray:
    """E[i, k](kappa) = H_ik(kappa) V_k(kappa); Hs (J, J, K, r, c), V (J, K, c, L)."""
    J = Hs.shape[0]
    return np.stack([np.stack([Hs[i, k] @ V[k] for k in range(J)]) for i in range(J)])


def covariance(E: np.ndarray, sigma2: np.ndarray) -> np.ndarray:
    """eq. (4) / eq. (25): Q_i = sum_k E_ik E_ik* + sigma_i^2 I; (J, K, r, r)."""
    J, _, K, r, _ = E.shape
    Q = np.zeros((J, K, r, r), dtype=np.complex128)
    for i in range(J):
        for k in range(J):
            Q[i] += E[i, k] @ np.conj(np.swapaxes(E[i, k], 1, 2))
        Q[i] += sigma2[i] * np.eye(r)[None]
    return Q


def sinr_literal(E: np.ndarray, sigma2: np.ndarray) -> np.ndarray:
    """eq. (3), (5), (6) as printed: W = Q^{-1} E_ii, s_r = |w_r* e_r|^2,
    SINR_r = s_r / (w_r* Q w_r - s_r).  Returns (J, K, L)."""
    J = E.shape[0]
    Q = covariance(E, sigma2)
    out = []
    for i in range(J):
        Eii = E[i, i]
        W = np.linalg.solve(Q[i], Eii)                                     # eq. (3)
        s = np.abs(np.einsum("kar,kar->kr", np.conj(W), Eii)) ** 2          # eq. (6)
        wQw = np.real(np.einsum("kar,kab,kbr->kr", np.conj(W), Q[i], W))
        out.append(s / (wQw - s))                                           # eq. (5)
    return np.stack(out)


def _trsm_lower(Lf: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Solve L X = Y for lower-triangular L (stacked), by forward substitution."""
    n = Lf.shape[-1]
    X = np.zeros(np.broadcast_shapes(Y.shape), dtype=np.complex128)
    for a in range(n):
        X[..., a, :] = (Y[..., a, :] - np.einsum("kb,kbr->kr", Lf[..., a, :a], X[..., :a, :])) \
            / Lf[..., a, a][..., None]
    return X


def sinr_stable(E: np.ndarray, sigma2: np.ndarray) -> np.ndarray:
    """The same SINR as eq. (5), arranged without cancellation.

    With R = Q_i - E_ii E_ii* (interference plus noise), Z = chol(R)^{-1} E_ii:
      x_r = [(I + Z*Z)^{-1}]_rr   (sum of squares of column r of chol(I+Z*Z)^{-1})
      a_r = z_r* (I + Z Z*)^{-1} z_r   (sum of squares of chol(I+ZZ*)^{-1} z_r)
    and a_r + x_r = 1, SINR_r = a_r / x_r (= 1/[(I + E*R^{-1}E)^{-1}]_rr - 1).
    """
    J = E.shape[0]
    Q = covariance(E, sigma2)
    out = []
    for i in range(J):
        Eii = E[i, i]
        K, r, L = Eii.shape
        R = Q[i] - Eii @ np.conj(np.swapaxes(Eii, 1, 2))
        Z = _trsm_lower(np.linalg.cholesky(R), Eii)
        ZH = np.conj(np.swapaxes(Z, 1, 2))
        F = np.eye(L)[None] + ZH @ Z
        Finv_chol = _trsm_lower(np.linalg.cholesky(F), np.broadcast_to(np.eye(L), (K, L, L)).copy())
        x = np.sum(np.abs(Finv_chol) ** 2, axis=1)
        Gm = np.eye(r)[None] + Z @ ZH
        Y = _trsm_lower(np.linalg.cholesky(Gm), Z)
        a = np.sum(np.abs(Y) ** 2, axis=1)
        out.append(a / x)
    return np.stack(out)


# -------------------------------------------------------------- whole paths
def compressed_channels(G, C, coef) -> np.ndarray:
    """H~ for every link and subcarrier; (J, J, K, m, n)."""
    J = G.shape[0]
    return np.stack([np.stack([compressed_channel(G[i, k], C[i, k], coef[i, k])
                               for k in range(J)]) for i in range(J)])


def dense_channels(X, coef) -> np.ndarray:
    """H for every link and subcarrier; (J, J, K, M, N)."""
    J = X.shape[0]
    return np.stack([np.stack([dense_channel(X[i, k], coef[i, k]) for k in range(J)])
                     for i in range(J)])


def _precoders(Hs, L, precoder, Pw):
    J, K = Hs.shape[0], Hs.shape[2]
    if precoder == "svd":
        return np.stack([svd_precoder(Hs[k, k], L) for k in range(J)])
    if precoder == "mmse":
        return np.stack([np.broadcast_to(Pw[k], (K,) + Pw[k].shape) for k in range(J)])
    raise ValueError(precoder)


def sinr_from_channels(Hs, sigma2, L, precoder="svd", Pw=None, form="stable"):
    """SINR (J, K, L) from per-link channels Hs (J, J, K, rows, cols)."""
    V = _precoders(Hs, L, precoder, Pw)
    E = effective_channels(Hs, V)
    return (sinr_stable if form == "stable" else sinr_literal)(E, sigma2)


def tucker_sinr(G, C, coef, sigma2, L, precoder="svd", Pt=None, form="stable"):
    """Compressed SINR, eq. (15), (23)-(28).  Pt: (J, n, L) projected precoders (mmse)."""
    return sinr_from_channels(compressed_channels(G, C, coef), sigma2, L, precoder, Pt, form)


def dense_sinr(X, coef, sigma2, L, precoder="svd", Pfull=None, form="stable"):
    """Uncompressed SINR, eq. (3)-(9).  Pfull: (J, N, L) wideband precoders (mmse)."""
    return sinr_from_channels(dense_channels(X, coef), sigma2, L, precoder, Pfull, form)


# ---------------------------------------------- several UEs per cell (Section 4)
def sinr_from_channels_multiuser(Hs, sigma2, L, form="stable"):
    """SVD-precoded SINR with U UEs per cell, as in the paper's experiments
    (Section 4: only the first UE of every other cell causes inter-cell
    interference; no intra-cell interference).

    Hs (U, J, J, K, rows, cols): Hs[u, i, k] is the channel from BS k to UE u
    of cell i; sigma2 (U, J).  UE (i, u) is served by BS i with the top-L
    right singular vectors of its own link Hs[u, i, i] (eq. 7); every other
    BS k transmits to its first UE, with the precoder of Hs[0, k, k].
    Returns (U, J, K, L)."""
    U, J = Hs.shape[:2]
    V0 = np.stack([svd_precoder(Hs[0, k, k], L) for k in range(J)])
    out = []
    for u in range(U):
        Vu = V0 if u == 0 else np.stack([svd_precoder(Hs[u, k, k], L) for k in range(J)])
        E = np.stack([np.stack([Hs[u, i, k] @ (Vu[k] if k == i else V0[k]) for k in range(J)])
                      for i in range(J)])
        out.append((sinr_stable if form == "stable" else sinr_literal)(E, sigma2[u]))
    return np.stack(out)


def tucker_sinr_multiuser(G, C, coef, sigma2, L, form="stable"):
    """Compressed form of sinr_from_channels_multiuser: G (U, J, J, m, n, p),
    C (U, J, J, P, p), coef (U, J, J, K, P), sigma2 (U, J)."""
    Hs = np.stack([compressed_channels(G[u], C[u], coef[u]) for u in range(G.shape[0])])
    return sinr_from_channels_multiuser(Hs, sigma2, L, form)


def dense_sinr_multiuser(X, coef, sigma2, L, form="stable"):
    """Dense form: X (U, J, J, M, N, P)."""
    Hs = np.stack([dense_channels(X[u], coef[u]) for u in range(X.shape[0])])
    return sinr_from_channels_multiuser(Hs, sigma2, L, form)


# -------------------------------------------------------------------- eq. 30
def mean_relative_error(sinr_ref: np.ndarray, sinr_cmp: np.ndarray) -> float:
    """e_c of eq. (30): mean over streams, UEs (and subcarriers) of |S - S~| / S."""
    return float(np.mean(np.abs((sinr_ref - sinr_cmp) / sinr_ref)))
