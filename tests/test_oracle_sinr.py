"""Pins of the oracle's SINR paths (no GPU).

Closed forms (diagonal channels, single cell, SVD precoding without
interference), brute force with explicit 2x2 inverses, the FFT form of the
subcarrier response, factor cancellation between the dense path on the
reconstructed channels and the compressed path (Section 3.3), and gauge
invariance of the compressed path.
"""
import numpy as np
import pytest

from oracle import sinr as S
from oracle import tucker as T
from paper_2401_09792_gb300 import synth


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(rng, r, c):
    Q, _ = np.linalg.qr(_rand(rng, (r, c)))
    return Q


def test_coefficients_match_fft_of_sampled_impulse_response():
    # with delays on the sample grid tau_p = t_p / (K df), the channel of
    # eq. (9) is the K-point DFT of the impulse response sum_p alpha_p X_p delta[t - t_p]
    rng = np.random.default_rng(0)
    K, df, P, M, N = 16, 15e3, 4, 2, 3
    taps = np.array([0, 3, 5, 11])
    tau = taps / (K * df)
    alpha = _rand(rng, P)
    X = _rand(rng, (M, N, P))
    c = S.coefficients(alpha, tau, K, df)
    H = S.dense_channel(X, c)
    h = np.zeros((K, M, N), dtype=complex)
    for q in range(P):
        h[taps[q]] += alpha[q] * X[:, :, q]
    np.testing.assert_allclose(H, np.fft.fft(h, axis=0), atol=1e-12)


def test_compressed_channel_is_mode3_product():
    # eq. (15): H~ = G x_3 (c* C), with x_3 taken from the tensor definitions
    rng = np.random.default_rng(1)
    G, C, c = _rand(rng, (3, 4, 2)), _rand(rng, (5, 2)), _rand(rng, (7, 5))
    Ht = S.compressed_channel(G, C, c)
    for x in range(7):
        row = (np.conj(c[x])[None, :] @ C)                       # 1 x p
        ref = T.mode_product(G, row, 2)[:, :, 0]
        np.testing.assert_allclose(Ht[x], ref, atol=1e-12)


def _diag_system(d, J=2, N=5, L=2):
    """X_ii = [diag(d) 0] on path 0 (c = 1), X_ik = 0 for i != k."""
    M = len(d)
    X = np.zeros((J, J, M, N, 1), dtype=complex)
    for i in range(J):
        X[i, i, :, :M, 0] = np.diag(d * (i + 1))
    coef = np.ones((J, J, 1, 1), dtype=complex)
    return X, coef


@pytest.mark.parametrize("form", ["stable", "literal"])
def test_diagonal_channel_closed_form(form):
    d = np.array([3.0 + 1j, 2.0, 0.5j])
    J, N, L, s2 = 2, 5, 2, np.array([0.1, 0.7])
    X, coef = _diag_system(d, J, N, L)
    # wideband precoder e_1..e_L: SINR_r = |d_r|^2 / sigma^2
    Pw = np.stack([np.eye(N)[:, :L]] * J)
    got = S.dense_sinr(X, coef, s2, L, "mmse", Pw, form)
    for i in range(J):
        np.testing.assert_allclose(got[i, 0], np.abs(d[:L] * (i + 1)) ** 2 / s2[i], rtol=1e-12)
    # SVD precoder picks the largest |d_r| first
    got = S.dense_sinr(X, coef, s2, L, "svd", None, form)
    ds = np.sort(np.abs(d))[::-1][:L]
    for i in range(J):
        np.testing.assert_allclose(got[i, 0], (ds * (i + 1)) ** 2 / s2[i], rtol=1e-12)


def test_single_cell_identity_and_forms():
    # no interference: SINR_r = 1/[(I + E*E/sigma^2)^{-1}]_rr - 1
    rng = np.random.default_rng(2)
    for M, L in ((4, 2), (3, 3), (6, 1)):
        E = _rand(rng, (1, 1, 5, M, L))
        s2 = np.array([0.3])
        lit = S.sinr_literal(E, s2)
        stb = S.sinr_stable(E, s2)
        ident = np.stack([1.0 / np.real(np.diag(np.linalg.inv(np.eye(L) + E[0, 0, x].conj().T
                                                              @ E[0, 0, x] / s2[0]))) - 1.0
                          for x in range(5)])
        np.testing.assert_allclose(lit[0], ident, rtol=1e-12)
        np.testing.assert_allclose(stb[0], ident, rtol=1e-12)


def test_svd_single_cell_is_singular_values_over_noise():
    # eq. (7) without interference: SINR_r = sigma_r(H)^2 / sigma^2
    rng = np.random.default_rng(3)
    M, N, L = 4, 7, 3
    X = _rand(rng, (1, 1, M, N, 2))
    coef = _rand(rng, (1, 1, 6, 2))
    s2 = np.array([0.05])
    got = S.dense_sinr(X, coef, s2, L, "svd")
    H = S.dense_channel(X[0, 0], coef[0, 0])
    sv = np.linalg.svd(H, compute_uv=False)[:, :L]
    np.testing.assert_allclose(got[0], sv ** 2 / s2[0], rtol=1e-11)


def test_brute_force_two_cells_2x2():
    # M = N = 2, L = 1, J = 2: every step written with scalars and the 2x2 adjugate
    rng = np.random.default_rng(4)
    X = _rand(rng, (2, 2, 2, 2, 1))
    coef = np.ones((2, 2, 1, 1), dtype=complex)
    s2 = np.array([0.2, 0.4])
    p = [np.array([1.0, 1j]) / np.sqrt(2), np.array([1.0, -1.0]) / np.sqrt(2)]
    Pw = np.stack([pp[:, None] for pp in p])
    got = S.dense_sinr(X, coef, s2, 1, "mmse", Pw, "literal")
    got_s = S.dense_sinr(X, coef, s2, 1, "mmse", Pw, "stable")
    for i in range(2):
        h = [X[i, k, :, :, 0] @ p[k] for k in range(2)]
        Q = np.zeros((2, 2), dtype=complex)
        for k in range(2):
            for a in range(2):
                for b in range(2):
                    Q[a, b] += h[k][a] * np.conj(h[k][b])
        Q[0, 0] += s2[i]
        Q[1, 1] += s2[i]
        det = Q[0, 0] * Q[1, 1] - Q[0, 1] * Q[1, 0]
        Qinv = np.array([[Q[1, 1], -Q[0, 1]], [-Q[1, 0], Q[0, 0]]]) / det
        w = Qinv @ h[i]
        s = abs(np.conj(w[0]) * h[i][0] + np.conj(w[1]) * h[i][1]) ** 2
        den = np.real(np.conj(w) @ Q @ w) - s
        assert abs(got[i, 0, 0] - s / den) < 1e-12 * (s / den)
        assert abs(got_s[i, 0, 0] - s / den) < 1e-12 * (s / den)


def _tucker_system(seed, J=3, M=4, N=10, P=6, m=3, n=5, p=4, K=5, L=2):
    rng = np.random.default_rng(seed)
    A = np.stack([_orth(rng, M, m) for _ in range(J)])
    B = np.stack([_orth(rng, N, n) for _ in range(J)])
    C = np.stack([[_orth(rng, P, p) for _ in range(J)] for _ in range(J)])
    G = _rand(rng, (J, J, m, n, p))
    coef = _rand(rng, (J, J, K, P))
    s2 = rng.uniform(0.05, 1.0, J)
    Pw = np.stack([_orth(rng, N, L) for _ in range(J)])
    return A, B, C, G, coef, s2, Pw


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_factor_cancellation(precoder):
    # Section 3.3: SINR of the dense path on X^ = G x_1 A x_2 B x_3 C equals the
    # compressed path on (G, C) -- A and B cancel
    A, B, C, G, coef, s2, Pw = _tucker_system(5)
    J, L = G.shape[0], Pw.shape[2]
    Xh = np.stack([np.stack([T.tucker_reconstruct(G[i, k], A[i], B[k], C[i, k])
                             for k in range(J)]) for i in range(J)])
    dense = S.dense_sinr(Xh, coef, s2, L, precoder, Pw)
    Pt = np.stack([S.project_precoder(B[k], Pw[k]) for k in range(J)])
    comp = S.tucker_sinr(G, C, coef, s2, L, precoder, Pt)
    np.testing.assert_allclose(comp, dense, rtol=1e-10)


def test_literal_equals_stable_with_interference():
    A, B, C, G, coef, s2, Pw = _tucker_system(6, J=4, m=4, L=3)
    for pre in ("svd", "mmse"):
        Pt = np.stack([S.project_precoder(B[k], Pw[k]) for k in range(4)]) if pre == "mmse" else None
        if pre == "mmse":
            Pt = np.stack([_orth(np.random.default_rng(k), 5, 3) for k in range(4)])
        lit = S.tucker_sinr(G, C, coef, s2, 3, pre, Pt, "literal")
        stb = S.tucker_sinr(G, C, coef, s2, 3, pre, Pt, "stable")
        np.testing.assert_allclose(stb, lit, rtol=1e-10)


def test_gauge_invariance_of_compressed_path():
    # C -> C W with G -> G x_3 W*, G -> G x_1 U and G -> G x_2 V (U, V, W unitary)
    # leave the SVD-precoded SINR unchanged
    rng = np.random.default_rng(7)
    A, B, C, G, coef, s2, Pw = _tucker_system(7)
    J, m, n, p = G.shape[0], G.shape[2], G.shape[3], G.shape[4]
    base = S.tucker_sinr(G, C, coef, s2, 2, "svd")
    G2, C2 = G.copy(), C.copy()
    for i in range(J):
        U = _orth(rng, m, m)
        for k in range(J):
            W = _orth(rng, p, p)
            C2[i, k] = C[i, k] @ W
            G2[i, k] = T.mode_product(T.mode_product(G[i, k], U, 0), W.conj().T, 2)
    for k in range(J):
        V = _orth(rng, n, n)
        for i in range(J):
            G2[i, k] = T.mode_product(G2[i, k], V, 1)
    np.testing.assert_allclose(S.tucker_sinr(G2, C2, coef, s2, 2, "svd"), base, rtol=1e-9)


def test_mean_relative_error_definition():
    a = np.array([1.0, 2.0, 4.0])
    assert S.mean_relative_error(a, a) == 0.0
    assert abs(S.mean_relative_error(a, 1.1 * a) - 0.1) < 1e-15


def test_small_workload_end_to_end_fit_then_sinr():
    # the small workload through the whole oracle: fit (Algorithm 2), then
    # compressed SINR vs dense SINR on the same channels; e_c is finite
    w = synth.SMALL
    X = synth.channel_submatrices(w)
    alpha, tau = synth.path_gains_delays(w)
    coef = S.coefficients(alpha, tau, w.K, w.delta_f_hz)
    s2 = synth.noise_powers(w)
    fit = T.fit_groupwise(X, (w.m, w.n, w.p), S=3)
    comp = S.tucker_sinr(fit["G"], fit["C"], coef, s2, w.L, "svd")
    dense = S.dense_sinr(X, coef, s2, w.L, "svd")
    assert comp.shape == dense.shape == (w.J, w.K, w.L)
    assert np.all(comp > 0) and np.all(dense > 0)
    assert np.isfinite(S.mean_relative_error(dense, comp))


# --------------------------------------------- several UEs per cell (Section 4)
def _multiuser_system(seed, U=3, J=3, M=4, N=10, P=6, m=3, n=5, p=4, K=4, L=2):
    rng = np.random.default_rng(seed)
    A = np.stack([[_orth(rng, M, m) for _ in range(J)] for _ in range(U)])      # per UE
    B = np.stack([_orth(rng, N, n) for _ in range(J)])                          # per BS
    C = np.stack([[[_orth(rng, P, p) for _ in range(J)] for _ in range(J)] for _ in range(U)])
    G = _rand(rng, (U, J, J, m, n, p))
    coef = _rand(rng, (U, J, J, K, P))
    s2 = rng.uniform(0.05, 1.0, (U, J))
    return A, B, C, G, coef, s2


def test_multiuser_first_group_is_the_single_ue_system():
    A, B, C, G, coef, s2 = _multiuser_system(11)
    got = S.tucker_sinr_multiuser(G, C, coef, s2, 2)
    np.testing.assert_allclose(got[0], S.tucker_sinr(G[0], C[0], coef[0], s2[0], 2, "svd"), rtol=1e-12)


def test_multiuser_interference_comes_from_the_first_ues_precoders():
    # UE (i, 1) with UE (i, 0)'s links and noise has UE (i, 0)'s SINR; the
    # serving link of UE (k, 1) changes no other UE's SINR (BS k interferes
    # with its first UE's precoder), while that of UE (k, 0) does
    A, B, C, G, coef, s2 = _multiuser_system(12)
    G[1], C[1], coef[1], s2[1] = G[0], C[0], coef[0], s2[0]
    base = S.tucker_sinr_multiuser(G, C, coef, s2, 2)
    np.testing.assert_allclose(base[1], base[0], rtol=1e-12)
    rng = np.random.default_rng(3)
    G1 = G.copy()
    G1[1, 2, 2] = _rand(rng, G1[1, 2, 2].shape)
    moved = S.tucker_sinr_multiuser(G1, C, coef, s2, 2)
    np.testing.assert_allclose(moved[0], base[0], rtol=1e-12)
    np.testing.assert_allclose(moved[1, :2], base[1, :2], rtol=1e-12)
    assert np.max(np.abs(moved[1, 2] - base[1, 2]) / base[1, 2]) > 1e-3
    G0 = G.copy()
    G0[0, 2, 2] = _rand(rng, G0[0, 2, 2].shape)
    moved0 = S.tucker_sinr_multiuser(G0, C, coef, s2, 2)
    assert np.max(np.abs(moved0[2, :2] - base[2, :2]) / base[2, :2]) > 1e-3


def test_multiuser_literal_equals_stable_and_brute_force():
    A, B, C, G, coef, s2 = _multiuser_system(13, U=2, J=2, m=2, n=2, p=2, L=1)
    lit = S.tucker_sinr_multiuser(G, C, coef, s2, 1, "literal")
    stb = S.tucker_sinr_multiuser(G, C, coef, s2, 1, "stable")
    np.testing.assert_allclose(stb, lit, rtol=1e-10)
    # UE (0, 1), subcarrier 0, by hand: 2 x 2 channels, rank-one precoders
    H = lambda u, i, k: S.compressed_channel(G[u, i, k], C[u, i, k], coef[u, i, k])[0]  # noqa: E731
    top = lambda M_: np.linalg.svd(M_)[2][0].conj()                                    # noqa: E731
    h_s = H(1, 0, 0) @ top(H(1, 0, 0))
    h_i = H(1, 0, 1) @ top(H(0, 1, 1))
    Q = np.outer(h_s, h_s.conj()) + np.outer(h_i, h_i.conj()) + s2[1, 0] * np.eye(2)
    w = np.linalg.inv(Q) @ h_s
    s = abs(w.conj() @ h_s) ** 2
    assert abs(stb[1, 0, 0, 0] - s / (np.real(w.conj() @ Q @ w) - s)) < 1e-10 * stb[1, 0, 0, 0]


def test_multiuser_factor_cancellation():
    # A per UE, B per BS: the dense path on X^ equals the compressed path
    A, B, C, G, coef, s2 = _multiuser_system(14)
    U, J = G.shape[:2]
    Xh = np.stack([np.stack([np.stack([T.tucker_reconstruct(G[u, i, k], A[u, i], B[k], C[u, i, k])
                                       for k in range(J)]) for i in range(J)]) for u in range(U)])
    np.testing.assert_allclose(S.tucker_sinr_multiuser(G, C, coef, s2, 2),
                               S.dense_sinr_multiuser(Xh, coef, s2, 2), rtol=1e-10)
