"""Pins of the oracle's tensor algebra and groupwise fit (no GPU).

Each test checks the oracle against something other than itself: the
elementwise definitions of Section 2.3 by brute-force loops, exact
reconstruction at full rank, the optimal-core identity of eq. (18), block
optimality of eq. (20)-(22), the Eckart-Young theorem through numpy's SVD,
and the storage ratios printed in Table 1.
"""
import os

import numpy as np
import pytest

from oracle import tucker as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(rng, r, c):
    Q, _ = np.linalg.qr(_rand(rng, (r, c)))
    return Q


def test_unfold_index_convention():
    # Section 2.3: [X_(1)]_{i1, i2 + I2 (i3 - 1)} = X_{i1 i2 i3} (1-based)
    rng = np.random.default_rng(0)
    X = _rand(rng, (3, 4, 5))
    X1 = T.unfold(X, 0)
    for i1 in range(3):
        for i2 in range(4):
            for i3 in range(5):
                assert X1[i1, i2 + 4 * i3] == X[i1, i2, i3]
    for mode in range(3):
        assert np.array_equal(T.fold(T.unfold(X, mode), mode, X.shape), X)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mode_product_elementwise(mode):
    # Section 2.3: (X x_n U)_{.. j ..} = sum_{i_n} x_{.. i_n ..} u_{j, i_n}
    rng = np.random.default_rng(1)
    X = _rand(rng, (3, 4, 5))
    U = _rand(rng, (2, X.shape[mode]))
    Y = T.mode_product(X, U, mode)
    ref = np.zeros(Y.shape, dtype=complex)
    for idx in np.ndindex(*Y.shape):
        j = idx[mode]
        for i in range(X.shape[mode]):
            src = list(idx)
            src[mode] = i
            ref[idx] += X[tuple(src)] * U[j, i]
    np.testing.assert_allclose(Y, ref, atol=1e-13)


def test_inner_and_norm_definitions():
    rng = np.random.default_rng(2)
    X, Y = _rand(rng, (2, 3, 2)), _rand(rng, (2, 3, 2))
    s = 0j
    for idx in np.ndindex(*X.shape):
        s += X[idx] * np.conj(Y[idx])
    assert abs(T.inner(X, Y) - s) < 1e-12
    assert abs(T.fro2(X) - np.linalg.norm(X.ravel()) ** 2) < 1e-10


def test_hosvd_full_rank_reconstructs_exactly():
    rng = np.random.default_rng(3)
    X = _rand(rng, (4, 6, 5))
    G, A, B, C = T.hosvd(X, X.shape)
    Xh = T.tucker_reconstruct(G, A, B, C)
    assert np.linalg.norm(X - Xh) / np.linalg.norm(X) < 1e-12


def test_hosvd_factors_are_leading_singular_vectors():
    # Algorithm 1: A spans the leading left singular subspace of X_(1)
    rng = np.random.default_rng(4)
    X = _rand(rng, (6, 7, 5))
    _, A, B, C = T.hosvd(X, (3, 4, 2))
    for F, mode in ((A, 0), (B, 1), (C, 2)):
        U, _, _ = np.linalg.svd(T.unfold(X, mode))
        r = F.shape[1]
        P1 = F @ F.conj().T
        P2 = U[:, :r] @ U[:, :r].conj().T
        assert np.linalg.norm(P1 - P2) < 1e-10


def _small_system(rng, J=2, M=4, N=6, P=5):
    return _rand(rng, (J, J, M, N, P))


def test_groupwise_fit_orthonormal_and_core_identity():
    rng = np.random.default_rng(5)
    X = _small_system(rng)
    fit = T.fit_groupwise(X, (2, 3, 3), S=4)
    J = X.shape[0]
    for i in range(J):
        assert np.linalg.norm(fit["A"][i].conj().T @ fit["A"][i] - np.eye(2)) < 1e-12
        assert np.linalg.norm(fit["B"][i].conj().T @ fit["B"][i] - np.eye(3)) < 1e-12
        for k in range(J):
            assert np.linalg.norm(fit["C"][i, k].conj().T @ fit["C"][i, k] - np.eye(3)) < 1e-12
    # eq. (18): f = ||X||^2 - g, with f computed by explicit reconstruction
    f = T.objective_f(X, fit["A"], fit["B"], fit["C"], fit["G"])
    g = sum(T.fro2(fit["G"][i, k]) for i in range(J) for k in range(J))
    assert abs(f - (T.fro2(X) - g)) < 1e-9 * T.fro2(X)


def test_groupwise_fit_full_rank_exact():
    rng = np.random.default_rng(6)
    X = _small_system(rng, J=2, M=3, N=4, P=3)
    fit = T.fit_groupwise(X, (3, 4, 3), S=1)
    f = T.objective_f(X, fit["A"], fit["B"], fit["C"], fit["G"])
    assert f < 1e-22 * T.fro2(X) + 1e-24


def test_g_non_decreasing_over_block_updates():
    # each block update of Algorithm 2 maximises g over that block exactly
    rng = np.random.default_rng(7)
    X = _small_system(rng, J=3, M=4, N=8, P=6)
    fit = T.fit_groupwise(X, (2, 3, 2), S=5, history=True)
    g = fit["g"]
    assert len(g) == 1 + 3 * 5
    assert np.all(np.diff(g) >= -1e-10 * g[0])
    assert g[-1] > g[0]


def test_block_update_is_a_maximiser():
    # eq. (20): the A update beats every other orthonormal A_i (random trials)
    rng = np.random.default_rng(8)
    X = _small_system(rng, J=2, M=5, N=6, P=4)
    A, B, C = T.hosvd_init(X, (2, 3, 2))
    A_new = T.update_A(X, B, C, 2)
    g_new = T.objective_g(X, A_new, B, C)
    for _ in range(20):
        A_try = A_new.copy()
        A_try[0] = _orth(rng, 5, 2)
        assert T.objective_g(X, A_try, B, C) <= g_new + 1e-10
    B_new = T.update_B(X, A_new, C, 3)
    g_b = T.objective_g(X, A_new, B_new, C)
    for _ in range(20):
        B_try = B_new.copy()
        B_try[1] = _orth(rng, 6, 3)
        assert T.objective_g(X, A_new, B_try, C) <= g_b + 1e-10
    C_new = T.update_C(X, A_new, B_new, 2)
    g_c = T.objective_g(X, A_new, B_new, C_new)
    for _ in range(20):
        C_try = C_new.copy()
        C_try[0, 1] = _orth(rng, 4, 2)
        assert T.objective_g(X, A_new, B_new, C_try) <= g_c + 1e-10


def test_single_link_single_path_is_eckart_young():
    # J = 1, P = p = 1: Algorithm 2 reduces to a truncated matrix SVD, so the
    # fit error is the sum of the discarded squared singular values
    rng = np.random.default_rng(9)
    Xm = _rand(rng, (6, 9))
    X = Xm[None, None, :, :, None]
    fit = T.fit_groupwise(X, (3, 3, 1), S=8)
    f = T.objective_f(X, fit["A"], fit["B"], fit["C"], fit["G"])
    s = np.linalg.svd(Xm, compute_uv=False)
    assert abs(f - np.sum(s[3:] ** 2)) < 1e-9 * np.sum(s ** 2)


def test_storage_ratio_table1():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_storage_ratio.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 12
    for model, J, M, N, P, K, m, n, p, rs in rows:
        got = T.storage_ratio(int(J), int(K), int(M), int(N), int(P), int(m), int(n), int(p), model)
        assert abs(got - float(rs)) < 1.5e-4, (model, got, rs)


# ------------------------------------------- shared and individual models
def _g_model(X, fit, model):
    J = X.shape[0]
    _, _, ga, gb = T.factor_groups(J, model)
    return sum(T.fro2(T.core(X[i, k], fit["A"][ga(i, k)], fit["B"][gb(i, k)], fit["C"][i, k]))
               for i in range(J) for k in range(J))


def test_model_fit_groupwise_is_algorithm_2():
    # the generic fit with groupwise groups reproduces fit_groupwise
    rng = np.random.default_rng(21)
    X = _small_system(rng, J=2, M=4, N=6, P=5)
    a = T.fit_model(X, (2, 3, 2), "groupwise", S=3, history=True)
    b = T.fit_groupwise(X, (2, 3, 2), S=3, history=True)
    np.testing.assert_allclose(a["g"], b["g"], rtol=1e-12)


def test_individual_init_is_hosvd_of_each_link():
    # individual model, no sweep: every link's factors are its own HOSVD
    # (Algorithm 1), whose subspaces come from numpy's SVD
    rng = np.random.default_rng(22)
    X = _small_system(rng, J=2, M=4, N=6, P=5)
    fit = T.fit_model(X, (2, 3, 2), "individual", S=0)
    for i in range(2):
        for k in range(2):
            _, A, B, C = T.hosvd(X[i, k], (2, 3, 2))
            proj = lambda F: F @ F.conj().T  # noqa: E731
            assert np.linalg.norm(proj(fit["A"][i * 2 + k]) - proj(A)) < 1e-9
            assert np.linalg.norm(proj(fit["B"][i * 2 + k]) - proj(B)) < 1e-9
            assert np.linalg.norm(proj(fit["C"][i, k]) - proj(C)) < 1e-9


@pytest.mark.parametrize("model", ["shared", "individual"])
def test_model_fit_identities(model):
    rng = np.random.default_rng(23)
    X = _small_system(rng, J=3, M=4, N=6, P=5)
    fit = T.fit_model(X, (2, 3, 2), model, S=4, history=True)
    g = fit["g"]
    # every block update maximises g over its block: non-decreasing
    assert np.all(np.diff(g) >= -1e-10 * g[0])
    # eq. (18) with the model's factors, by explicit reconstruction
    Xh = T.reconstruct_model(fit["G"], fit["A"], fit["B"], fit["C"], model)
    f = T.fro2(X - Xh)
    assert abs(f - (T.fro2(X) - g[-1])) < 1e-9 * T.fro2(X)
    assert abs(g[-1] - _g_model(X, fit, model)) < 1e-9 * g[-1]
    nA, nB, _, _ = T.factor_groups(3, model)
    assert fit["A"].shape == (nA, 4, 2) and fit["B"].shape == (nB, 6, 3)


def test_one_cell_models_coincide():
    # with one cell every model has one A, one B and one link: the same fit
    rng = np.random.default_rng(24)
    X = _small_system(rng, J=1, M=5, N=6, P=4)
    g = [T.fit_model(X, (2, 3, 2), mdl, S=3, history=True)["g"] for mdl in T.MODELS]
    np.testing.assert_allclose(g[1], g[0], rtol=1e-12)
    np.testing.assert_allclose(g[2], g[0], rtol=1e-12)


def test_model_storage_order_and_accuracy_order():
    # storage: shared < groupwise < individual entries (Table 1's R_s order);
    # fit quality: individual >= groupwise >= shared at full convergence of a
    # tiny system (more factors fit more)
    rng = np.random.default_rng(25)
    X = _small_system(rng, J=2, M=4, N=6, P=5)
    g = {mdl: T.fit_model(X, (2, 3, 2), mdl, S=20)["g"][-1] for mdl in T.MODELS}
    assert g["individual"] >= g["groupwise"] * (1 - 1e-9)
    assert g["groupwise"] >= g["shared"] * (1 - 1e-9)
    args = (2, 1, 4, 6, 5, 2, 3, 2)
    assert (T.storage_ratio(*args, model="shared") > T.storage_ratio(*args, model="groupwise")
            > T.storage_ratio(*args, model="individual"))
