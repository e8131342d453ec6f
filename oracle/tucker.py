"""Tensor algebra, HOSVD and the groupwise Tucker fit -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (Section 2.3 of the paper):
  * inner product <X, Y> = sum x * conj(y); norm ||X|| = sqrt(<X, X>);
  * mode-n unfolding X_(n): the mode-n fibres become columns, the remaining
    indices ordered with the earliest one fastest (the paper's
    [X_(1)]_{i1, i2 + I2 (i3 - 1)} = X_{i1 i2 i3});
  * mode-n product (X x_n U)_{.. j ..} = sum_{i_n} x_{.. i_n ..} u_{j, i_n},
    equivalently (X x_n U)_(n) = U X_(n);
  * "principal eigenvectors" are those of the largest eigenvalues, returned in
    descending eigenvalue order with the phase of each column fixed so that
    its largest-modulus entry is real and positive.

Groupwise model (eq. 14) with one UE per cell: channel (i, k) from BS k to the
UE of cell i, X[i, k] in C^{M x N x P};  A[i] (M x m) is shared by all links
into UE i, B[k] (N x n) by all links out of BS k, C[i, k] (P x p) and
G[i, k] (m x n x p) belong to one link.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- Section 2.3
def inner(X: np.ndarray, Y: np.ndarray) -> complex:
    """<X, Y> = sum x conj(y)."""
    return complex(np.sum(X * np.conj(Y)))


def fro2(X: np.ndarray) -> float:
    """||X||^2."""
    return float(np.real(np.sum(X * np.conj(X))))


def unfold(X: np.ndarray, mode: int) -> np.ndarray:
    """Mode-`mode` (0-based) unfolding X_(mode+1), earliest remaining index fastest."""
    Xm = np.moveaxis(X, mode, 0)
    return np.reshape(Xm, (Xm.shape[0], -1), order="F")


def fold(Y: np.ndarray, mode: int, shape: tuple) -> np.ndarray:
    """Inverse of `unfold` for a tensor of the given shape."""
    rest = [s for d, s in enumerate(shape) if d != mode]
    Xm = np.reshape(Y, [shape[mode]] + rest, order="F")
    return np.moveaxis(Xm, 0, mode)


def mode_product(X: np.ndarray, U: np.ndarray, mode: int) -> np.ndarray:
    """X x_mode U, written as the unfolding identity (X x_n U)_(n) = U X_(n)."""
    shape = list(X.shape)
    Y = U @ unfold(X, mode)
    shape[mode] = U.shape[0]
    return fold(Y, mode, tuple(shape))


def tucker_reconstruct(G, A, B, C) -> np.ndarray:
    """G x_1 A x_2 B x_3 C."""
    return mode_product(mode_product(mode_product(G, A, 0), B, 1), C, 2)


def principal_eigvecs(S: np.ndarray, r: int) -> np.ndarray:
    """r principal eigenvectors of the Hermitian matrix S (descending order)."""
    w, V = np.linalg.eigh(S)
    order = np.argsort(w)[::-1][:r]
    return _fix_phase(V[:, order])


def leading_left_singular_vectors(Y: np.ndarray, r: int) -> np.ndarray:
    """r leading left singular vectors of Y (Algorithm 1, each step)."""
    U, _, _ = np.linalg.svd(Y, full_matrices=False)
    if U.shape[1] < r:    # Y has fewer columns than r: complete with eigvecs of Y Y*
        return principal_eigvecs(Y @ Y.conj().T, r)
    return _fix_phase(U[:, :r])


def _fix_phase(V: np.ndarray) -> np.ndarray:
    V = V.copy()
    for j in range(V.shape[1]):
        t = np.argmax(np.abs(V[:, j]))
        if abs(V[t, j]) > 0:
            V[:, j] *= np.conj(V[t, j]) / abs(V[t, j])
    return V


# ------------------------------------------------------------- Algorithm 1
def hosvd(X: np.ndarray, ranks: tuple) -> tuple:
    """HOSVD (Algorithm 1): leading left singular vectors of each unfolding,
    then G = X x_1 A* x_2 B* x_3 C*.  Returns (G, A, B, C)."""
    A = leading_left_singular_vectors(unfold(X, 0), ranks[0])
    B = leading_left_singular_vectors(unfold(X, 1), ranks[1])
    C = leading_left_singular_vectors(unfold(X, 2), ranks[2])
    return core(X, A, B, C), A, B, C


# -------------------------------------------------- groupwise model, eq. 14-22
def core(X, A, B, C) -> np.ndarray:
    """Optimal core for fixed orthonormal factors, eq. (17)."""
    H = lambda U: U.conj().T  # noqa: E731
    return mode_product(mode_product(mode_product(X, H(A), 0), H(B), 1), H(C), 2)


def objective_g(X, A, B, C) -> float:
    """g of eq. (18)-(19): sum over links of ||X x_1 A_i* x_2 B_k* x_3 C_ik*||^2."""
    J = X.shape[0]
    return sum(fro2(core(X[i, k], A[i], B[k], C[i, k])) for i in range(J) for k in range(J))


def objective_f(X, A, B, C, G) -> float:
    """f of eq. (16): sum of squared reconstruction errors."""
    J = X.shape[0]
    return sum(fro2(X[i, k] - tucker_reconstruct(G[i, k], A[i], B[k], C[i, k]))
               for i in range(J) for k in range(J))


def _M1(Xik, Bk, Cik):
    """1M of eq. (20): (X x_2 B_k* x_3 C_ik*)_(1)."""
    return unfold(mode_product(mode_product(Xik, Bk.conj().T, 1), Cik.conj().T, 2), 0)


def _M2(Xik, Ai, Cik):
    """2M of eq. (21): (X x_1 A_i* x_3 C_ik*)_(2)."""
    return unfold(mode_product(mode_product(Xik, Ai.conj().T, 0), Cik.conj().T, 2), 1)


def _M3(Xik, Ai, Bk):
    """3M of eq. (22): (X x_1 A_i* x_2 B_k*)_(3)."""
    return unfold(mode_product(mode_product(Xik, Ai.conj().T, 0), Bk.conj().T, 1), 2)


def update_A(X, B, C, m) -> np.ndarray:
    """eq. (20): A_i = m principal eigenvectors of sum_k 1M 1M*."""
    J = X.shape[0]
    out = []
    for i in range(J):
        S = sum(_M1(X[i, k], B[k], C[i, k]) @ _M1(X[i, k], B[k], C[i, k]).conj().T
                for k in range(J))
        out.append(principal_eigvecs(S, m))
    return np.stack(out)


def update_B(X, A, C, n) -> np.ndarray:
    """eq. (21): B_k = n principal eigenvectors of sum_i 2M 2M*."""
    J = X.shape[0]
    out = []
    for k in range(J):
        S = sum(_M2(X[i, k], A[i], C[i, k]) @ _M2(X[i, k], A[i], C[i, k]).conj().T
                for i in range(J))
        out.append(principal_eigvecs(S, n))
    return np.stack(out)


def update_C(X, A, B, p) -> np.ndarray:
    """eq. (22): C_ik = p principal eigenvectors of 3M 3M*."""
    J = X.shape[0]
    C = np.empty((J, J, X.shape[4], p), dtype=np.complex128)
    for i in range(J):
        for k in range(J):
            M3 = _M3(X[i, k], A[i], B[k])
            C[i, k] = principal_eigvecs(M3 @ M3.conj().T, p)
    return C


def hosvd_init(X, ranks) -> tuple:
    """Initialisation of Algorithm 2 (Section 3.2).

    Reading: the singular vectors of the unfoldings, with the shared factors
    taken over every link that shares them -- A_i from sum_k X_(1) X_(1)*,
    B_k from sum_i X_(2) X_(2)*, C_ik from X_(3) of its own link.  This is
    eq. (20)-(22) with the other two factors set to the identity.
    """
    m, n, p = ranks
    J = X.shape[0]
    A = np.stack([principal_eigvecs(sum(unfold(X[i, k], 0) @ unfold(X[i, k], 0).conj().T
                                        for k in range(J)), m) for i in range(J)])
    B = np.stack([principal_eigvecs(sum(unfold(X[i, k], 1) @ unfold(X[i, k], 1).conj().T
                                        for i in range(J)), n) for k in range(J)])
    C = np.empty((J, J, X.shape[4], p), dtype=np.complex128)
    for i in range(J):
        for k in range(J):
            X3 = unfold(X[i, k], 2)
            C[i, k] = principal_eigvecs(X3 @ X3.conj().T, p)
    return A, B, C


def fit_groupwise(X: np.ndarray, ranks: tuple, S: int = 10, init=None,
                  history: bool = False):
    """Groupwise Tucker compression, Algorithm 2.

    X: (J, J, M, N, P).  S Gauss-Seidel sweeps: all A_i (eq. 20) with the
    previous B, C; then all B_k (eq. 21) with the new A; then all C_ik
    (eq. 22) with the new A, B.  The core (eq. 17) is formed once at the end.

    Returns dict(A, B, C, G, g) where g lists the objective of eq. (19) after
    the initialisation and after every block update (3 per sweep) when
    `history` is set, else only the final value.
    """
    m, n, p = ranks
    A, B, C = hosvd_init(X, ranks) if init is None else init
    g = [objective_g(X, A, B, C)] if history else []
    for _ in range(S):
        A = update_A(X, B, C, m)
        if history:
            g.append(objective_g(X, A, B, C))
        B = update_B(X, A, C, n)
        if history:
            g.append(objective_g(X, A, B, C))
        C = update_C(X, A, B, p)
        if history:
            g.append(objective_g(X, A, B, C))
    J = X.shape[0]
    G = np.empty((J, J, m, n, p), dtype=np.complex128)
    for i in range(J):
        for k in range(J):
            G[i, k] = core(X[i, k], A[i], B[k], C[i, k])
    if not history:
        g = [sum(fro2(G[i, k]) for i in range(J) for k in range(J))]
    return {"A": A, "B": B, "C": C, "G": G, "g": np.array(g)}


# ------------------------------------------- the three models of Section 3.1
# Which factor a link (i, k) uses: groupwise (eq. 14) A_i and B_k; shared
# (eq. 12) one A and one B for every link; individual (eq. 10) A_ik and
# B_ik of its own.  C_ik and G_ik are per link in all three.
MODELS = ("groupwise", "shared", "individual")


def factor_groups(J: int, model: str):
    """(number of A factors, number of B factors, a(i, k), b(i, k))."""
    if model == "groupwise":
        return J, J, (lambda i, k: i), (lambda i, k: k)
    if model == "shared":
        return 1, 1, (lambda i, k: 0), (lambda i, k: 0)
    if model == "individual":
        return J * J, J * J, (lambda i, k: i * J + k), (lambda i, k: i * J + k)
    raise ValueError(model)


def fit_model(X: np.ndarray, ranks: tuple, model: str = "groupwise", S: int = 10,
              history: bool = False):
    """Algorithm 2 for any of the three models: every factor is the leading
    eigenvectors of the mode Gram summed over the links that share it
    (eq. 20-22 with the sums over the sharing links), initialised with the
    other two factors set to the identity, then S Gauss-Seidel sweeps (all A,
    all B, all C), and the core of eq. (17).  For the groupwise model this is
    fit_groupwise.  Returns dict(A, B, C, G, g) with A: (nA, M, m),
    B: (nB, N, n), C: (J, J, P, p), G: (J, J, m, n, p)."""
    m, n, p = ranks
    J = X.shape[0]
    nA, nB, ga, gb = factor_groups(J, model)
    links = [(i, k) for i in range(J) for k in range(J)]

    def gram_sum(group_of, g, M_of):
        return sum(M_of(i, k) @ M_of(i, k).conj().T for (i, k) in links if group_of(i, k) == g)

    A = np.stack([principal_eigvecs(gram_sum(ga, g, lambda i, k: unfold(X[i, k], 0)), m)
                  for g in range(nA)])
    B = np.stack([principal_eigvecs(gram_sum(gb, g, lambda i, k: unfold(X[i, k], 1)), n)
                  for g in range(nB)])
    C = np.empty((J, J, X.shape[4], p), dtype=np.complex128)
    for i, k in links:
        X3 = unfold(X[i, k], 2)
        C[i, k] = principal_eigvecs(X3 @ X3.conj().T, p)

    def g_now():
        return sum(fro2(core(X[i, k], A[ga(i, k)], B[gb(i, k)], C[i, k])) for i, k in links)

    g = [g_now()] if history else []
    for _ in range(S):
        A = np.stack([principal_eigvecs(gram_sum(ga, g_, lambda i, k: _M1(X[i, k], B[gb(i, k)], C[i, k])), m)
                      for g_ in range(nA)])
        if history:
            g.append(g_now())
        B = np.stack([principal_eigvecs(gram_sum(gb, g_, lambda i, k: _M2(X[i, k], A[ga(i, k)], C[i, k])), n)
                      for g_ in range(nB)])
        if history:
            g.append(g_now())
        for i, k in links:
            M3 = _M3(X[i, k], A[ga(i, k)], B[gb(i, k)])
            C[i, k] = principal_eigvecs(M3 @ M3.conj().T, p)
        if history:
            g.append(g_now())
    G = np.empty((J, J, m, n, p), dtype=np.complex128)
    for i, k in links:
        G[i, k] = core(X[i, k], A[ga(i, k)], B[gb(i, k)], C[i, k])
    if not history:
        g = [sum(fro2(G[i, k]) for i, k in links)]
    return {"A": A, "B": B, "C": C, "G": G, "g": np.array(g)}


def reconstruct_model(G, A, B, C, model: str) -> np.ndarray:
    """X^_ik = G_ik x_1 A x_2 B x_3 C_ik with the model's factor of each link:
    (J, J, M, N, P)."""
    J = G.shape[0]
    _, _, ga, gb = factor_groups(J, model)
    return np.stack([np.stack([tucker_reconstruct(G[i, k], A[ga(i, k)], B[gb(i, k)], C[i, k])
                               for k in range(J)]) for i in range(J)])


# ------------------------------------------------- Table (Section 3.3), eq. 29
def storage_original(J, K, M, N, P) -> int:
    """Complex entries of all channel tensors before compression (Table, Section 3.3)."""
    return J * J * K * M * N * P


def storage_groupwise(J, K, M, N, P, m, n, p) -> int:
    """Complex entries after groupwise compression (Table, Section 3.3)."""
    return J * J * K * (m * n * p + P * p) + J * K * M * m + J * N * n


def storage_shared(J, K, M, N, P, m, n, p) -> int:
    """Shared model (eq. 12): one A, one B, per-link C and G."""
    return J * J * K * (m * n * p + P * p) + M * m + N * n


def storage_individual(J, K, M, N, P, m, n, p) -> int:
    """Individual model (eq. 10): every link stores its own A, B, C and G."""
    return J * J * K * (m * n * p + M * m + N * n + P * p)


def storage_ratio(J, K, M, N, P, m, n, p, model: str = "groupwise") -> float:
    """R_s of eq. (29) (groupwise), and the same ratio for the other two models."""
    comp = {"groupwise": storage_groupwise, "shared": storage_shared,
            "individual": storage_individual}[model](J, K, M, N, P, m, n, p)
    return storage_original(J, K, M, N, P) / comp
