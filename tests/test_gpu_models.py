"""The shared (eq. 12) and individual (eq. 10) compression models on the GPU,
against the FP64 oracle's Algorithm 2 for the same model.

Fit (ts_tucker_fit_model): the objective g after the initialisation and every
block update (relative 1e-8: all Grams of the small workload go through
Jacobi), factor subspaces, orthonormality and eq. (18) for the returned core.

Reconstruction (ts_tucker_reconstruct): X^ = G x_1 A x_2 B x_3 C with the
model's factor of each link, FP32, against the oracle's reconstruction from
the same factors (relative Frobenius error per link <= 1e-5).

SINR: the shared model's factors are common to every link, so they cancel as
the groupwise ones do (Section 3.3) and the compressed kernels evaluate it on
(G, C); the individual model's A_ik, B_ik differ between the links of one UE
and one BS, so its SINR is the dense path on the reconstructed channels.
Both are compared with the oracle on the same inputs, every SINR within
1e-5 relative (the FP32 bound of the single-model tests).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from oracle import tucker as T  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, assert_sinr_close  # noqa: E402

MODEL_ID = {"groupwise": ts.TS_MODEL_GROUPWISE, "shared": ts.TS_MODEL_SHARED,
            "individual": ts.TS_MODEL_INDIVIDUAL}
FIT_OP = {"groupwise": ts.TS_OP_TUCKER_FIT, "shared": ts.TS_OP_TUCKER_FIT_SHARED,
          "individual": ts.TS_OP_TUCKER_FIT_INDIVIDUAL}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


def _gpu_fit(X, ranks, S_, model, K=1, L=1):
    J, _, M, N, P = X.shape
    m, n, p = ranks
    nA, nB, _, _ = T.factor_groups(J, model)
    d = ts.Dims(J, M, N, P, m, n, p, K, L)
    Xd = ts.channels_to_device(X)
    dev = dict(dtype=torch.complex64, device="cuda")
    A = torch.empty(nA, M, m, **dev)
    B = torch.empty(nB, N, n, **dev)
    C = torch.empty(J * J, P, p, **dev)
    G = torch.empty(J * J, p, m, n, **dev)
    g = torch.empty(3 * S_ + 1, dtype=torch.float64, device="cuda")
    ws = ts.workspace(d, FIT_OP[model])
    ts.ts_tucker_fit_model(d, Xd, S_, 0, MODEL_ID[model], A, B, C, G, g, ws)
    torch.cuda.synchronize()
    return d, dict(A=A, B=B, C=C, G=G), g.cpu().numpy()


def _core_host(G, J, m, n, p):
    return np.transpose(_host(G).reshape(J, J, p, m, n), (0, 1, 3, 4, 2))


def _channels(w):
    return synth.channel_submatrices(w).astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("model", ["shared", "individual", "groupwise"])
def test_fit_model_matches_oracle(model):
    w = synth.SMALL
    X = _channels(w)
    ranks = (w.m, w.n, w.p)
    ref = T.fit_model(X, ranks, model, S=3, history=True)
    _, f, g = _gpu_fit(X, ranks, 3, model)
    np.testing.assert_allclose(g, ref["g"], rtol=1e-8)
    assert np.all(np.diff(g) >= -1e-9 * g[-1]), "g must not decrease over block updates"
    J = w.J
    proj = lambda F: F @ np.conj(np.swapaxes(F, -1, -2))  # noqa: E731
    C = _host(f["C"]).reshape(J, J, w.P, w.p)
    for got, want, r in ((_host(f["A"]), ref["A"], w.m), (_host(f["B"]), ref["B"], w.n), (C, ref["C"], w.p)):
        assert got.shape == want.shape
        assert np.max(np.abs(proj(got) - proj(want))) < 1e-4
        eye = np.conj(np.swapaxes(got, -1, -2)) @ got
        assert np.max(np.abs(eye - np.eye(r))) < 1e-5
    G = _core_host(f["G"], J, w.m, w.n, w.p)
    Xh = T.reconstruct_model(G, _host(f["A"]), _host(f["B"]), C, model)
    err = T.fro2(X - Xh)
    gG = T.fro2(G)
    assert abs(err - (T.fro2(X) - gG)) < 1e-5 * T.fro2(X)          # eq. (18)
    assert abs(gG - ref["g"][-1]) < 1e-5 * ref["g"][-1]


def test_model_ordering_of_the_objective():
    # individual factors are fitted per link, groupwise per UE/BS, shared once:
    # each model's feasible set contains the next one's, so the fitted energy
    # g = ||G||^2 orders individual >= groupwise >= shared (all from the same
    # initialisation family; checked on the GPU results)
    w = synth.SMALL
    X = _channels(w)
    ranks = (w.m, w.n, w.p)
    gs = {mdl: _gpu_fit(X, ranks, 4, mdl)[2][-1] for mdl in ("shared", "groupwise", "individual")}
    assert gs["individual"] >= gs["groupwise"] * (1 - 1e-9)
    assert gs["groupwise"] >= gs["shared"] * (1 - 1e-9)


@pytest.mark.parametrize("model", ["shared", "individual", "groupwise"])
def test_reconstruction_matches_oracle(model):
    w = dataclasses.replace(synth.SMALL, J=3)
    X = _channels(w)
    d, f, _ = _gpu_fit(X, (w.m, w.n, w.p), 2, model)
    J = w.J
    Xhat = torch.empty(J * J, w.P, w.M, w.N, dtype=torch.complex64, device="cuda")
    ws = ts.workspace(d, ts.TS_OP_RECONSTRUCT)
    ts.ts_tucker_reconstruct(d, MODEL_ID[model], f["A"], f["B"], f["C"], f["G"], Xhat, ws)
    torch.cuda.synchronize()
    got = np.transpose(_host(Xhat).reshape(J, J, w.P, w.M, w.N), (0, 1, 3, 4, 2))
    want = T.reconstruct_model(_core_host(f["G"], J, w.m, w.n, w.p), _host(f["A"]), _host(f["B"]),
                               _host(f["C"]).reshape(J, J, w.P, w.p), model)
    for i in range(J):
        for k in range(J):
            assert np.sqrt(T.fro2(got[i, k] - want[i, k]) / T.fro2(want[i, k])) < 1e-5


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_shared_model_sinr_through_compressed_kernels(precoder):
    w = dataclasses.replace(synth.SMALL, J=3, K=48)
    X = _channels(w)
    case = Case(w)
    d, f, _ = _gpu_fit(X, (w.m, w.n, w.p), 3, "shared", K=w.K, L=w.L)
    J = w.J
    # the shared fit's (G, C, B) replace the case's synthesised Tucker form
    case.tk = dict(case.tk, G=_core_host(f["G"], J, w.m, w.n, w.p),
                   C=_host(f["C"]).reshape(J, J, w.P, w.p), B=np.repeat(_host(f["B"]), J, axis=0))
    case.G, case.C = f["G"], f["C"]
    case.B = f["B"].expand(J, -1, -1).contiguous()
    case.Ptn = np.stack([S.project_precoder(case.tk["B"][k], case.Pw[k]) for k in range(J)])
    got, flags = case.gpu_sinr(precoder, "paths")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    ref = case.oracle_sinr(precoder)
    assert_sinr_close(got, ref, what=f"shared {precoder}")
    # the factors cancel: the dense oracle on X^ of the shared model gives the
    # same SINR (A and B re-orthonormalised in FP64: the FP32 factors are
    # orthonormal only to ~1e-7, which would bound the identity at that level)
    def orth(F):
        Q, R = np.linalg.qr(F)
        ph = np.diagonal(R, axis1=-2, axis2=-1)
        return Q * (ph / np.abs(ph))[..., None, :]        # F = Q R with diag(R) > 0: Q ~ F
    Aq, Bq = orth(_host(f["A"])), orth(_host(f["B"]))
    Xh = T.reconstruct_model(case.tk["G"], Aq, Bq, case.tk["C"], "shared")
    dense = S.dense_sinr(Xh, case.coef, case.s2, w.L, precoder, case.Pw if precoder == "mmse" else None)
    Ptq = np.stack([S.project_precoder(Bq[0], case.Pw[k]) for k in range(J)]) if precoder == "mmse" else None
    comp = S.tucker_sinr(case.tk["G"], case.tk["C"], case.coef, case.s2, w.L, precoder, Ptq)
    np.testing.assert_allclose(comp, dense, rtol=1e-8)


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_individual_model_sinr_through_reconstruction(precoder):
    w = dataclasses.replace(synth.SMALL, J=3, K=48)
    X = _channels(w)
    case = Case(w)
    d, f, _ = _gpu_fit(X, (w.m, w.n, w.p), 3, "individual", K=w.K, L=w.L)
    J = w.J
    Xhat = torch.empty(J * J, w.P, w.M, w.N, dtype=torch.complex64, device="cuda")
    ts.ts_tucker_reconstruct(d, ts.TS_MODEL_INDIVIDUAL, f["A"], f["B"], f["C"], f["G"], Xhat,
                             ts.workspace(d, ts.TS_OP_RECONSTRUCT))
    torch.cuda.synchronize()
    Xh = np.transpose(_host(Xhat).reshape(J, J, w.P, w.M, w.N), (0, 1, 3, 4, 2))
    case.X, case.Xd = Xh, Xhat
    got, flags = case.gpu_dense_sinr(precoder, "paths")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    ref = case.oracle_dense_sinr(precoder)
    assert_sinr_close(got, ref, what=f"individual {precoder}")
