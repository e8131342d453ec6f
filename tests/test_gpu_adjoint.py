"""Parity of the CUDA SINR adjoints (through the C ABI and the
torch.autograd.Function) with the FP64 oracle's vector-Jacobian products
(oracle.adjoint, itself pinned to central finite differences).

Tolerance (FP32 on the GPU): max |grad_gpu - grad_oracle| <= 1e-4 max |grad_oracle|
per gradient array, on systems whose serving channels have well separated
singular values (the SVD adjoint carries 1/(s_r^2 - s_s^2) factors).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as AD  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _dsinr(w, seed=0):
    return np.random.default_rng(seed).standard_normal((w.J, w.K, w.L))


def _to_host_core(dG, w):
    """device [J*J][p][m][n] -> oracle (J, J, m, n, p)."""
    a = dG.cpu().numpy().astype(np.complex128).reshape(w.J, w.J, w.p, w.m, w.n)
    return np.transpose(a, (0, 1, 3, 4, 2))


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _gpu_adjoint(case, precoder, ds):
    w = case.w
    cs, keep = case.coef_struct("paths")
    dsd = torch.from_numpy(ds.astype(np.float32)).cuda()
    dG = torch.empty_like(case.G)
    dC = torch.empty_like(case.C)
    sinr = torch.empty(w.J, w.K, w.L, device="cuda")
    out = {}
    if precoder == "svd":
        ws = ts.workspace(case.d, ts.TS_OP_SINR_SVD_ADJOINT)
        ts.ts_sinr_svd_adjoint(case.d, cs, case.G, case.C, case.sig, dsd, dG, dC, sinr, ws)
    else:
        Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device="cuda")
        ts.ts_project_precoder(case.d, case.B, case.Pf, Pt)
        dPt = torch.empty_like(Pt)
        ws = ts.workspace(case.d, ts.TS_OP_SINR_MMSE_ADJOINT)
        ts.ts_sinr_mmse_adjoint(case.d, cs, case.G, case.C, Pt, case.sig, dsd, dG, dC, dPt, sinr, ws)
        dB = torch.empty(w.J, w.N, w.n, dtype=torch.complex64, device="cuda")
        ts.ts_project_precoder_adjoint(case.d, case.Pf, dPt, dB)
        out["dB"] = dB.cpu().numpy().astype(np.complex128)
    torch.cuda.synchronize()
    del keep
    out["dG"] = _to_host_core(dG, w)
    out["dC"] = dC.cpu().numpy().astype(np.complex128).reshape(w.J, w.J, w.P, w.p)
    out["sinr"] = sinr.cpu().numpy().astype(np.float64)
    return out


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
@pytest.mark.parametrize("shape", ["small", "odd", "m12_L2"])
def test_adjoint_matches_oracle(precoder, shape):
    base = workload(synth.SMALL, K=16)
    if shape == "odd":
        base = workload(synth.SMALL, J=3, M=3, m=3, n=7, N=12, P=5, p=3, L=2, K=9)
    if shape == "m12_L2":                   # 16-lane groups with two streams
        base = workload(synth.SMALL, J=2, M=16, m=12, N=24, n=12, P=6, p=4, L=2, K=8)
    case = Case(base)
    ds = _dsinr(base)
    ref = AD.tucker_sinr_vjp(case.tk["G"], case.tk["C"], case.coef, case.s2, base.L, ds, precoder,
                             case.tk["B"], case.Pw)
    got = _gpu_adjoint(case, precoder, ds)
    np.testing.assert_allclose(got["sinr"], ref["sinr"], rtol=1e-4)
    assert _rel(got["dG"], ref["dG"]) < 1e-4, _rel(got["dG"], ref["dG"])
    assert _rel(got["dC"], ref["dC"]) < 1e-4, _rel(got["dC"], ref["dC"])
    if precoder == "mmse":
        assert _rel(got["dB"], ref["dB"]) < 1e-4, _rel(got["dB"], ref["dB"])


def test_differentiation_shapes_on_two_subcarriers():
    # the differentiation workload's sizes (J=16, M=16, N=1024, P=64,
    # ranks (16,96,32), L=8) on a 2-subcarrier slice
    w = workload(synth.DIFFERENTIATION, K=2)
    case = Case(w)
    ds = _dsinr(w, 1)
    ref = AD.tucker_sinr_vjp(case.tk["G"], case.tk["C"], case.coef, case.s2, w.L, ds, "svd")
    got = _gpu_adjoint(case, "svd", ds)
    assert _rel(got["dG"], ref["dG"]) < 1e-3, _rel(got["dG"], ref["dG"])
    assert _rel(got["dC"], ref["dC"]) < 1e-3, _rel(got["dC"], ref["dC"])


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_autograd_function(precoder):
    from paper_2401_09792_gb300.autograd import compressed_sinr
    w = workload(synth.SMALL, K=16)
    case = Case(w)
    ds = _dsinr(w, 2)
    G = case.G.clone().requires_grad_(True)
    C = case.C.clone().requires_grad_(True)
    Pt = None
    if precoder == "mmse":
        Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device="cuda")
        ts.ts_project_precoder(case.d, case.B, case.Pf, Pt)
    s = compressed_sinr(G, C, case.al, case.ta, case.sig, case.d, precoder, Pt)
    (s * torch.from_numpy(ds.astype(np.float32)).cuda()).sum().backward()
    ref = AD.tucker_sinr_vjp(case.tk["G"], case.tk["C"], case.coef, case.s2, w.L, ds, precoder,
                             case.tk["B"], case.Pw)
    assert _rel(_to_host_core(G.grad, w), ref["dG"]) < 1e-4
    assert _rel(C.grad.cpu().numpy().reshape(w.J, w.J, w.P, w.p), ref["dC"]) < 1e-4
