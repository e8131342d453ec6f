"""Parity of the CUDA SINR path (through the C ABI) with the FP64 oracle.

Tolerance: every SINR within 1e-5 relative of the oracle (FP32 arithmetic on
the GPU, complex128 in the oracle, the same complex64 inputs).  FP32
rounding of the compressed channels alone moves the SINR by ~5e-7 at these
sizes (the oracle's own channels rounded to complex64), so the bound leaves
room for the eigensolve and the solves but not for an unconverged precoder.
The one exception is a stream whose serving singular value is below 1e-2 of
the largest (only the square L = m = n edge case has them): its SINR is
fixed by the complex64 inputs only to ~u sigma_1 / sigma_r, and gets that
on top (tests/gpu_inputs.py, weak_stream_rtol).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, assert_sinr_close, weak_stream_rtol, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _check(case: Case, precoder: str, mode: str):
    got, flags = case.gpu_sinr(precoder, mode)
    ref = case.oracle_sinr(precoder)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    return assert_sinr_close(got, ref, weak_stream_rtol(case, precoder=precoder),
                             what=f"{case.w.name} {precoder} {mode}")


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
@pytest.mark.parametrize("mode", ["dense", "paths"])
def test_small_workload(precoder, mode):
    _check(Case(synth.SMALL), precoder, mode)


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_mid_workload_full_size(precoder):
    # J=8, M=8, N=256, P=32, K=1024, ranks (8,32,16), L=8: the benchmark's sizes
    rel = _check(Case(synth.MID), precoder, "paths")
    assert rel.shape == (8, 1024, 8)


EDGE = {
    "single_cell": dict(J=1, K=5),
    "ragged_K": dict(K=70),
    "one_subcarrier": dict(K=1),
    "odd_m_n_p1": dict(M=3, m=3, n=13, N=20, p=1, L=2),
    "one_stream": dict(L=1),
    "m1": dict(M=1, m=1, L=1),
    "m2_full": dict(M=2, m=2, L=2, n=2, N=8),
    "max_m16": dict(J=2, M=16, m=16, L=16, N=24, n=16, P=6, p=3, K=40),
    "m16_L8_n24": dict(J=3, M=16, m=12, L=8, N=40, n=24, P=10, p=5, K=33),
    # more rows than columns: the m x m Gram of every link has rank n < m
    "m_above_n": dict(M=16, m=16, N=8, n=4, L=2),
    "m8_n2": dict(M=8, m=8, N=4, n=2, L=1),
}


@pytest.mark.parametrize("name", sorted(EDGE))
@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_edge_cases(name, precoder):
    w = workload(synth.SMALL, **EDGE[name])
    _check(Case(w), precoder, "paths")


def test_coefficients_kernel():
    w = workload(synth.MID, K=3300)       # the largest subcarrier count of the workloads
    alpha, tau = synth.path_gains_delays(w)
    ref = S.coefficients(alpha, tau, w.K, w.delta_f_hz).reshape(w.J * w.J, w.K, w.P)
    d = ts.Dims.of(w)
    al = ts.factor_to_device(alpha.reshape(w.J * w.J, w.P))
    ta = ts.real_to_device(tau.reshape(w.J * w.J, w.P))
    c = torch.empty(w.J * w.J, w.K, w.P, dtype=torch.complex64, device="cuda")
    ts.ts_coefficients(d, al, ta, c)
    got = c.cpu().numpy()
    amp = np.abs(alpha.reshape(w.J * w.J, 1, w.P))
    assert np.all(np.abs(got - ref) <= 1e-6 * amp + 1e-30)


def test_nonfinite_input_flags_and_nan():
    case = Case(synth.SMALL)
    G = case.G.clone()
    G.view(-1)[0] = complex(float("nan"), 0.0)      # core of link (0, 0)
    case.G = G
    got, flags = case.gpu_sinr("mmse", "dense")
    assert np.isnan(got[0]).all()
    assert np.all(flags[0] != 0)


# ------------------------------------------------------- dense comparator
def _check_dense(case: Case, precoder: str):
    got, flags = case.gpu_dense_sinr(precoder, "paths")
    ref = case.oracle_dense_sinr(precoder)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    assert_sinr_close(got, ref, weak_stream_rtol(case, dense=True, precoder=precoder),
                      what=f"dense {case.w.name} {precoder}")


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_dense_comparator_small(precoder):
    _check_dense(Case(synth.SMALL).with_channels(), precoder)


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_dense_comparator_mid_full_size(precoder):
    # M=8, N=256, P=32, K=1024, J=8: the benchmark's dense comparator
    _check_dense(Case(synth.MID).with_channels(), precoder)


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_factor_cancellation_on_gpu(precoder):
    # Section 3.3: the dense GPU path on X^ = G x_1 A x_2 B x_3 C equals the
    # compressed GPU path on (G, C) (A and B cancel) -- two different kernel
    # configurations that must agree
    from oracle import tucker as T
    w = workload(synth.SMALL, J=3, K=40, L=2)
    case = Case(w)
    tk = case.tk
    Xh = np.stack([np.stack([T.tucker_reconstruct(tk["G"][i, k], tk["A"][i], tk["B"][k], tk["C"][i, k])
                             for k in range(w.J)]) for i in range(w.J)])
    case.with_channels(Xh)
    comp, _ = case.gpu_sinr(precoder, "paths")
    dense, _ = case.gpu_dense_sinr(precoder, "paths")
    np.testing.assert_allclose(dense, comp, rtol=2e-5)   # both within 1e-5 of one oracle value
