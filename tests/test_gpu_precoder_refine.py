"""Close pairs of singular values in the SVD precoders (eq. 7, eq. 23;
TS_FLAG_PRECODER_REFINED).

Two adjacent squared singular values of H~_kk among the L + 1 largest within
5e-3 of the largest make the individual singular vectors, and with them the
per-stream SINRs, sensitive to the FP32 rounding of H~ by ~u / gap.  Those
units' precoders are refined from H~ formed in double-float (a Rayleigh-Ritz
step on each adjacent pair).  Checks against the FP64 oracle, every SINR
within the flat 1e-5:
  * a constructed serving core with a close pair at every subcarrier: one
    core slice (p = 1), so H~_kk = (c* C) G_kk has G_kk's singular values up
    to a scale; the pair inside the kept streams or at their boundary
    (ranks L - 1, L); the register precoder (n up to 600 here) and the
    staged one (16 rows, n = 1000); every unit flagged;
  * the precision workload's subcarriers 1596 .. 1611 (a range call), where
    serving links have pairs 4e-4 .. 4e-3 apart;
  * with the refinement off (negative threshold) no unit is flagged.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, assert_sinr_close, svd_gap, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _orth(rng, rows, cols):
    z = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    q, _ = np.linalg.qr(z)
    return q


def close_pair_case(sv, n, L, K=24, J=3, seed=11):
    """Serving cores G_kk = U diag(sv) V* (complex64 values) with the given
    singular values; interfering cores as drawn."""
    m = len(sv)
    w = workload(synth.SMALL, name=f"close pair m{m} n{n} L{L}", J=J, M=m, m=m, N=n + 8, n=n,
                 P=12, p=1, L=L, K=K, sigma2=0.05)
    case = Case(w)
    rng = np.random.default_rng(seed)
    for k in range(J):
        Gk = (_orth(rng, m, m) * np.asarray(sv)[None, :]) @ _orth(rng, n, m).conj().T
        case.tk["G"][k, k, :, :, 0] = Gk.astype(np.complex64).astype(np.complex128)
    case.G = ts.core_to_device(case.tk["G"])
    return case


# relative squared gaps ~5e-5 (inside the kept streams) and ~3e-5 (ranks 3, 4)
INSIDE = [3.0, 2.5, 2.4999, 2.0, 1.5, 1.0, 0.8, 0.6]
BOUNDARY = [3.0, 2.5, 2.0, 1.5, 1.4999, 1.0, 0.8, 0.6]


TAIL = [0.5, 0.45, 0.4, 0.35, 0.3, 0.25, 0.2, 0.15]
CASES = {
    "inside": (INSIDE, 24, 4),
    "boundary": (BOUNDARY, 24, 4),
    "L_equals_m": (INSIDE[:4], 24, 4),
    "wide_n": (INSIDE, 600, 4),              # register precoder, fewer subcarriers per CTA
    "staged": (INSIDE + TAIL, 1000, 8),      # 16 rows, n > 512: the staged precoder
}


@pytest.mark.parametrize("mode", ["paths", "dense"])
@pytest.mark.parametrize("name", list(CASES))
def test_constructed_close_pairs(name, mode):
    sv, n, L = CASES[name]
    case = close_pair_case(sv, n, L)
    assert svd_gap(case).max() < 5e-3            # a close pair at every subcarrier
    got, flags = case.gpu_sinr("svd", mode)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    assert np.all(flags & ts.TS_FLAG_PRECODER_REFINED)
    rel = assert_sinr_close(got, case.oracle_sinr("svd"), what=f"close pair n={n} {mode}")
    print(f"\nclose pair n={n} L={L} {mode}: max {rel.max():.3e}")


def test_refinement_off_flags_nothing():
    ts.ts_set_refinement(-1.0)
    try:
        case = close_pair_case(INSIDE, 24, 4)
        _, flags = case.gpu_sinr("svd", "paths")
    finally:
        ts.ts_set_refinement(8.0)
    assert not np.any(flags & ts.TS_FLAG_PRECODER_REFINED)


def test_precision_workload_close_pairs():
    w = synth.PRECISION
    k0, cnt = 1596, 16
    tk = synth.direct_tucker(w)
    alpha, tau = synth.path_gains_delays(w)
    s2 = synth.noise_powers(w)
    coef = S.coefficients(alpha, tau, w.K, w.delta_f_hz)[:, :, k0:k0 + cnt]
    ref = S.tucker_sinr(tk["G"], tk["C"], coef, s2, w.L, "svd")
    d = ts.Dims.of(w)
    G = ts.core_to_device(tk["G"])
    C = ts.factor_to_device(tk["C"].reshape(w.J * w.J, w.P, w.p))
    cs, keep = ts.make_coef(alpha=ts.factor_to_device(alpha.reshape(w.J * w.J, w.P)),
                            tau=ts.real_to_device(tau.reshape(w.J * w.J, w.P)))
    sinr = torch.full((w.J, cnt, w.L), float("nan"), device="cuda")
    flags = torch.full((w.J, cnt), 255, dtype=torch.uint8, device="cuda")
    ws = ts.workspace(dataclasses.replace(d, K=cnt), ts.TS_OP_SINR_SVD)
    ts.ts_sinr_svd_range(d, k0, cnt, cs, G, C, ts.real_to_device(s2), ts.TS_PREC_FP32, sinr, flags, ws)
    torch.cuda.synchronize()
    del keep
    fl = flags.cpu().numpy()
    assert np.all((fl & ts.TS_FLAG_ERRORS) == 0), np.unique(fl)
    assert np.any(fl & ts.TS_FLAG_PRECODER_REFINED)
    rel = assert_sinr_close(sinr.cpu().numpy().astype(np.float64), ref, what="precision 1596..1611")
    print(f"\nprecision 1596..1611: max {rel.max():.3e}; "
          f"{int(np.sum((fl[0] & ts.TS_FLAG_PRECODER_REFINED) != 0))} of {cnt} subcarriers refined")
