"""Accurate re-evaluation of sensitive units (ts_set_refinement,
TS_FLAG_REFINED) against the FP64 oracle.

Units whose SINRs are sensitive to the FP32 rounding of
R = sum_{k != i} E_ik E_ik* + sigma^2 I (the estimate s of the header above
the threshold) are evaluated again: R in double-float
from the stored effective channels, three refinement steps of R^{-1} E_ii
with FP64 residuals, then the L x L system in FP64.  Checks, at
the precision workload's noise range (sigma^2 down to 1e-4): every SINR,
refined or not, within 1e-5 of the oracle; refinement lowers the error of
the units it lists (median) and never raises their maximum; unlisted units
are untouched (away from subcarriers whose SVD precoders were refined for
a close pair of singular values, TS_FLAG_PRECODER_REFINED); only listed
units carry the flag; a zero threshold (every unit refined) reproduces the
oracle on both precoders and odd shapes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, assert_sinr_close, interference_condition, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _run(case, precoder, threshold):
    ts.ts_set_refinement(threshold)
    try:
        return case.gpu_sinr(precoder, "paths")
    finally:
        ts.ts_set_refinement(8.0)


# the precision workload's shapes and noise range (sigma^2 in [1e-4, 1e-1]) on
# fewer cells and subcarriers; a threshold low enough that both precoders
# have units above it
ILL = dict(J=4, K=96)
THRESHOLD = 1.0


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_ill_conditioned_units_are_refined(precoder):
    case = Case(workload(synth.PRECISION, **ILL))
    ref = case.oracle_sinr(precoder)
    off, f_off = _run(case, precoder, -1.0)
    on, f_on = _run(case, precoder, THRESHOLD)
    assert not np.any(f_off & ts.TS_FLAG_REFINED)
    assert np.all((f_on & ts.TS_FLAG_ERRORS) == 0)
    refined = (f_on & ts.TS_FLAG_REFINED) != 0
    cond = interference_condition(case, precoder)
    assert refined.any(), f"no unit refined; max cond(R) {cond.max():.3e}"
    r_on = assert_sinr_close(on, ref, what=f"{precoder} refined")
    r_off = np.abs(off - ref) / np.abs(ref)
    sel = np.broadcast_to(refined[:, :, None], ref.shape)
    # subcarriers where a serving link's precoder was refined (close pair of
    # singular values; the SVD precoders only, flagged on every UE there)
    prec = np.broadcast_to(((f_on & ts.TS_FLAG_PRECODER_REFINED) != 0)[:, :, None], ref.shape)
    assert not np.any(f_off & ts.TS_FLAG_PRECODER_REFINED)
    # unrefined units are untouched; refined ones gain (median) and lose
    # nowhere beyond the rounding level of the unrefined result
    np.testing.assert_array_equal(on[~sel & ~prec], off[~sel & ~prec])
    assert np.median(r_on[sel]) < np.median(r_off[sel])
    assert r_on[sel].max() <= r_off[sel].max() + 1e-6
    print(f"\n{precoder}: {refined.sum()} of {refined.size} units refined; on refined units "
          f"max {r_off[sel].max():.3e} -> {r_on[sel].max():.3e}, median "
          f"{np.median(r_off[sel]):.3e} -> {np.median(r_on[sel]):.3e}")


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
@pytest.mark.parametrize("shape", ["small", "odd", "m16", "m12_L2"])
def test_refining_every_unit_matches_oracle(precoder, shape):
    w = {"small": synth.SMALL,
         "odd": workload(synth.SMALL, J=3, M=3, m=3, n=7, N=12, P=5, p=3, L=2, K=9),
         "m16": workload(synth.SMALL, J=2, M=16, m=16, L=8, N=40, n=24, P=10, p=5, K=33),
         "m12_L2": workload(synth.SMALL, J=2, M=16, m=12, L=2, N=40, n=24, P=10, p=5, K=33)}[shape]
    case = Case(w)
    got, flags = _run(case, precoder, 0.0)
    assert np.all((flags & (0xFF ^ ts.TS_FLAG_PRECODER_REFINED)) == ts.TS_FLAG_REFINED)
    ref = case.oracle_sinr(precoder)
    assert_sinr_close(got, ref, what=f"{shape} {precoder}, every unit refined")
