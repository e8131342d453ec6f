"""FP64-residual refinement of ill-conditioned SINR solves (ts_set_refinement,
TS_FLAG_REFINED) against the FP64 oracle.

Units whose FP32 Cholesky factor of R = sum_{k != i} E_ik E_ik* + sigma^2 I
shows cond(R) above the threshold are re-solved: two refinement steps of
R^{-1} E_ii with FP64 residuals, then the L x L system in FP64.  Checks: the
refined SINRs stay within the FP32 per-result tolerance of
tests/test_gpu_sinr.py, their error does not grow over the unrefined FP32
result of the same units, only listed units carry the flag, and a zero
threshold (every unit refined) reproduces the oracle on both precoders and
odd shapes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, interference_condition, svd_gap, workload  # noqa: E402

U32 = 2.0 ** -24


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
        ts.ts_set_refinement(1e3)


def _tol(case, precoder, shape):
    cond = interference_condition(case, precoder)
    tol = 1e-5 + 4 * U32 * cond
    if precoder == "svd":
        tol = tol + 8 * U32 / np.maximum(svd_gap(case), 1e-30)[None, :]
    return np.broadcast_to(tol[:, :, None], shape), cond


# the precision workload's shapes and noise range (sigma^2 in [1e-4, 1e-1]) on
# fewer cells and subcarriers; a threshold low enough that both precoders
# have units above it
ILL = dict(J=4, K=96)
THRESHOLD = 1e2


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_ill_conditioned_units_are_refined(precoder):
    case = Case(workload(synth.PRECISION, **ILL))
    ref = case.oracle_sinr(precoder)
    off, f_off = _run(case, precoder, -1.0)
    on, f_on = _run(case, precoder, THRESHOLD)
    assert not np.any(f_off & ts.TS_FLAG_REFINED)
    assert np.all((f_on & ts.TS_FLAG_ERRORS) == 0)
    refined = (f_on & ts.TS_FLAG_REFINED) != 0
    tol, cond = _tol(case, precoder, ref.shape)
    # the listing follows the condition number (the diagonal estimate is a
    # lower bound of cond(R))
    assert refined.any(), f"no unit refined; max cond(R) {cond.max():.3e}"
    assert not np.any(refined & (cond < 0.9 * THRESHOLD))
    r_on = np.abs(on - ref) / np.abs(ref)
    r_off = np.abs(off - ref) / np.abs(ref)
    assert np.all(r_on <= tol), f"max rel {r_on.max():.3e}"
    sel = np.broadcast_to(refined[:, :, None], ref.shape)
    # unrefined units are untouched; refined ones are no worse
    np.testing.assert_array_equal(on[~sel], off[~sel])
    assert r_on[sel].max() <= 1.5 * r_off[sel].max() + 1e-9
    assert np.median(r_on[sel]) <= np.median(r_off[sel]) * 1.0001 + 1e-9
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
    assert np.all(flags == ts.TS_FLAG_REFINED)
    ref = case.oracle_sinr(precoder)
    tol, _ = _tol(case, precoder, ref.shape)
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.all(rel <= tol), f"max rel {rel.max():.3e}"
