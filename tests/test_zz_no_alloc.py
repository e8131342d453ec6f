"""The allocation-free MMSE entry point, checked against the workspace one.

ts_sinr_mmse_noalloc exists for callers that cannot allocate device memory
when they evaluate SINR (a per-slot scheduler with a fixed latency budget,
where cudaMalloc may synchronise the device; a plug-in in a framework that
owns all device memory).  It runs the same kernels on a fixed scratch array
inside the library.  This file is collected last on purpose, so that a run
stopping at the first failure has run every other test; it also passes on
its own in a fresh process (it builds and loads the library itself).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _projected(case):
    w = case.w
    Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device=case.dev)
    ts.ts_project_precoder(case.d, case.B, case.Pf, Pt)
    return Pt


def _workspace_call(case, cs, Pt):
    w = case.w
    out = torch.empty(w.J, w.K, w.L, device=case.dev)
    ws = ts.workspace(case.d, ts.TS_OP_SINR_MMSE, case.dev)
    ts.ts_sinr_mmse(case.d, cs, case.G, case.C, Pt, case.sig, out, None, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _noalloc_call(case, cs, Pt):
    """One call of the allocation-free entry point, with the device's free
    memory read right before and right after it (outputs allocated first)."""
    w = case.w
    out = torch.full((w.J, w.K, w.L), float("nan"), device=case.dev)
    flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device=case.dev)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    ts.ts_sinr_mmse_noalloc(case.d, cs, case.G, case.C, Pt, case.sig, out, flags)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert np.all((flags.cpu().numpy() & ts.TS_FLAG_ERRORS) == 0)
    return out.cpu().numpy(), free_before, free_after


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    # two calls in a row on different systems (other subcarrier count, other
    # noise powers), so that a read of the previous call's scratch would show;
    # the same kernels run on both entry points, so the results are equal bit
    # for bit
    cases = [Case(workload(synth.MID, K=300)),                      # cut to fit the scratch
             Case(workload(synth.MID, K=180, sigma2_range=(1e-4, 1e-2), seed=3))]
    for call, case in enumerate(cases):
        cs, keep = case.coef_struct("paths")
        Pt = _projected(case)
        ref = _workspace_call(case, cs, Pt)
        got, free_before, free_after = _noalloc_call(case, cs, Pt)
        assert np.array_equal(got, ref), (call, float(np.nanmax(np.abs(got - ref) / np.abs(ref))))
        if call > 0:
            # the scratch was committed by the first call: this one allocates nothing
            assert free_before == free_after, (free_before, free_after)
        del keep


def test_noalloc_rejects_sizes_beyond_its_scratch():
    w = workload(synth.MID, K=1024)     # needs about 34 MB of scratch
    d = ts.Dims.of(w)
    assert ts.ts_workspace_bytes(d, ts.TS_OP_SINR_MMSE) > ts.TS_NOALLOC_SCRATCH_BYTES
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")
    sig = torch.ones(w.J, device="cuda")
    out = torch.zeros(w.J, w.K, w.L, device="cuda")
    cs, keep = ts.make_coef(c=dummy)
    with pytest.raises(ts.TsError) as err:
        ts.ts_sinr_mmse_noalloc(d, cs, dummy, dummy, dummy, sig, out, None)
    assert err.value.status == 4       # TS_ERR_WORKSPACE, before any launch
    del keep
