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


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    w = workload(synth.MID, K=300)      # mid-size system cut to fit the scratch
    case = Case(w)
    cs, keep = case.coef_struct("paths")
    Pt = _projected(case)
    ref = torch.empty(w.J, w.K, w.L, device=case.dev)
    ws = ts.workspace(case.d, ts.TS_OP_SINR_MMSE, case.dev)
    ts.ts_sinr_mmse(case.d, cs, case.G, case.C, Pt, case.sig, ref, None, ws)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((w.J, w.K, w.L), float("nan"), device=case.dev)
        flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device=case.dev)
        ts.ts_sinr_mmse_noalloc(case.d, cs, case.G, case.C, Pt, case.sig, out, flags)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(flags.cpu().numpy() == 0)
        rel = np.abs(got - ref) / np.abs(ref)
        assert rel.max() <= 1e-5, (call, rel.max())
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
