"""Failure detection without a GPU fault: the bounded mbarrier wait that the
tensor-core kernel uses (its operand copies and MMA completions) is made to
run out on a phase that nothing completes; it must give up within its
limit, report it, and leave the context usable (a SINR evaluation right
after still matches the oracle).  The positive control completes the
phase first."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def test_bounded_wait_gives_up_and_the_context_survives():
    out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    ts.ts_selftest_bounded_wait(1 << 12, False, out)
    torch.cuda.synchronize()
    assert int(out.item()) == 1, "the wait on a phase nothing completes must give up"
    assert time.perf_counter() - t0 < 30.0
    out.fill_(-1)
    ts.ts_selftest_bounded_wait(1 << 12, True, out)
    torch.cuda.synchronize()
    assert int(out.item()) == 0, "a completed phase must be seen"
    # the context is intact: a SINR evaluation still matches the oracle
    case = Case(synth.SMALL)
    got, flags = case.gpu_sinr("svd", "paths")
    ref = case.oracle_sinr("svd")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-4


def test_selftest_arguments_checked_before_launch():
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = ts.load()
    assert lib.ts_selftest_bounded_wait(0, 0, out.data_ptr(), None) == ts.TS_ERR_DIMS
    assert lib.ts_selftest_bounded_wait(1 << 25, 0, out.data_ptr(), None) == ts.TS_ERR_DIMS
    assert lib.ts_selftest_bounded_wait(16, 0, None, None) == ts.TS_ERR_NULL
