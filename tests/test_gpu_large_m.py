"""Units with more than 16 receive rows (m up to 64, as in the paper's
(64, 512, 401) channels with m = 60): the shared-memory precoder and
finalisation and the 32 / 64-row instances of the wide-core link kernel,
against the FP64 oracle at the FP32 SINR tolerance of the other tests,
with the dense comparator and several UEs per cell on the same path."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, assert_sinr_close  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _wl(name, **kw):
    base = dict(J=3, M=32, N=64, P=32, K=40, m=24, n=40, p=16, L=4, n_los=2, pdp_decay_s=300e-9,
                sigma2=None, seed=21)
    base.update(kw)
    return dataclasses.replace(synth.MID, name=name, **base)


CASES = {
    "m24": _wl("large m24"),                                                   # 32-row groups
    "m60": _wl("large m60", J=2, M=64, m=60, N=128, n=64, P=48, p=40, L=8, K=24),  # 64-row groups
    "m33_odd": _wl("large m33", M=40, m=33, n=37, L=3, K=19),                 # odd sizes
    # 64-row groups, rows masked, odd n and L, three subcarrier tiles of 16
    # with a ragged last one (256 threads, four subcarriers per lane)
    "m49_odd": _wl("large m49", M=56, m=49, N=64, n=45, P=40, p=36, L=3, K=37),
    # more rows than columns: the Gram of every serving link has rank n < m
    "m40_n12": _wl("large m40 n12", M=40, m=40, N=16, n=12, L=4),
    "one_cell_one_subcarrier": _wl("large J1 K1", J=1, K=1, L=1),             # no interferers
}


@pytest.mark.parametrize("mode", ["paths", "dense"])
@pytest.mark.parametrize("name", list(CASES))
def test_large_m_svd_sinr(name, mode):
    case = Case(CASES[name])
    got, flags = case.gpu_sinr("svd", mode)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    ref = case.oracle_sinr("svd")
    assert_sinr_close(got, ref, what=f"{name} {mode}")


@pytest.mark.parametrize("M", [24, 64])
def test_large_m_dense_comparator(M):
    w = _wl(f"large dense M{M}", M=M, m=M, N=32, n=32, P=24 if M < 64 else 40, p=24, L=4, K=30)
    case = Case(w).with_channels()
    got, flags = case.gpu_dense_sinr("svd", "paths")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    ref = case.oracle_dense_sinr("svd")
    assert_sinr_close(got, ref, what=f"dense M{M}")


def test_large_m_limits():
    w = CASES["m24"]
    d = ts.Dims.of(w)
    assert ts.ts_workspace_bytes(d, ts.TS_OP_SINR_SVD) > 0
    for op in (ts.TS_OP_SINR_MMSE, ts.TS_OP_SINR_SVD_ADJOINT, ts.TS_OP_SINR_SVD_TF32):
        assert ts.ts_workspace_bytes(d, op) == 0
    # more than 8 streams, or more than 64 rows, are refused
    assert ts.ts_workspace_bytes(ts.Dims.of(dataclasses.replace(w, L=12, m=24)), ts.TS_OP_SINR_SVD) == 0
    assert ts.ts_workspace_bytes(ts.Dims.of(dataclasses.replace(w, M=80, m=65)), ts.TS_OP_SINR_SVD) == 0
