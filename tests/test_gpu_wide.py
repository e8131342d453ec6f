"""The wide-core SVD path: ranks p beyond the narrow kernels' staging (p > 32,
or P p > 8192), as in the paper's experiments (p = 120-190 of P = 401 paths),
and the dense-channel comparator at large P.  The projection reads C_ik from
L2 and the core streams through shared memory in slabs of 16, so the cases
below cover one and several slabs with a ragged last slab, a ragged
subcarrier tile, m below the lane group, both group sizes, dense and
path-form coefficients.  Parity with the FP64 oracle at the FP32 SINR
tolerance of the narrow-path tests."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case, interference_condition, svd_gap  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _wl(name, **kw):
    base = dict(J=3, M=8, N=64, P=64, K=80, m=8, n=40, p=48, L=4, n_los=2, pdp_decay_s=300e-9,
                sigma2=None, seed=5)
    base.update(kw)
    return dataclasses.replace(synth.MID, name=name, **base)


def _tolerance(case, dense):
    tol = 1e-5 + 4 * U32 * interference_condition(case, "svd", dense)
    tol = tol + 8 * U32 / np.maximum(svd_gap(case, dense), 1e-30)[None, :]
    return tol[:, :, None]


CASES = {
    "p48": _wl("wide p48"),                                   # three slabs, last one full
    "p120_P401": _wl("wide p120 P401", P=401, p=120, n=24, K=70),   # the paper's P, ragged slab
    "p20_P512": _wl("wide p20 P512", P=512, p=20, n=16, K=64),      # p <= 32 but P p > 8192
    "m3": _wl("wide m3", M=4, m=3, L=2, p=40, n=20),                 # rows masked in the group
    "m12": _wl("wide m12", M=16, m=12, L=8, p=36, n=24, K=33),      # 16-lane groups
    "odd": _wl("wide odd", m=7, n=23, L=3, p=40, K=45),             # 8-byte copies (odd n, L)
    "one_cell_one_subcarrier": _wl("wide J1 K1", J=1, K=1),         # no interferers, one subcarrier
    "m1": _wl("wide m1", M=2, m=1, L=1, n=5, p=40, K=20),           # rank-one rows, one stream
    "p256": _wl("wide p256", M=4, m=4, L=2, n=8, P=300, p=256, K=40),  # the largest rank, many passes
}


@pytest.mark.parametrize("mode", ["paths", "dense"])
@pytest.mark.parametrize("name", list(CASES))
def test_wide_core_svd_sinr(name, mode):
    case = Case(CASES[name])
    d = case.d
    assert ts.ts_workspace_bytes(d, ts.TS_OP_SINR_SVD) > 0
    got, flags = case.gpu_sinr("svd", mode)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    ref = case.oracle_sinr("svd")
    rel = np.abs(got - ref) / np.abs(ref)
    tol = _tolerance(case, dense=False)
    assert np.all(rel <= tol), f"max rel {rel.max():.3e} (max rel/tol {(rel / tol).max():.2f})"


def test_wide_paths_reject_the_narrow_only_operations():
    d = CASES["p48"]
    dd = ts.Dims.of(d)
    assert ts.ts_workspace_bytes(dd, ts.TS_OP_SINR_SVD) > 0
    assert ts.ts_workspace_bytes(dd, ts.TS_OP_SINR_MMSE) == 0
    assert ts.ts_workspace_bytes(dd, ts.TS_OP_SINR_SVD_ADJOINT) == 0
    assert ts.ts_workspace_bytes(dd, ts.TS_OP_SINR_SVD_TF32) == 0


@pytest.mark.parametrize("P,N,M", [(64, 48, 8), (401, 32, 4), (1024, 8, 2)])
def test_dense_comparator_at_large_P(P, N, M):
    # C = I, p = P: the wide kernel evaluates w = c* per slab
    w = _wl(f"dense P{P}", P=P, N=N, M=M, m=M, n=min(16, N), p=16, L=2, K=70)
    case = Case(w).with_channels()
    got, flags = case.gpu_dense_sinr("svd", "paths")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    ref = case.oracle_dense_sinr("svd")
    rel = np.abs(got - ref) / np.abs(ref)
    tol = _tolerance(case, dense=True)
    assert np.all(rel <= tol), f"max rel {rel.max():.3e}"
