"""Subcarrier ranges (ts_sinr_svd_range, ts_sinr_mmse_range): the partition
of one system's subcarriers across devices, with G, C and the coefficients
replicated.  Every (UE, subcarrier) unit is independent (the precoders of
eq. 7 are per subcarrier), so the ranges of a split must reproduce the
whole-system call bit for bit, whatever the split points (tile boundaries of
the kernels or not) and for every arithmetic mode."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2401_09792_gb300 import partition  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import Case  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _whole(case, precoder, prec, mode):
    w = case.w
    cs, keep = case.coef_struct(mode)
    sinr = torch.full((w.J, w.K, w.L), float("nan"), device="cuda")
    flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device="cuda")
    if precoder == "svd":
        op = {ts.TS_PREC_FP32: ts.TS_OP_SINR_SVD, ts.TS_PREC_TF32X3: ts.TS_OP_SINR_SVD_TF32X3}[prec]
        ts.ts_sinr_svd_prec(case.d, cs, case.G, case.C, case.sig, prec, sinr, flags, ts.workspace(case.d, op))
    else:
        ts.ts_sinr_mmse(case.d, cs, case.G, case.C, case.Pt, case.sig, sinr, flags,
                        ts.workspace(case.d, ts.TS_OP_SINR_MMSE))
    torch.cuda.synchronize()
    del keep
    return sinr.cpu().numpy(), flags.cpu().numpy()


def _ranges(case, precoder, prec, mode, bounds):
    w = case.w
    cs, keep = case.coef_struct(mode)
    outs, fls = [], []
    for k0, k1 in bounds:
        cnt = k1 - k0
        dr = dataclasses.replace(case.d, K=cnt)
        sinr = torch.full((w.J, cnt, w.L), float("nan"), device="cuda")
        flags = torch.full((w.J, cnt), 255, dtype=torch.uint8, device="cuda")
        if precoder == "svd":
            op = {ts.TS_PREC_FP32: ts.TS_OP_SINR_SVD, ts.TS_PREC_TF32X3: ts.TS_OP_SINR_SVD_TF32X3}[prec]
            ts.ts_sinr_svd_range(case.d, k0, cnt, cs, case.G, case.C, case.sig, prec, sinr, flags,
                                 ts.workspace(dr, op))
        else:
            ts.ts_sinr_mmse_range(case.d, k0, cnt, cs, case.G, case.C, case.Pt, case.sig, sinr, flags,
                                  ts.workspace(dr, ts.TS_OP_SINR_MMSE))
        torch.cuda.synchronize()
        outs.append(sinr.cpu().numpy())
        fls.append(flags.cpu().numpy())
    del keep
    return np.concatenate(outs, axis=1), np.concatenate(fls, axis=1)


@pytest.mark.parametrize("precoder,prec", [("svd", ts.TS_PREC_FP32), ("svd", ts.TS_PREC_TF32X3),
                                           ("mmse", ts.TS_PREC_FP32)])
@pytest.mark.parametrize("mode", ["paths", "dense"])
def test_ranges_equal_the_whole_call_bit_for_bit(precoder, prec, mode):
    case = Case(dataclasses.replace(synth.MID, K=700))
    w = case.w
    case.Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device="cuda")
    ts.ts_project_precoder(case.d, case.B, case.Pf, case.Pt)
    whole, fw = _whole(case, precoder, prec, mode)
    # three ranks of an uneven split, and a split at odd points
    for bounds in (partition.subcarrier_ranges(w.K, 3), [(0, 1), (1, 357), (357, 700)]):
        got, fg = _ranges(case, precoder, prec, mode, bounds)
        assert np.array_equal(got, whole), bounds
        assert np.array_equal(fg, fw), bounds


def test_two_kernel_precoder_ranges():
    """Serving channels from the serving pass (m n p > 8192: the serving
    pass, then the eigensolve and the rest of the precoder as two kernels,
    and in TF32X3 the serving channels on the tensor cores): ranges
    reproduce the whole call bit for bit, split at a multiple of the
    kernels' tiles or not."""
    from tests.gpu_inputs import workload
    w = workload(synth.SMALL, name="two-kernel precoder", J=3, M=16, m=16, N=80, n=64, P=40, p=32, L=8,
                 K=300, sigma2=0.05)
    assert w.m * w.n * w.p > 8192
    case = Case(w)
    for prec in (ts.TS_PREC_FP32, ts.TS_PREC_TF32X3):
        whole, fw = _whole(case, "svd", prec, "paths")
        for bounds in ([(0, 100), (100, 300)], [(0, 101), (101, 300)], [(0, 1), (1, 257), (257, 300)]):
            got, fg = _ranges(case, "svd", prec, "paths", bounds)
            assert np.array_equal(got, whole), (prec, bounds)
            assert np.array_equal(fg, fw), (prec, bounds)


def test_range_arguments_are_checked():
    case = Case(synth.SMALL)
    cs, keep = case.coef_struct("paths")
    w = case.w
    sinr = torch.empty(w.J, w.K, w.L, device="cuda")
    ws = ts.workspace(case.d, ts.TS_OP_SINR_SVD)
    for k0, cnt in ((-1, 4), (0, 0), (w.K - 3, 4)):
        with pytest.raises(ts.TsError) as e:
            ts.ts_sinr_svd_range(case.d, k0, cnt, cs, case.G, case.C, case.sig, ts.TS_PREC_FP32, sinr, None, ws)
        assert e.value.status == ts.TS_ERR_DIMS
    del keep
