"""Batched evaluation (ts_batch_plan_create / ts_batch_launch): many systems
with their own numbers of cells, antennas, ranks, streams and subcarriers,
drawn from the batching workload's ranges (scaled down so that the oracle
finishes), evaluated by one graph launch.  Each instance's SINR must equal
the single-system call on the same inputs (the same kernels run), match the
FP64 oracle within the FP32 tolerance, follow in-place input changes on a
replay, and stay within tolerance when the autotuner picks the launch
shapes."""
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


def _systems(count=10, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        M = int(rng.choice([2, 4, 8]))
        N = int(rng.choice([64, 128, 256]))
        n = int(rng.choice([16, 32]))
        w = dataclasses.replace(synth.SMALL, name=f"batch{j}", J=int(rng.integers(2, 6)), M=M, m=M, L=M,
                                N=N, n=n, P=16, p=int(rng.choice([8, 16])), K=int(rng.integers(16, 200)),
                                n_los=2, pdp_decay_s=300e-9, sigma2=None, sigma2_range=(1e-3, 1.0),
                                seed=100 + j)
        op = ts.TS_OP_SINR_MMSE if j % 3 == 2 else ts.TS_OP_SINR_SVD
        prec = ts.TS_PREC_TF32 if j == 4 else ts.TS_PREC_FP32
        out.append((Case(w), op, prec))
    return out


def _instances(systems):
    insts, outs, keep = [], [], []
    for case, op, prec in systems:
        w = case.w
        cs, k = case.coef_struct("paths")
        sinr = torch.full((w.J, w.K, w.L), float("nan"), device="cuda")
        flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device="cuda")
        Pt = None
        if op == ts.TS_OP_SINR_MMSE:
            Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device="cuda")
            ts.ts_project_precoder(case.d, case.B, case.Pf, Pt)
        insts.append(ts.instance(case.d, op, cs, case.G, case.C, case.sig, sinr, flags, Pt, prec))
        outs.append((sinr, flags))
        keep.append((k, Pt))
    return insts, outs, keep


def _single(case, op, prec, Pt):
    w = case.w
    cs, keep = case.coef_struct("paths")
    sinr = torch.empty(w.J, w.K, w.L, device="cuda")
    if op == ts.TS_OP_SINR_MMSE:
        ws = ts.workspace(case.d, ts.TS_OP_SINR_MMSE)
        ts.ts_sinr_mmse(case.d, cs, case.G, case.C, Pt, case.sig, sinr, None, ws)
    else:
        opw = {ts.TS_PREC_FP32: ts.TS_OP_SINR_SVD, ts.TS_PREC_TF32: ts.TS_OP_SINR_SVD_TF32}[prec]
        ts.ts_sinr_svd_prec(case.d, cs, case.G, case.C, case.sig, prec, sinr, None, ts.workspace(case.d, opw))
    torch.cuda.synchronize()
    del keep
    return sinr.cpu().numpy().astype(np.float64)


def _check_oracle(case, op, got, prec):
    precoder = "mmse" if op == ts.TS_OP_SINR_MMSE else "svd"
    ref = case.oracle_sinr(precoder)
    # FP32: the flat bound; TF32 core contraction: 2e-2 (tests/test_gpu_precision.py
    # bounds it per result)
    rtol = 2e-2 if prec == ts.TS_PREC_TF32 else 1e-5
    assert_sinr_close(got, ref, rtol, what=case.w.name)


def test_batch_matches_single_calls_and_oracle():
    systems = _systems()
    insts, outs, keep = _instances(systems)
    ws = ts.batch_workspace(insts)
    plan = ts.BatchPlan(insts, ws)
    plan.launch()
    torch.cuda.synchronize()
    for (case, op, prec), (sinr, flags), (_, Pt) in zip(systems, outs, keep):
        got = sinr.cpu().numpy().astype(np.float64)
        assert np.all((flags.cpu().numpy() & ts.TS_FLAG_ERRORS) == 0)
        np.testing.assert_array_equal(got, _single(case, op, prec, Pt))
        _check_oracle(case, op, got, prec)
    # a replay reads the inputs again: halve every noise power in place
    for case, _, _ in systems:
        case.sig.mul_(0.5)
        case.s2 = case.s2 * 0.5
    for sinr, _ in outs:
        sinr.fill_(float("nan"))
    plan.launch()
    torch.cuda.synchronize()
    for (case, op, prec), (sinr, _), (_, Pt) in zip(systems, outs, keep):
        got = sinr.cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(got, _single(case, op, prec, Pt))
    plan.close()


def test_autotuned_batch(tmp_path):
    systems = _systems(count=6, seed=11)
    insts, outs, keep = _instances(systems)
    ws = ts.batch_workspace(insts)
    plan = ts.BatchPlan(insts, ws, autotune=True)
    plan.launch()
    torch.cuda.synchronize()
    for (case, op, prec), (sinr, _), _ in zip(systems, outs, keep):
        _check_oracle(case, op, sinr.cpu().numpy().astype(np.float64), prec)
    path = tmp_path / "tuning.txt"
    assert ts.load().ts_autotune_save(str(path).encode()) == 0
    # every SVD shape class of the batch has an entry
    lines = path.read_text().splitlines()
    keys = {f"op0_prec{prec}_J{c.w.J}_m{c.w.m}_n{c.w.n}_p{c.w.p}_P{c.w.P}_L{c.w.L}_K{c.w.K}_coef1"
            for c, op, prec in systems if op == ts.TS_OP_SINR_SVD}
    assert keys <= {ln.split()[0] for ln in lines}
    plan.close()


def test_batch_with_wide_and_large_instances():
    # a batch mixing a narrow system, a wide-core one (p = 48 of P = 64) and
    # one with 24 receive rows: each instance equals its single call
    base = dict(n_los=2, pdp_decay_s=300e-9, sigma2=None, sigma2_range=(1e-3, 1.0))
    ws_ = [dataclasses.replace(synth.SMALL, name="narrow", J=3, K=50, seed=201, **base),
           dataclasses.replace(synth.SMALL, name="wide", J=3, M=8, m=8, N=64, n=24, P=64, p=48,
                               L=4, K=70, seed=202, **base),
           dataclasses.replace(synth.SMALL, name="large", J=2, M=32, m=24, N=64, n=40, P=32, p=16,
                               L=4, K=33, seed=203, **base)]
    systems = [(Case(w), ts.TS_OP_SINR_SVD, ts.TS_PREC_FP32) for w in ws_]
    insts, outs, keep = _instances(systems)
    plan = ts.BatchPlan(insts, ts.batch_workspace(insts))
    plan.launch()
    torch.cuda.synchronize()
    for (case, op, prec), (sinr, flags), (_, Pt) in zip(systems, outs, keep):
        got = sinr.cpu().numpy().astype(np.float64)
        assert np.all((flags.cpu().numpy() & ts.TS_FLAG_ERRORS) == 0)
        np.testing.assert_array_equal(got, _single(case, op, prec, Pt))
    plan.close()
