"""Reduced-precision modes of the SVD-precoded SINR (ts_sinr_svd_prec): the
interfering links' core contraction H~ = G x_3 (c* C) (eq. 15) on the tensor
cores in TF32 or in BF16 with split high and low parts, against the FP64
oracle.

Per-result bound.  With e the relative error bound of one product w_q G_q in
the mode (TF32: both operands rounded to 11 significant bits, e = 2^-10;
BF16X2: hi*hi + lo*hi + hi*lo drops lo*lo and the residuals of the split,
e = 3 * 2^-16; TF32X3: the same with 11-bit parts, e = 2^-20 including the
tensor cores' FP32 accumulation), each interfering effective channel moves by
||dE_ik|| <= e gamma_ik ||H~_ik||_F with gamma_ik = ||sum_q |w_q| |G_q| ||_F /
||H~_ik||_F (the cancellation in the sum over the core slabs), so the
interference covariance moves by ||dR|| <= 2 e sum_k gamma_ik ||H~_ik||_F^2.
The SINR is a function of Z*Z = E_ii* R^{-1} E_ii, whose relative change is
at most eps = ||dR|| / lambda_min(R); the test allows 2 eps on top of the flat
FP32 bound 1e-5 of tests/test_gpu_sinr.py.  Every mode also has to differ from the
FP32 path (the tensor-core kernel really ran) and BF16X2 has to be more
accurate than TF32.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import FP32_RTOL, Case, assert_sinr_close, workload  # noqa: E402

E_PROD = {ts.TS_PREC_TF32: 2.0 ** -10, ts.TS_PREC_BF16X2: 3 * 2.0 ** -16, ts.TS_PREC_TF32X3: 2.0 ** -20}
OPS = {ts.TS_PREC_TF32: ts.TS_OP_SINR_SVD_TF32, ts.TS_PREC_BF16X2: ts.TS_OP_SINR_SVD_BF16X2,
       ts.TS_PREC_TF32X3: ts.TS_OP_SINR_SVD_TF32X3}
NAMES = {ts.TS_PREC_TF32: "tf32", ts.TS_PREC_BF16X2: "bf16x2", ts.TS_PREC_TF32X3: "tf32x3"}
MODES = [ts.TS_PREC_TF32, ts.TS_PREC_BF16X2, ts.TS_PREC_TF32X3]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _gpu(case: Case, prec: int, mode: str = "paths"):
    w = case.w
    cs, keep = case.coef_struct(mode)
    sinr = torch.full((w.J, w.K, w.L), float("nan"), device="cuda")
    flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device="cuda")
    op = ts.TS_OP_SINR_SVD if prec == ts.TS_PREC_FP32 else OPS[prec]
    ws = ts.workspace(case.d, op)
    ts.ts_sinr_svd_prec(case.d, cs, case.G, case.C, case.sig, prec, sinr, flags, ws)
    torch.cuda.synchronize()
    del keep
    return sinr.cpu().numpy().astype(np.float64), flags.cpu().numpy()


def _reduced_bound(case: Case, prec: int) -> np.ndarray:
    """2 eps per (UE, subcarrier), eps = ||dR|| / lambda_min(R) as above: (J, K)."""
    w = case.w
    G, C, coef = case.tk["G"], case.tk["C"], case.coef
    Hs = S.compressed_channels(G, C, coef)                        # (J, J, K, m, n)
    V = S._precoders(Hs, w.L, "svd", None)
    E = S.effective_channels(Hs, V)
    Q = S.covariance(E, case.s2)
    out = np.empty((w.J, w.K))
    for i in range(w.J):
        dR = np.zeros(w.K)
        for k in range(w.J):
            if k == i:
                continue
            wq = np.einsum("Pq,KP->Kq", C[i, k], np.conj(coef[i, k]))      # (K, p)
            absum = np.einsum("Kq,abq->Kab", np.abs(wq), np.abs(G[i, k]))   # (K, m, n)
            h2 = np.sum(np.abs(Hs[i, k]) ** 2, axis=(1, 2))
            gamma = np.sqrt(np.sum(absum ** 2, axis=(1, 2)) / np.maximum(h2, 1e-300))
            dR += 2 * E_PROD[prec] * gamma * h2
        R = Q[i] - E[i, i] @ np.conj(np.swapaxes(E[i, i], 1, 2))
        lam = np.linalg.eigvalsh(R)[:, 0]
        out[i] = 2 * dR / lam
    return out


def _check(case: Case, prec: int, mode: str = "paths"):
    got, flags = _gpu(case, prec, mode)
    ref = case.oracle_sinr("svd")
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    tol = FP32_RTOL + _reduced_bound(case, prec)
    rel = assert_sinr_close(got, ref, tol[:, :, None], what=NAMES[prec])
    return rel, got


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("mode", ["dense", "paths"])
def test_small_workload(prec, mode):
    _check(Case(synth.SMALL), prec, mode)


@pytest.mark.parametrize("prec", MODES)
def test_mid_workload_full_size(prec):
    case = Case(synth.MID)
    rel, got = _check(case, prec)
    fp32, _ = _gpu(case, ts.TS_PREC_FP32)
    # the tensor-core path ran: its results are not the FP32 ones
    assert np.max(np.abs(got - fp32) / np.abs(fp32)) > 1e-6
    print(f"\n{NAMES[prec]} mid: max {rel.max():.3e}  p99 {np.percentile(rel, 99):.3e}  "
          f"median {np.median(rel):.3e}")


def test_tf32x3_meets_the_fp32_bound():
    # three TF32 products (w_hi G_hi + w_hi G_lo + w_lo G_hi) keep ~22
    # significant bits: the SINR stays within the flat FP32 bound
    case = Case(synth.MID)
    got, flags = _gpu(case, ts.TS_PREC_TF32X3)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    rel = assert_sinr_close(got, case.oracle_sinr("svd"), what="tf32x3 mid")
    print(f"\ntf32x3 mid: max {rel.max():.3e}  p99 {np.percentile(rel, 99):.3e}")


def test_bf16x2_more_accurate_than_tf32():
    case = Case(workload(synth.MID, K=256))
    r_tf, _ = _check(case, ts.TS_PREC_TF32)
    r_bf, _ = _check(case, ts.TS_PREC_BF16X2)
    assert np.median(r_bf) < 0.1 * np.median(r_tf)


EDGE = {
    "ragged_K": dict(K=200),                      # one full tile of 128 and a ragged one
    "odd_m_n_p": dict(J=3, M=3, m=3, n=7, N=12, P=5, p=3, L=2, K=9),
    "m16_L8": dict(J=3, M=16, m=16, L=8, N=80, n=64, P=40, p=32, K=130),
    "m12_L2": dict(J=3, M=16, m=12, L=2, N=40, n=24, P=10, p=5, K=33),   # 16-lane groups, L <= 2
    "m2": dict(M=2, m=2, L=2, n=8, N=16, K=64),
    # precoder-row layouts of the link pass: rows of 6 and 4 16-byte pieces
    # (padded stride) beside the 8- and 16-piece rows (permuted) above
    "m16_L6": dict(J=3, M=16, m=16, L=6, N=48, n=40, P=20, p=12, K=140),
    "m14_L4": dict(J=3, M=16, m=14, L=4, N=40, n=30, P=16, p=9, K=129),
    "single_cell": dict(J=1, K=5),
}


@pytest.mark.parametrize("name", sorted(EDGE))
@pytest.mark.parametrize("prec", MODES)
def test_edge_cases(name, prec):
    _check(Case(workload(synth.SMALL, **EDGE[name])), prec)


def test_precision_argument_errors():
    case = Case(synth.SMALL)
    cs, keep = case.coef_struct("paths")
    w = case.w
    sinr = torch.empty(w.J, w.K, w.L, device="cuda")
    ws = ts.workspace(case.d, ts.TS_OP_SINR_SVD_BF16X2)
    with pytest.raises(ts.TsError) as e:
        ts.ts_sinr_svd_prec(case.d, cs, case.G, case.C, case.sig, 7, sinr, None, ws)
    assert e.value.status == 6
    # the FP32 workspace is too small for a tensor-core mode
    ws32 = ts.workspace(case.d, ts.TS_OP_SINR_SVD)
    with pytest.raises(ts.TsError) as e:
        ts.ts_sinr_svd_prec(case.d, cs, case.G, case.C, case.sig, ts.TS_PREC_TF32, sinr, None, ws32)
    assert e.value.status == 4
    del keep
