"""Full-size parity at the two largest single-GPU workloads, in the launch
configuration the benchmark times (path-form coefficients, whole system in
one call):

  precision        J=16, M=16, N=512, P=64, K=2048, ranks (16,64,32), L=8,
                   sigma^2 log-uniform in [1e-4, 1e-1] (FP64 refinement of
                   the ill-conditioned units at the default threshold)
  differentiation  J=16, M=16, N=1024, P=64, K=3300, ranks (16,96,32), L=8

The GPU evaluates every (UE, subcarrier); the FP64 oracle evaluates 32
subcarriers spread over the whole range (both ends, the middle, 28 drawn
from a fixed seed), and every SINR of every UE and stream there is compared
element by element: FP32 within 1e-5 relative; the tensor-core modes within
1e-5 plus the per-result bound of tests/test_gpu_precision.py; TF32X3 (three
TF32 products) also within the flat 1e-5 at the differentiation workload.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import FP32_RTOL, assert_sinr_close  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def sampled_subcarriers(K: int, count: int = 32, seed: int = 5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    fixed = {0, 1, K // 2, K - 1}
    rest = rng.choice(np.setdiff1d(np.arange(K), list(fixed)), count - len(fixed), replace=False)
    return np.sort(np.concatenate([np.array(sorted(fixed)), rest]))


class FullSystem:
    """One full-size system on the device and the oracle's inputs at the
    sampled subcarriers."""

    def __init__(self, w):
        self.w = w
        J, P = w.J, w.P
        self.tk = synth.direct_tucker(w)
        self.alpha, self.tau = synth.path_gains_delays(w)
        self.s2 = synth.noise_powers(w)
        self.ks = sampled_subcarriers(w.K)
        self.coef = S.coefficients(self.alpha, self.tau, w.K, w.delta_f_hz)[:, :, self.ks]
        self.d = ts.Dims.of(w)
        self.G = ts.core_to_device(self.tk["G"])
        self.C = ts.factor_to_device(self.tk["C"].reshape(J * J, P, w.p))
        self.al = ts.factor_to_device(self.alpha.reshape(J * J, P))
        self.ta = ts.real_to_device(self.tau.reshape(J * J, P))
        self.sig = ts.real_to_device(self.s2)

    def run(self, precoder="svd", prec=ts.TS_PREC_FP32):
        w = self.w
        cs, keep = ts.make_coef(alpha=self.al, tau=self.ta)
        sinr = torch.full((w.J, w.K, w.L), float("nan"), device="cuda")
        flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device="cuda")
        if precoder == "svd":
            op = {ts.TS_PREC_FP32: ts.TS_OP_SINR_SVD, ts.TS_PREC_TF32: ts.TS_OP_SINR_SVD_TF32,
                  ts.TS_PREC_BF16X2: ts.TS_OP_SINR_SVD_BF16X2,
                  ts.TS_PREC_TF32X3: ts.TS_OP_SINR_SVD_TF32X3}[prec]
            ws = ts.workspace(self.d, op)
            ts.ts_sinr_svd_prec(self.d, cs, self.G, self.C, self.sig, prec, sinr, flags, ws)
        else:
            Pw = synth.wideband_precoders(w)
            self.Pt_host = np.stack([S.project_precoder(self.tk["B"][k], Pw[k]) for k in range(w.J)])
            Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device="cuda")
            ts.ts_project_precoder(self.d, ts.factor_to_device(self.tk["B"]), ts.factor_to_device(Pw), Pt)
            ws = ts.workspace(self.d, ts.TS_OP_SINR_MMSE)
            ts.ts_sinr_mmse(self.d, cs, self.G, self.C, Pt, self.sig, sinr, flags, ws)
        torch.cuda.synchronize()
        del keep, ws
        got = sinr[:, torch.as_tensor(self.ks, device="cuda")].cpu().numpy().astype(np.float64)
        fl = flags.cpu().numpy()
        assert np.all((fl & ts.TS_FLAG_ERRORS) == 0), np.unique(fl)
        assert torch.isfinite(sinr).all().item()
        return got, fl[:, self.ks]

    def oracle(self, precoder="svd"):
        Pt = self.Pt_host if precoder == "mmse" else None
        return S.tucker_sinr(self.tk["G"], self.tk["C"], self.coef, self.s2, self.w.L, precoder, Pt)


@pytest.fixture(scope="module")
def precision_system():
    return FullSystem(synth.PRECISION)


@pytest.fixture(scope="module")
def diff_system():
    return FullSystem(synth.DIFFERENTIATION)


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_precision_workload_full_size(precision_system, precoder):
    sysm = precision_system
    got, flags = sysm.run(precoder)
    rel = assert_sinr_close(got, sysm.oracle(precoder), what=f"precision {precoder}")
    print(f"\nprecision {precoder}: max {rel.max():.3e} p99 {np.quantile(rel, 0.99):.3e}; "
          f"{int(np.sum((flags & ts.TS_FLAG_REFINED) != 0))} of {flags.size} sampled units refined")


@pytest.mark.parametrize("precoder", ["svd", "mmse"])
def test_differentiation_workload_full_size(diff_system, precoder):
    sysm = diff_system
    got, _ = sysm.run(precoder)
    rel = assert_sinr_close(got, sysm.oracle(precoder), what=f"differentiation {precoder}")
    print(f"\ndifferentiation {precoder}: max {rel.max():.3e} p99 {np.quantile(rel, 0.99):.3e}")


def _reduced_bound(sysm, eprod):
    """Per-result bound of a reduced-precision core contraction (as in
    tests/test_gpu_precision.py), at the sampled subcarriers: (J, k)."""
    w = sysm.w
    G, C, coef = sysm.tk["G"], sysm.tk["C"], sysm.coef
    Hs = S.compressed_channels(G, C, coef)
    V = S._precoders(Hs, w.L, "svd", None)
    E = S.effective_channels(Hs, V)
    Q = S.covariance(E, sysm.s2)
    out = np.empty((w.J, len(sysm.ks)))
    for i in range(w.J):
        dR = np.zeros(len(sysm.ks))
        for k in range(w.J):
            if k == i:
                continue
            wq = np.einsum("Pq,KP->Kq", C[i, k], np.conj(coef[i, k]))
            absum = np.einsum("Kq,abq->Kab", np.abs(wq), np.abs(G[i, k]))
            h2 = np.sum(np.abs(Hs[i, k]) ** 2, axis=(1, 2))
            gamma = np.sqrt(np.sum(absum ** 2, axis=(1, 2)) / np.maximum(h2, 1e-300))
            dR += 2 * eprod * gamma * h2
        R = Q[i] - E[i, i] @ np.conj(np.swapaxes(E[i, i], 1, 2))
        out[i] = 2 * dR / np.linalg.eigvalsh(R)[:, 0]
    return out


@pytest.mark.parametrize("prec", [ts.TS_PREC_TF32, ts.TS_PREC_BF16X2, ts.TS_PREC_TF32X3])
def test_precision_workload_tensor_core_modes(precision_system, prec):
    sysm = precision_system
    got, _ = sysm.run("svd", prec)
    eprod = {ts.TS_PREC_TF32: 2.0 ** -10, ts.TS_PREC_BF16X2: 3 * 2.0 ** -16,
             ts.TS_PREC_TF32X3: 2.0 ** -20}[prec]
    tol = FP32_RTOL + _reduced_bound(sysm, eprod)
    rel = assert_sinr_close(got, sysm.oracle("svd"), tol[:, :, None], what=f"precision prec={prec}")
    print(f"\nprecision prec={prec}: max {rel.max():.3e} p99 {np.quantile(rel, 0.99):.3e}")


def test_differentiation_workload_tf32x3_meets_the_fp32_bound(diff_system):
    sysm = diff_system
    got, _ = sysm.run("svd", ts.TS_PREC_TF32X3)
    rel = assert_sinr_close(got, sysm.oracle("svd"), what="differentiation tf32x3")
    print(f"\ndifferentiation tf32x3: max {rel.max():.3e} p99 {np.quantile(rel, 0.99):.3e}")
