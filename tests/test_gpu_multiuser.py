"""Several UEs per cell with first-UE inter-cell interference (Section 4),
ts_sinr_svd_multiuser and ts_dense_sinr_svd_multiuser, against the FP64
oracle (oracle.sinr.tucker_sinr_multiuser / dense_sinr_multiuser) on the same
inputs, every SINR within 1e-5 relative (the FP32 bound of the single-UE
tests).  U = 1 must give ts_sinr_svd's result bit for bit."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinr as S  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402
from paper_2401_09792_gb300 import tuckersinr as ts  # noqa: E402
from tests.gpu_inputs import assert_sinr_close  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


class System:
    """U UE groups of one synthetic system: host arrays and device copies."""

    def __init__(self, w, U, dense=False):
        self.w, self.U = w, U
        tks = [synth.direct_tucker(w, ue=u) for u in range(U)]
        pg = [synth.path_gains_delays(w, ue=u) for u in range(U)]
        self.G = np.stack([t["G"] for t in tks])
        self.C = np.stack([t["C"] for t in tks])
        self.alpha = np.stack([a for a, _ in pg])
        self.tau = np.stack([t for _, t in pg])
        self.s2 = np.stack([synth.noise_powers(w, ue=u) for u in range(U)])
        self.coef = np.stack([S.coefficients(self.alpha[u], self.tau[u], w.K, w.delta_f_hz)
                              for u in range(U)])
        J, P = w.J, w.P
        self.d = ts.Dims.of(w)
        self.Gd = torch.cat([ts.core_to_device(self.G[u]) for u in range(U)])
        self.Cd = ts.factor_to_device(self.C.reshape(U * J * J, P, w.p))
        self.cd = ts.factor_to_device(self.coef.reshape(U * J * J, w.K, P))
        self.ad = ts.factor_to_device(self.alpha.reshape(U * J * J, P))
        self.td = ts.real_to_device(self.tau.reshape(U * J * J, P))
        self.sd = ts.real_to_device(self.s2.reshape(U * J))
        if dense:
            self.X = np.stack([synth.channel_submatrices(w, ue=u) for u in range(U)])
            self.Xd = torch.cat([ts.channels_to_device(self.X[u]) for u in range(U)])

    def coef_struct(self, mode):
        return ts.make_coef(c=self.cd) if mode == "dense" else ts.make_coef(alpha=self.ad, tau=self.td)

    def gpu(self, mode="paths", dense=False, U=None, per_group_ws=False):
        w, U = self.w, U or self.U
        cs, keep = self.coef_struct(mode)
        sinr = torch.full((U, w.J, w.K, w.L), float("nan"), device="cuda")
        flags = torch.full((U, w.J, w.K), 255, dtype=torch.uint8, device="cuda")
        if dense:
            ws = ts.workspace(self.d, ts.TS_OP_DENSE_SVD_MULTIUSER)
            ts.ts_dense_sinr_svd_multiuser(self.d, U, cs, self.Xd, self.sd, sinr, flags, ws)
        else:
            ws = ts.workspace(self.d, ts.TS_OP_SINR_SVD_MULTIUSER)
            if per_group_ws:
                # one single-UE workspace per group: the groups run concurrently
                ws = torch.empty(U * (ws.numel() // 2), dtype=torch.uint8, device="cuda")
            ts.ts_sinr_svd_multiuser(self.d, U, cs, self.Gd, self.Cd, self.sd, sinr, flags, ws)
        torch.cuda.synchronize()
        del keep
        return sinr.cpu().numpy().astype(np.float64), flags.cpu().numpy()

    def channels(self, dense=False):
        if dense:
            return np.stack([S.dense_channels(self.X[u], self.coef[u]) for u in range(self.U)])
        return np.stack([S.compressed_channels(self.G[u], self.C[u], self.coef[u]) for u in range(self.U)])


def _wl(**kw):
    base = dict(name="multiuser", J=3, M=4, N=32, P=8, K=64, m=4, n=8, p=4, L=2, n_los=1,
                sigma2=None, pdp_decay_s=300e-9, seed=9)
    base.update(kw)
    return dataclasses.replace(synth.SMALL, **base)


@pytest.mark.parametrize("mode", ["paths", "dense"])
@pytest.mark.parametrize("shape", ["narrow", "wide"])
def test_multiuser_svd_sinr(shape, mode):
    w = _wl() if shape == "narrow" else _wl(M=8, m=8, N=64, n=24, P=64, p=48, L=4, K=70)
    sysm = System(w, U=3)
    got, flags = sysm.gpu(mode)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0), np.unique(flags)
    ref = S.tucker_sinr_multiuser(sysm.G, sysm.C, sysm.coef, sysm.s2, w.L)
    assert_sinr_close(got, ref, what=f"multiuser {shape} {mode}")


def test_multiuser_with_one_group_is_ts_sinr_svd():
    w = _wl()
    sysm = System(w, U=2)
    got, _ = sysm.gpu("paths", U=1)
    cs, keep = sysm.coef_struct("paths")
    one = torch.empty(w.J, w.K, w.L, device="cuda")
    nl = w.J * w.J
    ts.ts_sinr_svd(sysm.d, cs, sysm.Gd[:nl], sysm.Cd[:nl], sysm.sd[:w.J], one, None,
                   ts.workspace(sysm.d, ts.TS_OP_SINR_SVD))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got[0], one.cpu().numpy().astype(np.float64))


def test_dense_multiuser_comparator():
    w = _wl(K=40)
    sysm = System(w, U=2, dense=True)
    got, flags = sysm.gpu("paths", dense=True)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    ref = S.dense_sinr_multiuser(sysm.X, sysm.coef, sysm.s2, w.L)
    assert_sinr_close(got, ref, what="dense multiuser")


@pytest.mark.parametrize("U", [3, 6])
def test_concurrent_groups_match_sequential(U):
    # one workspace per group: groups 1.. on side streams, bit-identical
    # results (the same kernels on the same inputs)
    w = _wl(M=8, m=8, N=64, n=24, P=64, p=48, L=4, K=70)
    sysm = System(w, U=U)
    seq, _ = sysm.gpu("paths")
    con, flags = sysm.gpu("paths", per_group_ws=True)
    assert np.all((flags & ts.TS_FLAG_ERRORS) == 0)
    np.testing.assert_array_equal(con, seq)
