"""The paper-scale system (J = 21 cells, (M, N, P) = (8, 256, 401), compressed
sizes (8, 130, 120), K = 64 subcarriers, L = 4) with two UEs per cell, in the
launch configuration the benchmark times (ts_sinr_svd_multiuser, wide-core
kernel), checked on sampled subcarriers against the FP64 oracle
(oracle.sinr.tucker_sinr_multiuser on the same UE groups), every sampled
SINR within 1e-5 relative (the FP32 bound)."""
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


def test_paper_scale_two_ue_groups_sampled():
    w = dataclasses.replace(synth.PAPER_U5, U=2)
    U, J, K, L, P, m, n, p = w.U, w.J, w.K, w.L, w.P, w.m, w.n, w.p
    nl = J * J
    tks = [synth.direct_tucker(w, ue=u) for u in range(U)]
    pg = [synth.path_gains_delays(w, ue=u) for u in range(U)]
    s2 = np.stack([synth.noise_powers(w, ue=u) for u in range(U)])
    d = ts.Dims.of(w)
    Gd = torch.cat([ts.core_to_device(t["G"]) for t in tks])
    Cd = torch.cat([ts.factor_to_device(t["C"].reshape(nl, P, p)) for t in tks])
    ad = torch.cat([ts.factor_to_device(a.reshape(nl, P)) for a, _ in pg])
    td = torch.cat([ts.real_to_device(t.reshape(nl, P)) for _, t in pg])
    sd = ts.real_to_device(s2.reshape(U * J))
    cs, keep = ts.make_coef(alpha=ad, tau=td)
    sinr = torch.full((U, J, K, L), float("nan"), device="cuda")
    flags = torch.full((U, J, K), 255, dtype=torch.uint8, device="cuda")
    ws = ts.workspace(d, ts.TS_OP_SINR_SVD_MULTIUSER)
    ts.ts_sinr_svd_multiuser(d, U, cs, Gd, Cd, sd, sinr, flags, ws)
    torch.cuda.synchronize()
    got = sinr.cpu().numpy().astype(np.float64)
    assert np.all((flags.cpu().numpy() & ts.TS_FLAG_ERRORS) == 0)
    assert np.all(np.isfinite(got))
    del keep

    ks = [0, 31, 63]
    coef = np.stack([S.coefficients(a, t, K, w.delta_f_hz)[:, :, ks] for a, t in pg])
    G = np.stack([t["G"] for t in tks])
    C = np.stack([t["C"] for t in tks])
    ref = S.tucker_sinr_multiuser(G, C, coef, s2, L)
    assert_sinr_close(got[:, :, ks], ref, what="paper scale, two UE groups")
