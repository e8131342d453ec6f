"""Shared set-up for the GPU parity tests: seeded inputs through the oracle
(expected values) and through the C ABI (device results)."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from oracle import sinr as S
from paper_2401_09792_gb300 import synth
from paper_2401_09792_gb300 import tuckersinr as ts

# Parity bound of the FP32 path: relative SINR error against the FP64 oracle,
# per SINR, flat (the target precision of the method's FP32 evaluation).
FP32_RTOL = 1e-5


def assert_sinr_close(got: np.ndarray, ref: np.ndarray, rtol=FP32_RTOL, what: str = "") -> np.ndarray:
    """Element-by-element relative error |got - ref| / |ref| within `rtol`
    (a scalar or an array broadcast against the SINRs); returns the errors."""
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite SINR"
    rel = np.abs(got - ref) / np.abs(ref)
    tol = np.broadcast_to(rtol, rel.shape)
    bad = rel > tol
    if bad.any():
        at = np.unravel_index(np.argmax(rel / tol), rel.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {rel.size} SINRs beyond the bound; "
                             f"max rel {rel.max():.3e} (bound there {tol[at]:.3e}) at {at}; "
                             f"p99 {np.quantile(rel, 0.99):.3e}")
    return rel


def weak_stream_rtol(case, dense: bool = False, precoder: str = "svd") -> np.ndarray:
    """The FP32 bound per SINR (J, K, L) for SVD precoding: FP32_RTOL, plus
    4 u sigma_1 / sigma_r for a stream whose serving singular value sigma_r
    is below 1e-2 sigma_1.  Such a stream's SINR is fixed by the complex64
    inputs only to about that: the FP32 rounding of the compressed channel
    moves sigma_r by ~u sigma_1, whatever the algorithm.  Other streams keep
    the flat bound."""
    w = case.w
    tol = np.full((w.J, w.K, w.L), FP32_RTOL)
    if precoder != "svd":
        return tol
    Hs = S.dense_channels(case.X, case.coef) if dense else \
        S.compressed_channels(case.tk["G"], case.tk["C"], case.coef)
    for i in range(w.J):
        sv = np.linalg.svd(Hs[i, i], compute_uv=False)[:, :w.L]      # (K, L)
        ratio = sv[:, :1] / np.maximum(sv, 1e-300)
        tol[i] = np.where(ratio > 1e2, FP32_RTOL + 4 * 2.0 ** -24 * ratio, FP32_RTOL)
    return tol


def workload(base: synth.Workload, **kw) -> synth.Workload:
    return dataclasses.replace(base, **kw)


class Case:
    """One synthetic system: host (float64) arrays and device (complex64) copies."""

    def __init__(self, w: synth.Workload, dev="cuda"):
        self.w = w
        self.tk = synth.direct_tucker(w)
        self.alpha, self.tau = synth.path_gains_delays(w)
        self.s2 = synth.noise_powers(w)
        self.Pw = synth.wideband_precoders(w)
        self.coef = S.coefficients(self.alpha, self.tau, w.K, w.delta_f_hz)
        self.Ptn = np.stack([S.project_precoder(self.tk["B"][k], self.Pw[k]) for k in range(w.J)])
        J, P = w.J, w.P
        self.d = ts.Dims.of(w)
        self.dev = dev
        self.G = ts.core_to_device(self.tk["G"], dev)
        self.C = ts.factor_to_device(self.tk["C"].reshape(J * J, P, w.p), dev)
        self.c = ts.factor_to_device(self.coef.reshape(J * J, w.K, P), dev)
        self.al = ts.factor_to_device(self.alpha.reshape(J * J, P), dev)
        self.ta = ts.real_to_device(self.tau.reshape(J * J, P), dev)
        self.sig = ts.real_to_device(self.s2, dev)
        self.B = ts.factor_to_device(self.tk["B"], dev)
        self.Pf = ts.factor_to_device(self.Pw, dev)

    def coef_struct(self, mode: str):
        if mode == "dense":
            return ts.make_coef(c=self.c)
        return ts.make_coef(alpha=self.al, tau=self.ta)

    def gpu_sinr(self, precoder: str, mode: str = "paths"):
        w = self.w
        cs, keep = self.coef_struct(mode)
        sinr = torch.full((w.J, w.K, w.L), float("nan"), device=self.dev)
        flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device=self.dev)
        if precoder == "svd":
            ws = ts.workspace(self.d, ts.TS_OP_SINR_SVD, self.dev)
            ts.ts_sinr_svd(self.d, cs, self.G, self.C, self.sig, sinr, flags, ws)
        else:
            Pt = torch.empty(w.J, w.n, w.L, dtype=torch.complex64, device=self.dev)
            ts.ts_project_precoder(self.d, self.B, self.Pf, Pt)
            ws = ts.workspace(self.d, ts.TS_OP_SINR_MMSE, self.dev)
            ts.ts_sinr_mmse(self.d, cs, self.G, self.C, Pt, self.sig, sinr, flags, ws)
        torch.cuda.synchronize()
        del keep
        return sinr.cpu().numpy().astype(np.float64), flags.cpu().numpy()

    def with_channels(self, X=None):
        """Attach dense channels (default: drawn by the channel model) for the
        dense-comparator path."""
        self.X = synth.channel_submatrices(self.w) if X is None else X
        self.Xd = ts.channels_to_device(self.X, self.dev)
        return self

    def gpu_dense_sinr(self, precoder: str, mode: str = "paths"):
        w = self.w
        cs, keep = self.coef_struct(mode)
        sinr = torch.full((w.J, w.K, w.L), float("nan"), device=self.dev)
        flags = torch.full((w.J, w.K), 255, dtype=torch.uint8, device=self.dev)
        if precoder == "svd":
            ws = ts.workspace(self.d, ts.TS_OP_DENSE_SVD, self.dev)
            ts.ts_dense_sinr_svd(self.d, cs, self.Xd, self.sig, sinr, flags, ws)
        else:
            ws = ts.workspace(self.d, ts.TS_OP_DENSE_MMSE, self.dev)
            ts.ts_dense_sinr_mmse(self.d, cs, self.Xd, self.Pf, self.sig, sinr, flags, ws)
        torch.cuda.synchronize()
        del keep
        return sinr.cpu().numpy().astype(np.float64), flags.cpu().numpy()

    def oracle_dense_sinr(self, precoder: str):
        Pw = self.Pw if precoder == "mmse" else None
        return S.dense_sinr(self.X, self.coef, self.s2, self.w.L, precoder, Pw)

    def oracle_sinr(self, precoder: str):
        Pt = self.Ptn if precoder == "mmse" else None
        return S.tucker_sinr(self.tk["G"], self.tk["C"], self.coef, self.s2, self.w.L, precoder, Pt)


def svd_gap(case: Case, dense: bool = False) -> np.ndarray:
    """Smallest relative gap between the squared singular values that the SVD
    precoder must separate (within the top L, and between L and L+1), over all
    serving links, per subcarrier: (K,)."""
    w = case.w
    gaps = np.full(w.K, np.inf)
    if dense:
        Hs = S.dense_channels(case.X, case.coef)
    else:
        Hs = S.compressed_channels(case.tk["G"], case.tk["C"], case.coef)
    for k in range(w.J):
        sv = np.linalg.svd(Hs[k, k], compute_uv=False) ** 2          # (K, min(m, n))
        top = sv[:, :min(w.L + 1, sv.shape[1])]
        d = -np.diff(top, axis=1) / sv[:, :1]
        if d.shape[1]:
            gaps = np.minimum(gaps, d.min(axis=1))
    return gaps


def interference_condition(case: Case, precoder: str, dense: bool = False) -> np.ndarray:
    """2-norm condition number of each UE's interference-plus-noise covariance
    R_i(kappa) = sum_{k != i} E_ik E_ik* + sigma_i^2 I (eq. 4 / eq. 25 without the
    serving term), from the oracle: (J, K).  FP32 rounding of the effective
    channels perturbs the SINR by up to ~u cond(R) relative."""
    w = case.w
    if dense:
        Hs = S.dense_channels(case.X, case.coef)
        Pw = case.Pw
    else:
        Hs = S.compressed_channels(case.tk["G"], case.tk["C"], case.coef)
        Pw = case.Ptn
    V = S._precoders(Hs, w.L, precoder, Pw if precoder == "mmse" else None)
    E = S.effective_channels(Hs, V)
    Q = S.covariance(E, case.s2)
    out = np.empty((w.J, w.K))
    for i in range(w.J):
        R = Q[i] - E[i, i] @ np.conj(np.swapaxes(E[i, i], 1, 2))
        out[i] = np.linalg.cond(R)
    return out
