"""The synthetic input generators (shared by the oracle and the GPU tests):
seeded reproducibility, UE-group independence, and the spatially correlated
NLOS option (its second-order statistics match the exponential model)."""
import dataclasses

import numpy as np

from paper_2401_09792_gb300 import synth


def test_exponential_correlation_square_root():
    S = synth._exp_corr_sqrt(9, 0.8)
    a = np.arange(9)
    np.testing.assert_allclose(S @ S, 0.8 ** np.abs(a[:, None] - a[None, :]), atol=1e-12)
    np.testing.assert_allclose(S, S.T, atol=0)


def test_correlated_nlos_second_order_statistics():
    w = dataclasses.replace(synth.SMALL, J=3, M=6, N=12, P=200, n_los=1, nlos_corr=(0.5, 0.9))
    X = synth.channel_submatrices(w)[:, :, :, :, 1:]                 # NLOS only
    Y = np.moveaxis(X, 4, 2).reshape(-1, w.M, w.N)                   # samples of M x N
    a_r, a_t = np.arange(w.M), np.arange(w.N)
    Rt = np.einsum("sab,sac->bc", Y, Y.conj()) / (Y.shape[0] * w.M)
    Rr = np.einsum("sab,scb->ac", Y, Y.conj()) / (Y.shape[0] * w.N)
    assert np.max(np.abs(Rt - 0.9 ** np.abs(a_t[:, None] - a_t[None, :]))) < 0.06
    assert np.max(np.abs(Rr - 0.5 ** np.abs(a_r[:, None] - a_r[None, :]))) < 0.06


def test_seeds_and_ue_groups():
    w = dataclasses.replace(synth.SMALL, J=2)
    np.testing.assert_array_equal(synth.channel_submatrices(w), synth.channel_submatrices(w))
    t0, t1 = synth.direct_tucker(w, ue=0), synth.direct_tucker(w, ue=1)
    np.testing.assert_array_equal(t0["B"], t1["B"])               # one B per BS for every UE
    assert not np.allclose(t0["A"], t1["A"]) and not np.allclose(t0["G"], t1["G"])
    assert not np.allclose(synth.noise_powers(dataclasses.replace(w, sigma2=None), ue=1),
                           synth.noise_powers(dataclasses.replace(w, sigma2=None), ue=0))
