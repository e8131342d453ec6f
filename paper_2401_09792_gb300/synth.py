"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random draws only -- no step of the compression or of the
SINR evaluation.  Both the FP64 oracle and the CUDA path consume what it
returns, so it is the one module the two sides share.

What is drawn (Section 2.2, eq. 2 and Section 4):

* channel submatrices: ``n_los`` line-of-sight submatrices, each an outer
  product of two half-wavelength uniform-linear-array steering vectors with
  angles drawn uniformly in [-pi/2, pi/2], followed by i.i.d. CN(0, 1)
  non-line-of-sight submatrices (the paper's 3GPP TR 38.901 channels are not
  available; these stand in for them with the same shapes);
* per-path complex gains ``alpha`` and delays ``tau`` (seconds, float32
  values so that every consumer sees the same numbers);
* per-UE noise powers ``sigma2``;
* wideband precoders with orthonormal columns (Haar-random);
* a Tucker form drawn directly (orthonormal factors from QR of Gaussian
  matrices, a Gaussian core with geometric energy decay along each mode),
  used where fitting the channels would be too slow or too large.

Indexing follows the paper's groupwise model with one UE per cell: channel
(i, k) is the link from base station k to the UE of cell i.  Arrays are
complex128 / float64 here; the binding casts them to the device layout.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    """Shape and distribution of one synthetic multi-cell system."""

    name: str
    J: int            # cells = base stations = groups (one UE per cell)
    M: int            # UE (receive) antennas
    N: int            # BS (transmit) antennas
    P: int            # submatrices (paths) per channel
    K: int            # OFDM subcarriers
    m: int            # Tucker rank, mode 1
    n: int            # Tucker rank, mode 2
    p: int            # Tucker rank, mode 3
    L: int            # spatial streams per UE
    n_los: int = 1    # LOS submatrices among the P
    tau_max_s: float = 1e-6
    pdp_decay_s: float | None = None    # exponential power-delay profile of alpha
    sigma2: float | None = 0.1          # fixed noise power, or None -> log-uniform
    sigma2_range: tuple = (1e-3, 1.0)
    delta_f_hz: float = 15e3
    seed: int = 0
    U: int = 1        # UEs per cell (UE groups; group 0 = the first UE of every cell)
    # NLOS submatrices: None = i.i.d. CN(0, 1) entries; (rho_rx, rho_tx) =
    # Kronecker model R_rx^{1/2} W R_tx^{1/2} with exponential correlation
    # R[a, b] = rho^|a - b| across the UE and the BS array
    nlos_corr: tuple | None = None
    extra: dict = field(default_factory=dict)


# The paper's experiments use 3GPP channels (Section 4); these are the
# synthetic stand-ins with the shapes of the five evaluation workloads.
SMALL = Workload("small J2 M4 N32 P8 K64 r(4,8,4) L2", J=2, M=4, N=32, P=8, K=64,
                 m=4, n=8, p=4, L=2, n_los=1, sigma2=0.1)
MID = Workload("mid J8 M8 N256 P32 K1024 r(8,32,16) L8", J=8, M=8, N=256, P=32, K=1024,
               m=8, n=32, p=16, L=8, n_los=2, pdp_decay_s=300e-9, sigma2=None)
PRECISION = Workload("precision J16 M16 N512 P64 K2048 r(16,64,32) L8", J=16, M=16, N=512,
                     P=64, K=2048, m=16, n=64, p=32, L=8, n_los=2, pdp_decay_s=300e-9,
                     sigma2=None, sigma2_range=(1e-4, 1e-1))
DIFFERENTIATION = Workload("diff J16 M16 N1024 P64 K3300 r(16,96,32) L8", J=16, M=16, N=1024,
                           P=64, K=3300, m=16, n=96, p=32, L=8, n_los=2,
                           pdp_decay_s=300e-9, sigma2=None)

# The paper's own system sizes (Section 4, table of compression results,
# (M, N, P) = (8, 256, 401)): 21 cells with 5 or 10 UEs per cell and the
# compressed sizes the paper tunes for them; the paper gives no subcarrier
# count or stream count, so K = 64 subcarriers and L = 4 streams.
PAPER_U5 = Workload("paper J21 U5 M8 N256 P401 K64 r(8,130,120) L4", J=21, M=8, N=256, P=401,
                    K=64, m=8, n=130, p=120, L=4, n_los=2, pdp_decay_s=300e-9, sigma2=None, U=5)
PAPER_U10 = Workload("paper J21 U10 M8 N256 P401 K64 r(8,140,140) L4", J=21, M=8, N=256, P=401,
                     K=64, m=8, n=140, p=140, L=4, n_los=2, pdp_decay_s=300e-9, sigma2=None, U=10)

# The paper's larger channels ((M, N, P) = (64, 512, 401)) with the first
# row of its table: 5 UEs per cell and ranks (60, 230, 150); L = 8 streams.
PAPER64_U5 = Workload("paper64 J21 U5 M64 N512 P401 K64 r(60,230,150) L8", J=21, M=64, N=512,
                      P=401, K=64, m=60, n=230, p=150, L=8, n_los=2, pdp_decay_s=300e-9,
                      sigma2=None, U=5)

# The same channels and ranks with 8 cells: a few GB on the device, the
# size for profiling the 64-row kernels.
PAPER64_J8 = replace(PAPER64_U5, name="paper64-j8 J8 U5 M64 N512 P401 K64 r(60,230,150) L8", J=8)

# The mid system with spatially correlated NLOS submatrices (exponential
# correlation 0.7 across the 8 UE antennas, 0.95 across the 256 BS antennas):
# compressible in modes 1 and 2, as measured array channels are.
MID_CORR = replace(MID, name="mid-corr J8 M8 N256 P32 K1024 r(8,32,16) L8 rho(0.7,0.95)",
                   nlos_corr=(0.7, 0.95))

WORKLOADS = {"small": SMALL, "mid": MID, "precision": PRECISION, "diff": DIFFERENTIATION,
             "paper_u5": PAPER_U5, "paper_u10": PAPER_U10, "paper64_u5": PAPER64_U5,
             "paper64_j8": PAPER64_J8, "mid_corr": MID_CORR}


def _rng(seed: int, *path: int) -> np.random.Generator:
    """Independent PCG64 stream for one (seed, path...) key."""
    ss = np.random.SeedSequence([int(seed)] + [int(x) for x in path])
    return np.random.Generator(np.random.PCG64(ss))


def _cn(rng: np.random.Generator, shape, var: float = 1.0) -> np.ndarray:
    """Circularly-symmetric complex Gaussian CN(0, var)."""
    s = np.sqrt(var / 2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def _ula(n: int, theta: float) -> np.ndarray:
    """Half-wavelength ULA steering vector, unit-modulus entries."""
    return np.exp(1j * np.pi * np.arange(n) * np.sin(theta))


def ue_key(ue: int) -> tuple:
    """Extra seed-path entries of UE group `ue` (UE ue of every cell); the
    first UEs (ue = 0) draw exactly the single-UE system."""
    return () if ue == 0 else (1000 + int(ue),)


def channel_submatrices(w: Workload, ue: int = 0) -> np.ndarray:
    """X[i, k] in C^{M x N x P}: the submatrices of eq. (2) stacked on mode 3,
    for UE `ue` of every cell.

    Returns shape (J, J, M, N, P), complex128.
    """
    X = np.empty((w.J, w.J, w.M, w.N, w.P), dtype=np.complex128)
    if w.nlos_corr is not None:
        Sr, St = (_exp_corr_sqrt(d, rho) for d, rho in zip((w.M, w.N), w.nlos_corr))
    for i in range(w.J):
        for k in range(w.J):
            rng = _rng(w.seed, 1, i, k, *ue_key(ue))
            for q in range(w.P):
                if q < w.n_los:
                    th, ph = rng.uniform(-np.pi / 2, np.pi / 2, 2)
                    X[i, k, :, :, q] = np.outer(_ula(w.M, th), np.conj(_ula(w.N, ph)))
                elif w.nlos_corr is None:
                    X[i, k, :, :, q] = _cn(rng, (w.M, w.N))
                else:
                    X[i, k, :, :, q] = Sr @ _cn(rng, (w.M, w.N)) @ St
    return X


def _exp_corr_sqrt(d: int, rho: float) -> np.ndarray:
    """Symmetric square root of the d x d exponential correlation matrix
    R[a, b] = rho^|a - b| (real, positive definite for 0 <= rho < 1)."""
    a = np.arange(d)
    R = float(rho) ** np.abs(a[:, None] - a[None, :])
    lam, V = np.linalg.eigh(R)
    return (V * np.sqrt(np.maximum(lam, 0.0))) @ V.T


def path_gains_delays(w: Workload, ue: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """alpha[i, k, P] complex128 and tau[i, k, P] seconds (float32 values)."""
    alpha = np.empty((w.J, w.J, w.P), dtype=np.complex128)
    tau = np.empty((w.J, w.J, w.P), dtype=np.float64)
    for i in range(w.J):
        for k in range(w.J):
            rng = _rng(w.seed, 2, i, k, *ue_key(ue))
            t = rng.uniform(0.0, w.tau_max_s, w.P).astype(np.float32).astype(np.float64)
            var = np.ones(w.P) if w.pdp_decay_s is None else np.exp(-t / w.pdp_decay_s)
            a = _cn(rng, w.P) * np.sqrt(var)
            alpha[i, k] = a.astype(np.complex64).astype(np.complex128)
            tau[i, k] = t
    return alpha, tau


def noise_powers(w: Workload, ue: int = 0) -> np.ndarray:
    """sigma2[i] per UE (float32 values)."""
    if w.sigma2 is not None:
        return np.full(w.J, np.float32(w.sigma2), dtype=np.float64)
    rng = _rng(w.seed, 3, *ue_key(ue))
    lo, hi = np.log(w.sigma2_range[0]), np.log(w.sigma2_range[1])
    return np.exp(rng.uniform(lo, hi, w.J)).astype(np.float32).astype(np.float64)


def orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Haar-distributed matrix with orthonormal columns (QR of a Gaussian)."""
    Z = _cn(rng, (rows, cols))
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def direct_tucker_device(w: Workload, decay=(0.85, 0.97, 0.9), ue: int = 0, device="cuda") -> dict:
    """The Tucker form of direct_tucker drawn on the device with PyTorch's
    seeded generator (same distribution, other values), for systems whose
    cores hold billions of entries: A [J][M][m], B [J][N][n] (shared by the
    UE groups), C [J*J][P][p], G [J*J][p][m][n] (the library's layouts),
    complex64 device tensors."""
    import torch
    gen = torch.Generator(device=device)

    def seeded(*path):
        ss = np.random.SeedSequence([int(w.seed)] + [int(x) for x in path])
        gen.manual_seed(int(ss.generate_state(1, dtype=np.uint64)[0] >> 1))
        return gen

    def orth(batch, rows, cols, *path):
        z = torch.randn(batch, rows, cols, dtype=torch.complex64, device=device, generator=seeded(*path))
        q, r = torch.linalg.qr(z)
        d = torch.diagonal(r, dim1=-2, dim2=-1)
        return (q * (d / d.abs()).unsqueeze(-2)).contiguous()

    J, nl = w.J, w.J * w.J
    sa = torch.tensor(decay[0], device=device) ** torch.arange(w.m, device=device)
    sb = torch.tensor(decay[1], device=device) ** torch.arange(w.n, device=device)
    sq = torch.tensor(decay[2], device=device) ** torch.arange(w.p, device=device)
    scale = sq[:, None, None] * sa[None, :, None] * sb[None, None, :]          # [p][m][n]
    G = torch.randn(nl, w.p, w.m, w.n, dtype=torch.complex64, device=device,
                    generator=seeded(8, *ue_key(ue))) * scale
    return {"A": orth(J, w.M, w.m, 5, *ue_key(ue)), "B": orth(J, w.N, w.n, 6),
            "C": orth(nl, w.P, w.p, 7, *ue_key(ue)), "G": G}


def wideband_precoders(w: Workload) -> np.ndarray:
    """P_k in C^{N x L} with orthonormal columns, shape (J, N, L)."""
    return np.stack([orthonormal(_rng(w.seed, 4, k), w.N, w.L) for k in range(w.J)])


def direct_tucker(w: Workload, decay=(0.85, 0.97, 0.9), ue: int = 0) -> dict:
    """A Tucker form drawn directly, without fitting any channel.

    A[i] (M x m), B[k] (N x n), C[i, k] (P x p) have orthonormal columns;
    G[i, k] (m x n x p) is CN(0, 1) scaled by decay[0]**a * decay[1]**b *
    decay[2]**q along its three modes.  All values are complex64-representable.
    For UE group `ue` the receive factors A, the C and the cores are its own;
    the transmit factors B (one per BS) are the same for every group.
    """
    A = np.stack([orthonormal(_rng(w.seed, 5, i, *ue_key(ue)), w.M, w.m) for i in range(w.J)])
    B = np.stack([orthonormal(_rng(w.seed, 6, k), w.N, w.n) for k in range(w.J)])
    C = np.empty((w.J, w.J, w.P, w.p), dtype=np.complex128)
    G = np.empty((w.J, w.J, w.m, w.n, w.p), dtype=np.complex128)
    sa = decay[0] ** np.arange(w.m)
    sb = decay[1] ** np.arange(w.n)
    sq = decay[2] ** np.arange(w.p)
    scale = sa[:, None, None] * sb[None, :, None] * sq[None, None, :]
    for i in range(w.J):
        for k in range(w.J):
            C[i, k] = orthonormal(_rng(w.seed, 7, i, k, *ue_key(ue)), w.P, w.p)
            G[i, k] = _cn(_rng(w.seed, 8, i, k, *ue_key(ue)), (w.m, w.n, w.p)) * scale
    c64 = lambda x: x.astype(np.complex64).astype(np.complex128)  # noqa: E731
    return {"A": c64(A), "B": c64(B), "C": c64(C), "G": c64(G)}
