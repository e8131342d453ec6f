"""Host logic of the multi-device partition (paper_2401_09792_gb300.partition)
as two gloo ranks on the CPU.

SINR: the subcarrier ranges cover [0, K) once, in order, balanced; each rank
evaluates its range of one system (here the FP64 oracle stands in for the
device call, whose range form is checked against the whole call on the GPU
in tests/test_gpu_partition.py) and gather_sinr reassembles the whole
system's SINR on every rank, equal to one evaluation of all subcarriers.

Fit: the summed mode Grams of eq. (20)-(21) -- over the BSs k for A_i, over
the UEs i for B_k -- from each rank's channel shard, all-reduced, equal the
Grams of all channels."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2401_09792_gb300 import partition  # noqa: E402


@pytest.mark.parametrize("K,world", [(64, 2), (70, 3), (5, 5), (1, 1), (3300, 8)])
def test_subcarrier_ranges_cover_and_balance(K, world):
    r = partition.subcarrier_ranges(K, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == K
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [k1 - k0 for k0, k1 in r]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def test_channel_shards_partition_the_links():
    J, world = 5, 3
    seen = sorted(ch for r in range(world) for ch in partition.channel_shard(J, r, world))
    assert seen == [(i, k) for i in range(J) for k in range(J)]


def _system():
    import dataclasses
    from paper_2401_09792_gb300 import synth
    return dataclasses.replace(synth.SMALL, J=3, K=37)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from oracle import sinr as S
    from oracle import tucker as T
    from paper_2401_09792_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _system()
        tk = synth.direct_tucker(w)
        alpha, tau = synth.path_gains_delays(w)
        s2 = synth.noise_powers(w)
        k0, k1 = partition.subcarrier_ranges(w.K, world)[rank]
        coef = S.coefficients(alpha, tau, w.K, w.delta_f_hz)[:, :, k0:k1]
        local = torch.from_numpy(S.tucker_sinr(tk["G"], tk["C"], coef, s2, w.L, "svd"))
        whole = partition.gather_sinr(local, w.K).numpy()
        # summed mode-1 and mode-2 Grams of eq. (20)-(21) over this rank's links
        X = synth.channel_submatrices(w)
        gA = torch.zeros(w.J, w.M, w.M, dtype=torch.complex128)
        gB = torch.zeros(w.J, w.N, w.N, dtype=torch.complex128)
        for i, k in partition.channel_shard(w.J, rank, world):
            X1 = T.unfold(X[i, k], 0)
            X2 = T.unfold(X[i, k], 1)
            gA[i] += torch.from_numpy(X1 @ X1.conj().T)
            gB[k] += torch.from_numpy(X2 @ X2.conj().T)
        partition.allreduce_grams([gA, gB])
        out.put((rank, whole, gA.numpy(), gB.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_split_gather_and_gram_sums():
    from oracle import sinr as S
    from oracle import tucker as T
    from paper_2401_09792_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _system()
    tk = synth.direct_tucker(w)
    alpha, tau = synth.path_gains_delays(w)
    ref = S.tucker_sinr(tk["G"], tk["C"], S.coefficients(alpha, tau, w.K, w.delta_f_hz),
                        synth.noise_powers(w), w.L, "svd")
    X = synth.channel_submatrices(w)
    gA = np.stack([sum(T.unfold(X[i, k], 0) @ T.unfold(X[i, k], 0).conj().T for k in range(w.J))
                   for i in range(w.J)])
    gB = np.stack([sum(T.unfold(X[i, k], 1) @ T.unfold(X[i, k], 1).conj().T for i in range(w.J))
                   for k in range(w.J)])
    for rank, whole, a, b in res:
        # the gathered ranges are the whole system (each unit is independent)
        np.testing.assert_allclose(whole, ref, rtol=1e-12)
        np.testing.assert_allclose(a, gA, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(b, gB, rtol=1e-12, atol=1e-9)
