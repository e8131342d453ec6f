"""Host logic of bench.py's multi-rank path (one process per GPU, weak
scaling), run as two gloo ranks on the CPU: every rank gets the slowest
rank's time, the whole-job value counts all ranks' units, the ranks share
one system (same draws) and evaluate disjoint subcarrier ranges that cover
it, and the reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2401_09792_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 7.5 * rank
        slowest = bench.max_over_ranks(local_ms, world)
        w = bench.partition_workload(world)
        alpha, _ = synth.path_gains_delays(w)
        k0, k1 = bench.rank_range(rank, world)
        out.put((rank, slowest, (k0, k1, w.K), complex(alpha.ravel()[0]),
                 bench.whole_job_value(world, k1 - k0, 3, slowest)))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_subcarrier_partition():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, g0, a0, v0), (r1, t1, g1, a1, v1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 17.5                       # both ranks see the slowest rank's time
    assert a0 == a1                               # one shared system
    import bench
    w = bench.WORKLOAD
    # disjoint ranges of WORKLOAD.K subcarriers covering the shared 2 K
    assert g0 == (0, w.K, 2 * w.K) and g1 == (w.K, 2 * w.K, 2 * w.K)
    assert v0 == v1 == pytest.approx(2 * w.K * 3 / 17.5e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_value(1, 8192, 10, 2.0) == pytest.approx(8192 * 10 / 2e-3)


def test_reference_arm_only_on_rank_zero():
    env = {**os.environ, "RANK": "1", "WORLD_SIZE": "2"}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
