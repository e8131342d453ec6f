#!/usr/bin/env python
"""Throughput of Tucker-form SINR evaluation on GB300 (subcarrier-SINRs/s).

One step = one SVD-precoded MMSE SINR evaluation of the whole system of the
largest single-GPU workload (J=16 cells, M=16, N=1024, P=64, K=3300
subcarriers, ranks (16,96,32), L=8): path coefficients (a0), projection c*C
(a1), core contraction (a2), SVD precoders through the Jacobi eigensolve
(a3), effective channels (a4), covariance (a5), Cholesky solves and SINR
(a6), all in the CUDA library, called through its C ABI.  Inputs are
resident in HBM; L2 is flushed before every timed step.  Prints one JSON
line (rank 0); the mid and precision workloads are reported in it too.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the ranks share one system of N times the subcarriers, G, C
and the path coefficients replicated, and every rank evaluates its own
range of K subcarriers (weak scaling, no collective on the data path); the
value is all ranks' SINRs divided by the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the same workload instead
(rank 0 only).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2401_09792_gb300 import synth  # noqa: E402

WORKLOAD = synth.DIFFERENTIATION  # the default line; --workload selects another
WORKLOAD_NAME = "diff"
METRIC = "subcarrier-SINRs/s"
FLUSH_BYTES = 256 << 20          # > 129 MB of L2


def select_workload(name: str):
    global WORKLOAD, WORKLOAD_NAME
    WORKLOAD, WORKLOAD_NAME = synth.WORKLOADS[name], name


def set_ue_groups(U: int):
    global WORKLOAD
    WORKLOAD = dataclasses.replace(WORKLOAD, U=max(1, int(U)))


def set_nlos_corr(rho):
    global WORKLOAD
    WORKLOAD = dataclasses.replace(WORKLOAD, nlos_corr=rho)


def workload_config(w, precoder="svd", name=None):
    cells = (f"J={w.J} cells" if w.U == 1 else
             f"J={w.J} cells x U={w.U} UEs, first-UE inter-cell interference")
    return {
        "workload": (f"{name or WORKLOAD_NAME}: {cells}, M={w.M}, N={w.N}, P={w.P}, K={w.K} subcarriers, "
                     f"ranks (m,n,p)=({w.m},{w.n},{w.p}), L={w.L} streams; {precoder}-precoded "
                     f"MMSE SINR; path-form coefficients; Tucker form drawn directly"),
        "precoder": precoder,
        "l2": "flushed before every timed step (256 MiB write)",
        "units_per_step": w.U * w.J * w.K,
    }


# --------------------------------------------------------------- flop counts
def link_flops(w, precoder="svd") -> int:
    """Algorithmic real flops of one launch of the interfering-link kernel
    (k_sinr_link_blk; k_sinr_link fold mode for the wideband precoder).

    One CTA column per (UE i, link k, subcarrier); per unit, in complex
    multiply-adds (8 flops each):
      P p                projection c* C (eq. 15)
      m n p              core contraction H~ = G x_3 (c* C) (eq. 15)   [svd]
      m n L              effective channel E = H~ V~ (eq. 24)          [svd]
      p m L              E = sum_q w_q F[q] (wideband precoder)
    over J (J - 1) interfering links (svd: the serving link comes from the
    precoder phase) or J^2 links (wideband precoder) and K subcarriers.  The
    covariance of eq. (25) is formed by the finalisation from the stored E.
    """
    J, m, n, p, P, L = w.J, w.m, w.n, w.p, w.P, w.L
    if precoder == "svd":
        return int(8 * w.K * J * (J - 1) * (P * p + m * n * p + m * n * L))
    return int(8 * w.K * J * J * (P * p + p * m * L))


PREC_CHAINS = {"tf32": 1, "tf32x3": 3, "bf16x2": 3}


def tensor_peak(precision: str) -> tuple[float, str]:
    """Dense tensor-core peak (TFLOP/s) of the MMA kind a mode runs on: the
    measured BF16 GEMM rate of the GB300s, and for TF32 that times
    the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    bf16 = float(peaks().get("bf16_tflops", 1900.0))
    if precision == "bf16x2":
        return bf16, "measured BF16 (MEASURED_PEAKS.json bf16_tflops)"
    return bf16 * 1.1 / 2.25, "measured BF16 x nominal TF32/BF16 ratio 1.1/2.25"


def link_roofline(torch, dev, w, precision: str, kernel_ms: float) -> dict:
    """Roofline of one interfering-link launch.  FP32 mode: every flop of
    link_flops on the FMA pipe.  Tensor-core modes: the core contraction
    (8 m n p per unit and product chain: 1 for TF32, 3 for TF32X3 and
    BF16X2) on the tensor pipe, the effective channel (8 m n L per unit) on
    the FMA pipe (the projection runs in its own kernel); the kernel is
    bound by the slower pipe, and `frac` is that pipe's time over the
    measured time."""
    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12       # TFLOP/s, FFMA on every lane
    units = w.K * w.J * (w.J - 1)
    t = kernel_ms * 1e-3
    if precision == "fp32":
        fl = link_flops(w, "svd")
        ach = fl / t / 1e12
        return {"kernel": "k_sinr_link_blk (svd)", "bound": "alu", "achieved": round(ach, 3),
                "peak": round(fp32_peak, 2), "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                "traffic": recorded_traffic("k_sinr_link_blk", WORKLOAD_NAME),
                "peak_basis": f"FP32 FFMA: {sms} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz "
                              "(unit counts and maximum SM clock)",
                "flops_per_launch": fl, "kernel_ms": round(kernel_ms, 5),
                "fma": {"achieved": round(ach, 3), "peak": round(fp32_peak, 2)}}
    tc_fl = 8 * w.m * w.n * w.p * units * PREC_CHAINS[precision]
    fma_fl = 8 * w.m * w.n * w.L * units
    tc_peak, tc_basis = tensor_peak(precision)
    t_tc, t_fma = tc_fl / (tc_peak * 1e12), fma_fl / (fp32_peak * 1e12)
    bound_tensor = t_tc >= t_fma
    ach_tc, ach_fma = tc_fl / t / 1e12, fma_fl / t / 1e12
    return {"kernel": f"k_sinr_link_tc ({precision})", "bound": "tensor" if bound_tensor else "alu",
            "achieved": round(ach_tc if bound_tensor else ach_fma, 3),
            "peak": round(tc_peak if bound_tensor else fp32_peak, 2), "unit": "TFLOP/s",
            "frac": round(max(t_tc, t_fma) / t, 4),
            "traffic": recorded_traffic(f"k_sinr_link_tc_{precision}", WORKLOAD_NAME),
            "peak_basis": (f"tensor: {tc_basis}; FMA: {sms} SMs x 128 lanes x 2 flop x "
                           f"{sm_max:.0f} MHz"),
            "kernel_ms": round(kernel_ms, 5),
            "tensor": {"flops_per_launch": tc_fl, "achieved": round(ach_tc, 3), "peak": round(tc_peak, 2),
                       "frac": round(t_tc / t, 4)},
            "fma": {"flops_per_launch": fma_fl, "achieved": round(ach_fma, 3), "peak": round(fp32_peak, 2),
                    "frac": round(t_fma / t, 4)}}


def precoder_flops(w) -> int:
    """Algorithmic flops of the SVD precoder phase: H~_kk (Pp + mnp), Gram m^2 n,
    V~ = H~* U / sigma (m n L) per (BS, subcarrier); the Jacobi sweeps are not counted."""
    J, m, n, p, P, L = w.J, w.m, w.n, w.p, w.P, w.L
    return int(8 * w.K * J * (P * p + m * n * p + m * m * n + m * n * L))


def svd_launches(w, prec_id=None) -> int:
    """Kernels one SVD-precoded SINR call launches (path-form coefficients):
    phase steps; the serving pass (FP32: one kernel, two for wide cores;
    TF32X3: the serving projections and the tensor-core serving pass), unless
    the precoder forms the serving channels itself; the precoder (two phases
    when it reads the serving pass's channels of up to 512 columns and 16
    rows) and, for up to 16 rows, the close-pair refinement; the
    interfering-link pass (tensor-core modes: core operand, projection
    operand, precoder tiles and the link kernel); finalize and refine."""
    from paper_2401_09792_gb300 import tuckersinr as ts
    tc = prec_id is not None and prec_id != ts.TS_PREC_FP32
    tf32x3 = prec_id == ts.TS_PREC_TF32X3
    fused = w.m * w.n * w.p <= 8192
    wide = w.p > 32 or w.P * w.p > 8192
    serve = 0 if fused else (2 if (wide or tf32x3) else 1)
    precoder = 2 if (not fused and w.m <= 16 and w.n <= 512) else 1
    close = 1 if w.m <= 16 else 0
    links = 4 if tc else 1
    return 1 + serve + precoder + close + links + 2


# ----------------------------------------------------------------- helpers
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# the sources each profiled kernel is built from (its summary under
# profiles/ stays valid while none of them changes)
KERNEL_SOURCES = {
    "k_sinr_link_blk": ("sinr_impl.cuh", "common.cuh", "kernels.h"),
    "k_svd_precoder": ("sinr_impl.cuh", "common.cuh", "kernels.h"),
    "k_sinr_finalize": ("sinr_impl.cuh", "common.cuh", "kernels.h"),
    "k_sinr_link_wide": ("sinr_wide.cuh", "sinr_impl.cuh", "common.cuh", "kernels.h"),
    "k_sinr_link_tc_tf32": ("sinr_tc.cu", "common.cuh", "kernels.h"),
    "k_sinr_link_tc_bf16x2": ("sinr_tc.cu", "common.cuh", "kernels.h"),
    "k_sinr_link_tc_tf32x3": ("sinr_tc.cu", "common.cuh", "kernels.h"),
    "k_precoder_refine": ("precoder_refine.cu", "common.cuh", "kernels.h"),
}


def _code_only(text: str) -> str:
    """C++/CUDA source without comments, trailing blanks and empty lines: a
    comment edit leaves a kernel's hash (and its captured profile) valid."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2401_09792_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        h.update(_code_only(open(os.path.join(csrc, name)).read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current sources of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    mh = re.search(r"kernel_source_hash:\s*(\w+)", text)
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not mh or not mb or mh.group(1) != kernel_source_hash(kernel):
        return None
    return float(mb.group(1))


def wide_link_traffic(w):
    """DRAM bytes per launch of the wide-core link kernel on workload w, and
    where the figure comes from: the workload's own capture, or (for the
    paper64 channels on 21 cells, too large to capture) the 8-cell capture
    scaled by the number of interfering links, since every link's core is
    read once per launch."""
    t = recorded_traffic("k_sinr_link_wide", WORKLOAD_NAME)
    if t is not None:
        return t, "ncu capture of this workload"
    small = {"paper64_u5": "paper64_j8"}.get(WORKLOAD_NAME)
    if small is not None:
        t = recorded_traffic("k_sinr_link_wide", small)
        if t is not None:
            ws = synth.WORKLOADS[small]
            return (t * (w.J * (w.J - 1)) / (ws.J * (ws.J - 1)),
                    f"ncu capture of {small} x {w.J * (w.J - 1)}/{ws.J * (ws.J - 1)} links")
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[0] == str(self.index):
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------- multi-rank host logic
def partition_workload(world: int):
    """The one system the ranks share: the selected workload with `world`
    times its subcarriers.  Every rank holds its G, C and path coefficients
    (replicated) and evaluates one contiguous range of WORKLOAD.K subcarriers
    with the range entry points (weak scaling, no data-path collective)."""
    return synth.Workload(**{**WORKLOAD.__dict__, "K": WORKLOAD.K * world})


def rank_range(rank: int, world: int) -> tuple[int, int]:
    """[k0, k1) of the shared system's subcarriers evaluated by `rank`."""
    from paper_2401_09792_gb300 import partition
    return partition.subcarrier_ranges(WORKLOAD.K * world, world)[rank]


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's time (all ranks get it); `x` unchanged at world 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, units_per_rank: int, steps: int, max_ms: float) -> float:
    """Subcarrier-SINRs per second of the whole job: every rank's units over
    the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2401_09792_gb300 import tuckersinr as ts

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    ts.load()

    # this rank's view of the shared system: its K subcarriers from kappa0 on
    w = WORKLOAD
    kappa0, kappa1 = rank_range(rank, world)
    d_all = ts.Dims.of(partition_workload(world))
    J, K, L, P = w.J, w.K, w.L, w.P
    assert kappa1 - kappa0 == K
    tk = synth.direct_tucker(w)
    alpha, tau = synth.path_gains_delays(w)
    s2 = synth.noise_powers(w)
    d = ts.Dims.of(w)
    host = {
        "G": torch.from_numpy(np.ascontiguousarray(np.transpose(tk["G"], (0, 1, 4, 2, 3))
                                                   .reshape(J * J, w.p, w.m, w.n)).astype(np.complex64)),
        "C": torch.from_numpy(tk["C"].reshape(J * J, P, w.p).astype(np.complex64)),
        "alpha": torch.from_numpy(alpha.reshape(J * J, P).astype(np.complex64)),
        "tau": torch.from_numpy(tau.reshape(J * J, P).astype(np.float32)),
        "sigma2": torch.from_numpy(s2.astype(np.float32)),
    }
    dv = {k: v.to(dev) for k, v in host.items()}
    coef, keep = ts.make_coef(alpha=dv["alpha"], tau=dv["tau"])
    sinr = torch.empty(J, K, L, device=dev)
    flags = torch.empty(J, K, dtype=torch.uint8, device=dev)
    prec_id = {"fp32": ts.TS_PREC_FP32, "tf32": ts.TS_PREC_TF32, "bf16x2": ts.TS_PREC_BF16X2,
               "tf32x3": ts.TS_PREC_TF32X3}[args.precision]
    ws_op = {"fp32": ts.TS_OP_SINR_SVD, "tf32": ts.TS_OP_SINR_SVD_TF32,
             "bf16x2": ts.TS_OP_SINR_SVD_BF16X2, "tf32x3": ts.TS_OP_SINR_SVD_TF32X3}[args.precision]
    ws = ts.workspace(d, ws_op, dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e0=None, e1=None, e2=None, k0=None, k1=None):
        if e0 is not None:
            e0.record(stream)
        # one call; the library records e1 between its precoder and link
        # phases and k0, k1 around the link kernel
        ts.ts_set_phase_event(e1)
        ts.ts_set_timing_events(k0, k1)
        if world > 1:
            # one range of the shared system
            ts.ts_sinr_svd_range(d_all, kappa0, K, coef, dv["G"], dv["C"], dv["sigma2"], prec_id,
                                 sinr, flags, ws, stream)
        else:
            ts.ts_sinr_svd_prec(d, coef, dv["G"], dv["C"], dv["sigma2"], prec_id, sinr, flags, ws,
                                stream)
        ts.ts_set_timing_events(None, None)
        ts.ts_set_phase_event(None)
        if e2 is not None:
            e2.record(stream)

    # path phase steps, precoders (with the serving links), links, finalize;
    # tensor-core modes add the core rewrite (a memset and a kernel)
    launches_per_step = svd_launches(w, prec_id)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    evs = [tuple(ev() for _ in range(5)) for _ in range(args.steps)]
    for e in evs:
        for x in e:
            x.record(stream)          # create the events before their handles are used
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    time.sleep(0.5 if sampler else 0.0)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for e0, e1, e2, k0, k1 in evs:
        flush.zero_()
        step(e0, e1, e2, k0, k1)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    link_ms = [e[3].elapsed_time(e[4]) for e in evs]
    pre_ms = [e[0].elapsed_time(e[1]) for e in evs]
    fin_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, dev)
    units = J * K
    value = whole_job_value(world, units, args.steps, total_ms)
    assert int((flags & ts.TS_FLAG_ERRORS).max().item()) == 0, "numerical flags raised in the timed steps"

    if args.step_only:
        e2e_value = h2d = d2h = mm_ms = dense_value = dense_ms = dense_steps = None
        prec = {}
    else:
        e2e_value, h2d, d2h, mm_ms, dense_value, dense_ms, dense_steps = _extras(
            args, ts, torch, dist, world, dev, w, tk, host, dv, coef, d, ws, sinr, flags, flush,
            stream, ev, units, prec_id)
        prec = _precision_variants(args, ts, torch, dev, w, dv, coef, d, sinr, flags, flush, stream,
                                   ev, units)
        if args.adjoint:
            prec["adjoint"] = _adjoint_timing(args, ts, torch, dev, w, dv, coef, d, flush, stream, ev,
                                              units)
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    _report(args, ts, torch, world, dev, w, tk, alpha, tau, s2, d, coef, dv, ws, stream, units,
            value, total_ms, step_ms, link_ms, pre_ms, fin_ms, wall, clocks, launches_per_step,
            e2e_value, h2d, d2h, mm_ms, dense_value, dense_ms, dense_steps, prec)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    del keep


def _extras(args, ts, torch, dist, world, dev, w, tk, host, dv, coef, d, ws, sinr, flags, flush,
            stream, ev, units, prec_id):
    """End-to-end, wideband-precoder and dense-comparator timings."""
    J, K, L, P = w.J, w.K, w.L, w.P
    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    pinned = {k: v.pin_memory() for k, v in host.items()}
    out_host = torch.empty(J, K, L).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = out_host.numel() * out_host.element_size()

    def e2e_step():
        for k in pinned:
            dv[k].copy_(pinned[k], non_blocking=True)
        ts.ts_sinr_svd_prec(d, coef, dv["G"], dv["C"], dv["sigma2"], prec_id, sinr, flags, ws, stream)
        out_host.copy_(sinr, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = whole_job_value(world, units, args.steps, e2e_ms)

    # ---- the MMSE variant (wideband precoders), same timing discipline
    Pw = synth.wideband_precoders(w)
    B = torch.from_numpy(tk["B"].astype(np.complex64)).to(dev)
    Pf = torch.from_numpy(Pw.astype(np.complex64)).to(dev)
    Pt = torch.empty(J, w.n, L, dtype=torch.complex64, device=dev)
    ts.ts_project_precoder(d, B, Pf, Pt, stream)
    ws_m = ts.workspace(d, ts.TS_OP_SINR_MMSE, dev)
    for _ in range(args.warmup):
        ts.ts_sinr_mmse(d, coef, dv["G"], dv["C"], Pt, dv["sigma2"], sinr, flags, ws_m, stream)
    mm_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        ts.ts_sinr_mmse(d, coef, dv["G"], dv["C"], Pt, dv["sigma2"], sinr, flags, ws_m, stream)
        b.record(stream)
        b.synchronize()
        mm_ms += a.elapsed_time(b)

    # ---- dense-channel comparator on the same system: full M x N channels per
    # subcarrier (eq. 9), precoders and solves at (M, N); same kernels, C = I
    if ts.ts_workspace_bytes(d, ts.TS_OP_DENSE_SVD) == 0:
        # the dense kernels stage one M x N channel per subcarrier: M <= 64,
        # N <= 1024, P <= 1024
        return e2e_value, h2d, d2h, mm_ms, None, None, None
    if w == synth.MID:
        # the channel model's own channels (the method figures below use them)
        X = synth.channel_submatrices(w)
        Xd = torch.from_numpy(np.ascontiguousarray(np.transpose(X, (0, 1, 4, 2, 3))
                                                   .reshape(J * J, P, w.M, w.N)).astype(np.complex64)).to(dev)
        del X
    else:
        # X^ = G x_1 A x_2 B x_3 C reconstructed on the GPU from the same
        # Tucker form: both paths then compute the same SINR (A and B cancel)
        Xd = _reconstructed_channels(ts, torch, dev, w, tk, dv, d)
    ws_d = ts.workspace(d, ts.TS_OP_DENSE_SVD, dev)
    for _ in range(args.warmup):
        ts.ts_dense_sinr_svd(d, coef, Xd, dv["sigma2"], sinr, flags, ws_d, stream)
    dense_ms = 0.0
    dense_steps = max(3, args.steps // 10)
    for _ in range(dense_steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        ts.ts_dense_sinr_svd(d, coef, Xd, dv["sigma2"], sinr, flags, ws_d, stream)
        b.record(stream)
        b.synchronize()
        dense_ms += a.elapsed_time(b)
    assert int((flags & ts.TS_FLAG_ERRORS).max().item()) == 0, "numerical flags raised in the dense steps"
    dense_value = units * dense_steps / (dense_ms * 1e-3)
    _extras.dense_sinr = sinr.cpu().numpy().astype(np.float64)
    if w != synth.MID:
        del Xd, ws_d
        return e2e_value, h2d, d2h, mm_ms, dense_value, dense_ms, dense_steps
    _method_error.result = _method_error(ts, torch, dev, w, Xd, coef, dv, d, stream, ev, flush,
                                         dense_ms / dense_steps)
    # the same on spatially correlated NLOS channels (compressible in modes
    # 1 and 2, as measured array channels are)
    del Xd
    wc = synth.MID_CORR if w == synth.MID else dataclasses.replace(w, nlos_corr=synth.MID_CORR.nlos_corr)
    Xd = ts.channels_to_device(synth.channel_submatrices(wc), dev)
    corr = _method_error(ts, torch, dev, w, Xd, coef, dv, d, stream, ev, flush, dense_ms / dense_steps,
                         fit_speed=True)
    corr["channels"] = (f"NLOS Kronecker model, exponential correlation {wc.nlos_corr[0]} (UE array) "
                        f"and {wc.nlos_corr[1]} (BS array)")
    _method_error.result["correlated_channels"] = corr
    del Xd, ws_d
    return e2e_value, h2d, d2h, mm_ms, dense_value, dense_ms, dense_steps


def _reconstructed_channels(ts, torch, dev, w, tk, dv, d):
    """X^_ik = G_ik x_1 A_i x_2 B_k x_3 C_ik of every link on the GPU
    (ts_tucker_reconstruct), in the dense comparator's layout [J*J][P][M][N]."""
    A = torch.from_numpy(tk["A"].astype(np.complex64)).to(dev)
    B = torch.from_numpy(tk["B"].astype(np.complex64)).to(dev)
    Xd = torch.empty(w.J * w.J, w.P, w.M, w.N, dtype=torch.complex64, device=dev)
    wsr = ts.workspace(d, ts.TS_OP_RECONSTRUCT, dev)
    ts.ts_tucker_reconstruct(d, ts.TS_MODEL_GROUPWISE, A, B, dv["C"], dv["G"], Xd, wsr)
    torch.cuda.synchronize()
    del wsr
    return Xd


def _method_error(ts, torch, dev, w, Xd, coef, dv, d, stream, ev, flush, dense_step_ms, sweeps=10,
                  fit_speed=False):
    """The paper's model comparison (Section 4, Table of compression results)
    on these channels, for the groupwise (eq. 14), shared (eq. 12) and
    individual (eq. 10) models: fit each on the GPU (Algorithm 2, `sweeps`
    sweeps), then
      e_c  eq. (30): mean |SINR_model - SINR_dense| / SINR_dense over UEs,
           subcarriers and streams, both SINRs on the GPU;
      R_s  eq. (29) and the storage table of Section 3.3, exact;
      R_t  t_dense / t_model: the dense-channel SINR time over the model's
           SINR time on the same GPU (groupwise and shared through the
           compressed kernels, whose factors cancel; individual through the
           reconstruction X^ and the dense kernels).
    With i.i.d. NLOS submatrices the channels are far less compressible than
    the paper's 3GPP data, so e_c is far above its ~10%."""
    from oracle import tucker as T
    J, M, N, P, m, n, p, K, L = w.J, w.M, w.N, w.P, w.m, w.n, w.p, w.K, w.L
    s_d = torch.empty(J, K, L, device=dev)
    ts.ts_dense_sinr_svd(d, coef, Xd, dv["sigma2"], s_d, None, ts.workspace(d, ts.TS_OP_DENSE_SVD, dev),
                         stream)
    torch.cuda.synchronize()
    sd = s_d.double()
    x2 = float((Xd.abs() ** 2).sum().item())

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        return total / reps

    models = {}
    for name, mid, op in (("groupwise", ts.TS_MODEL_GROUPWISE, ts.TS_OP_TUCKER_FIT),
                          ("shared", ts.TS_MODEL_SHARED, ts.TS_OP_TUCKER_FIT_SHARED),
                          ("individual", ts.TS_MODEL_INDIVIDUAL, ts.TS_OP_TUCKER_FIT_INDIVIDUAL)):
        nA, nB, _, _ = T.factor_groups(J, name)
        A = torch.empty(nA, M, m, dtype=torch.complex64, device=dev)
        B = torch.empty(nB, N, n, dtype=torch.complex64, device=dev)
        C = torch.empty(J * J, P, p, dtype=torch.complex64, device=dev)
        G = torch.empty(J * J, p, m, n, dtype=torch.complex64, device=dev)
        g = torch.empty(3 * sweeps + 1, dtype=torch.float64, device=dev)
        wsf = ts.workspace(d, op, dev)
        a, b = ev(), ev()
        a.record(stream)
        ts.ts_tucker_fit_model(d, Xd, sweeps, 0, mid, A, B, C, G, g, wsf, stream)
        b.record(stream)
        b.synchronize()
        fit_ms = a.elapsed_time(b)
        del wsf
        s_t = torch.empty(J, K, L, device=dev)
        if name != "individual":
            wss = ts.workspace(d, ts.TS_OP_SINR_SVD, dev)

            def run():
                ts.ts_sinr_svd(d, coef, G, C, dv["sigma2"], s_t, None, wss, stream)
            how = "compressed kernels on (G, C)"
        else:
            Xh = torch.empty_like(Xd)
            wsr = ts.workspace(d, ts.TS_OP_RECONSTRUCT, dev)
            wsd = ts.workspace(d, ts.TS_OP_DENSE_SVD, dev)

            def run():
                ts.ts_tucker_reconstruct(d, mid, A, B, C, G, Xh, wsr, stream)
                ts.ts_dense_sinr_svd(d, coef, Xh, dv["sigma2"], s_t, None, wsd, stream)
            how = "reconstruction X^ then the dense kernels"
        t_ms = timed(run)
        st = s_t.double()
        # one UE per cell: the storage table's K (UEs per BS) is 1
        models[name] = {"e_c": float(((st - sd).abs() / sd.abs()).mean().item()),
                        "R_s": T.storage_ratio(J, 1, M, N, P, m, n, p, name),
                        "R_t": dense_step_ms / t_ms, "sinr_ms": round(t_ms, 4), "sinr_path": how,
                        "fit_ms": round(fit_ms, 2), "g_over_x2": float(g[-1].item()) / x2}
        del A, B, C, G, s_t
    speed = None
    if fit_speed:
        # fewer inner iterations of the B-mode eigensolves (N > 72): time per
        # fit against the fitted energy and e_c
        speed = []
        for it in (40, 8, 2):
            ts.ts_set_fit_iterations(it)
            A = torch.empty(J, M, m, dtype=torch.complex64, device=dev)
            B = torch.empty(J, N, n, dtype=torch.complex64, device=dev)
            C = torch.empty(J * J, P, p, dtype=torch.complex64, device=dev)
            G = torch.empty(J * J, p, m, n, dtype=torch.complex64, device=dev)
            g = torch.empty(3 * sweeps + 1, dtype=torch.float64, device=dev)
            wsf = ts.workspace(d, ts.TS_OP_TUCKER_FIT, dev)
            a, b = ev(), ev()
            a.record(stream)
            ts.ts_tucker_fit(d, Xd, sweeps, 0, A, B, C, G, g, wsf, stream)
            b.record(stream)
            b.synchronize()
            s_t = torch.empty(J, K, L, device=dev)
            ts.ts_sinr_svd(d, coef, G, C, dv["sigma2"], s_t, None,
                           ts.workspace(d, ts.TS_OP_SINR_SVD, dev), stream)
            torch.cuda.synchronize()
            st = s_t.double()
            speed.append({"inner_iterations": it, "fit_ms": round(a.elapsed_time(b), 2),
                          "ms_per_sweep": round(a.elapsed_time(b) / sweeps, 2),
                          "g_over_x2": float(g[-1].item()) / x2,
                          "e_c": float(((st - sd).abs() / sd.abs()).mean().item())})
            del A, B, C, G, wsf
        ts.ts_set_fit_iterations(0)
    gw = models["groupwise"]
    return {"e_c": gw["e_c"], "fit_inner_iterations": speed, "what": "eq. (30) for the groupwise form fitted on the GPU "
                                      f"({sweeps} sweeps of Algorithm 2) from the synthetic channels; "
                                      "models: the same for the three compression models, with the "
                                      "storage ratio R_s (eq. 29) and the speedup R_t = t_dense / t_model",
            "fit_ms": gw["fit_ms"], "g_over_x2": gw["g_over_x2"], "storage_ratio": gw["R_s"],
            "models": models}


def _adjoint_timing(args, ts, torch, dev, w, dv, coef, d, flush, stream, ev, units):
    """The adjoint of the SVD-precoded SINR (dSINR -> dG, dC; the forward
    quantities are recomputed inside), same timing discipline."""
    dsinr = torch.ones(w.J, w.K, w.L, device=dev)
    dG = torch.empty_like(dv["G"])
    dC = torch.empty_like(dv["C"])
    wsa = ts.workspace(d, ts.TS_OP_SINR_SVD_ADJOINT, dev)
    for _ in range(args.warmup):
        ts.ts_sinr_svd_adjoint(d, coef, dv["G"], dv["C"], dv["sigma2"], dsinr, dG, dC, None, wsa, stream)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 10)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        ts.ts_sinr_svd_adjoint(d, coef, dv["G"], dv["C"], dv["sigma2"], dsinr, dG, dC, None, wsa, stream)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    del wsa
    return {"value": units * steps / (total * 1e-3), "unit": "subcarrier-SINR gradients/s",
            "ms_per_step": total / steps, "steps": steps,
            "what": "d(sum_r dSINR_r SINR_r)/d(G, C), forward recomputed, workspace "
                    f"{ts.ts_workspace_bytes(d, ts.TS_OP_SINR_SVD_ADJOINT) / 2**30:.2f} GiB"}


def _precision_variants(args, ts, torch, dev, w, dv, coef, d, sinr, flags, flush, stream, ev, units):
    """The same step with the interfering links' core contraction on the
    tensor cores (TF32, BF16 hi+lo): throughput, link-pass time, and the
    SINRs of one evaluation for the error report."""
    out = {}
    for name, prec, op in (("fp32", ts.TS_PREC_FP32, ts.TS_OP_SINR_SVD),
                           ("tf32", ts.TS_PREC_TF32, ts.TS_OP_SINR_SVD_TF32),
                           ("bf16x2", ts.TS_PREC_BF16X2, ts.TS_OP_SINR_SVD_BF16X2),
                           ("tf32x3", ts.TS_PREC_TF32X3, ts.TS_OP_SINR_SVD_TF32X3)):
        if name == args.precision or ts.ts_workspace_bytes(d, op) == 0:
            continue
        wsp = ts.workspace(d, op, dev)

        def step(k0=None, k1=None):
            ts.ts_set_timing_events(k0, k1)
            ts.ts_sinr_svd_prec(d, coef, dv["G"], dv["C"], dv["sigma2"], prec, sinr, flags, wsp, stream)
            ts.ts_set_timing_events(None, None)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        evs = [tuple(ev() for _ in range(4)) for _ in range(args.steps)]
        for e in evs:
            for x in e:
                x.record(stream)      # create the events before the library records them
        torch.cuda.synchronize()
        for a, b, k0, k1 in evs:
            flush.zero_()
            a.record(stream)
            step(k0, k1)
            b.record(stream)
        torch.cuda.synchronize()
        total = float(np.sum([a.elapsed_time(b) for a, b, _, _ in evs]))
        link = float(np.mean([k0.elapsed_time(k1) for _, _, k0, k1 in evs]))
        assert int((flags & ts.TS_FLAG_ERRORS).max().item()) == 0, f"numerical flags raised in the {name} steps"
        ts.ts_sinr_svd_prec(d, coef, dv["G"], dv["C"], dv["sigma2"], prec, sinr, None, wsp, stream)
        torch.cuda.synchronize()
        out[name] = {"value": units * args.steps / (total * 1e-3), "ms_per_step": total / args.steps,
                     "link_ms": round(link, 5), "roofline": link_roofline(torch, dev, w, name, link),
                     "sinr": sinr.cpu().numpy().astype(np.float64)}
        del wsp
    return out


def _report(args, ts, torch, world, dev, w, tk, alpha, tau, s2, d, coef, dv, ws, stream, units,
            value, total_ms, step_ms, link_ms, pre_ms, fin_ms, wall, clocks, launches_per_step,
            e2e_value, h2d, d2h, mm_ms, dense_value, dense_ms, dense_steps, prec):
    link_mean = float(np.mean(link_ms))
    roofline = link_roofline(torch, dev, w, args.precision, link_mean)
    roofline["share_of_step"] = round(float(np.sum(link_ms)) / float(np.sum(step_ms)), 3)

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"f32 + {args.precision} (tensor-core core contraction)",
        "data": "synthetic",
        "config": workload_config(w),
        "parallelism": (f"subcarrier partition x{world}: one system of {world} x {w.K} subcarriers, "
                        f"G, C and the path coefficients replicated, a range of {w.K} per rank"
                        if world > 1 else "one GPU"),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "phases_ms": {"precoders": round(float(np.mean(pre_ms)), 5),
                      "links_and_finalize": round(float(np.mean(fin_ms)), 5),
                      "links": round(link_mean, 5)},
        "variants": None if mm_ms is None else {
            "mmse_wideband_precoder": {"value": units * args.steps / (mm_ms * 1e-3),
                                       "ms_per_step": mm_ms / args.steps},
            **{f"svd_{k}": {"value": v["value"], "ms_per_step": v["ms_per_step"],
                            "link_ms": v["link_ms"], "roofline": v["roofline"],
                            "what": ("all arithmetic FP32 on the FMA pipe" if k == "fp32" else
                                     "interfering links' core contraction on the tensor cores "
                                     f"({k}), everything else FP32")}
               for k, v in prec.items() if k != "adjoint"},
            **({"svd_adjoint": prec["adjoint"]} if "adjoint" in prec else {})},
        "method": getattr(_method_error, "result", None),
        "dense_comparator": {"unavailable": "dense kernels need M <= 64, N <= 1024, P <= 1024"}
        if dense_ms is None else {
            "value": dense_value, "unit": METRIC, "ms_per_step": dense_ms / dense_steps,
            "what": "same SVD-precoded SINR from the uncompressed channels "
                    f"(M={w.M}, N={w.N}, P={w.P}) on the same GPU kernels"
                    + ("" if w == synth.MID else
                       "; channels X^ = G x1 A x2 B x3 C reconstructed on the GPU from the same "
                       "Tucker form, so both paths compute the same SINR"),
            "tucker_over_dense": value / world / dense_value},
        "wall_s_timed_region": round(wall, 4),
    }
    if args.step_only:
        for key in ("e2e", "variants", "dense_comparator", "method"):
            line.pop(key)
    if world == 1 and not args.step_only:
        pk_meas = ts.ts_device_peaks(stream)
        line["device_peaks"] = {**{k: round(v, 2) for k, v in pk_meas.items()}, "unit": "TFLOP/s",
                                "what": "measured by the library's microbenchmarks on this GPU"}
        line["roofline"]["frac_of_measured_fp32"] = round(line["roofline"]["fma"]["achieved"] /
                                                          pk_meas["fp32_fma"], 4)
    if world == 1 and not args.no_cpu_baseline:
        gpu_out = {"headline": _gpu_svd_sinr(ts, d, coef, dv, ws, stream, args.precision)}
        gpu_out.update({k: v["sinr"] for k, v in prec.items() if "sinr" in v})
        if "dense_comparator" in line and getattr(_extras, "dense_sinr", None) is not None:
            gpu_out["dense"] = _extras.dense_sinr
        line["cpu_baseline"], errs = cpu_baseline(w, tk, alpha, tau, s2, gpu_out)
        line["sinr_err"] = errs.pop("headline", None)
        if "dense" in errs:
            line["dense_comparator"]["sinr_err"] = errs.pop("dense")
        for k, e in errs.items():
            line["variants"][f"svd_{k}"]["sinr_err"] = e
    if world == 1 and not args.step_only:
        line["workloads"] = {name: _workload_summary(name, args, ts, torch, dev)
                             for name in ("mid", "precision") if name != WORKLOAD_NAME}
    print(json.dumps(line), flush=True)


def _workload_summary(name, args, ts, torch, dev, kcount=32):
    """Another workload's SVD-precoded SINR step (same timing discipline,
    fewer steps): throughput, link-pass roofline fraction, and the error of
    every SINR at `kcount` subcarriers spread over the range against the
    FP64 oracle."""
    from oracle import sinr as S
    w = synth.WORKLOADS[name]
    tk = synth.direct_tucker(w)
    alpha, tau = synth.path_gains_delays(w)
    s2 = synth.noise_powers(w)
    d = ts.Dims.of(w)
    G = ts.core_to_device(tk["G"], dev)
    C = ts.factor_to_device(tk["C"].reshape(w.J * w.J, w.P, w.p), dev)
    al = ts.factor_to_device(alpha.reshape(w.J * w.J, w.P), dev)
    ta = ts.real_to_device(tau.reshape(w.J * w.J, w.P), dev)
    sig = ts.real_to_device(s2, dev)
    coef, keep = ts.make_coef(alpha=al, tau=ta)
    sinr = torch.empty(w.J, w.K, w.L, device=dev)
    flags = torch.empty(w.J, w.K, dtype=torch.uint8, device=dev)
    prec = {"fp32": ts.TS_PREC_FP32, "tf32": ts.TS_PREC_TF32, "bf16x2": ts.TS_PREC_BF16X2,
            "tf32x3": ts.TS_PREC_TF32X3}[args.precision]
    op = {"fp32": ts.TS_OP_SINR_SVD, "tf32": ts.TS_OP_SINR_SVD_TF32, "bf16x2": ts.TS_OP_SINR_SVD_BF16X2,
          "tf32x3": ts.TS_OP_SINR_SVD_TF32X3}[args.precision]
    ws = ts.workspace(d, op, dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    steps = max(5, min(args.steps, 50))
    for _ in range(args.warmup):
        ts.ts_sinr_svd_prec(d, coef, G, C, sig, prec, sinr, flags, ws, stream)
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(steps)]
    for e in evs:
        for x in e:
            x.record(stream)
    torch.cuda.synchronize()
    for a, b, k0, k1 in evs:
        flush.zero_()
        a.record(stream)
        ts.ts_set_timing_events(k0, k1)
        ts.ts_sinr_svd_prec(d, coef, G, C, sig, prec, sinr, flags, ws, stream)
        ts.ts_set_timing_events(None, None)
        b.record(stream)
    torch.cuda.synchronize()
    total = float(np.sum([a.elapsed_time(b) for a, b, _, _ in evs]))
    link = float(np.mean([k0.elapsed_time(k1) for _, _, k0, k1 in evs]))
    assert int((flags & ts.TS_FLAG_ERRORS).max().item()) == 0, f"numerical flags raised on {name}"
    got = sinr.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    ks = np.unique(np.concatenate([[0, w.K - 1], rng.choice(w.K, kcount - 2, replace=False)]))
    coef_h = S.coefficients(alpha, tau, w.K, w.delta_f_hz)[:, :, ks]
    ref = S.tucker_sinr(tk["G"], tk["C"], coef_h, s2, w.L, "svd")
    rel = np.abs(got[:, ks] - ref) / np.abs(ref)
    roof = link_roofline(torch, dev, w, args.precision, link)
    del keep
    return {"value": w.J * w.K * steps / (total * 1e-3), "unit": METRIC, "ms_per_step": total / steps,
            "steps": steps, "config": workload_config(w, name=name)["workload"],
            "dtype": "f32" if args.precision == "fp32" else f"f32 + {args.precision}",
            "link_kernel": {"ms": round(link, 5), "bound": roof["bound"], "frac": roof["frac"]},
            "sinr_err": {"max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99)),
                         "median_rel": float(np.median(rel)), "n": int(rel.size),
                         "vs": f"FP64 oracle at {len(ks)} subcarriers spread over the range"}}


def _gpu_svd_sinr(ts, d, coef, dv, ws, stream, precision="fp32"):
    import torch
    J, K, L = d.J, d.K, d.L
    out = torch.empty(J, K, L, device=dv["G"].device)
    prec = {"fp32": ts.TS_PREC_FP32, "tf32": ts.TS_PREC_TF32, "bf16x2": ts.TS_PREC_BF16X2,
            "tf32x3": ts.TS_PREC_TF32X3}[precision]
    ts.ts_sinr_svd_prec(d, coef, dv["G"], dv["C"], dv["sigma2"], prec, out, None, ws, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def cpu_baseline(w, tk, alpha, tau, s2, gpu_sinr=None, budget_s=12.0, kslice=128):
    """The FP64 oracle, as it stands, on subcarrier slices of the same system,
    for about `budget_s` seconds; also the error of each GPU result
    (`gpu_sinr`: name -> SINR array) on those slices."""
    from oracle import sinr as S
    J = w.J
    coef = S.coefficients(alpha, tau, w.K, w.delta_f_hz)
    t0 = time.perf_counter()
    c0 = time.process_time()
    gpu_sinr = gpu_sinr or {}
    done, errs, start, passes = 0, {k: [] for k in gpu_sinr}, 0, 0
    while time.perf_counter() - t0 < budget_s:
        sl = slice(start, min(start + kslice, w.K))
        ref = S.tucker_sinr(tk["G"], tk["C"], coef[:, :, sl], s2, w.L, "svd")
        if passes == 0:
            for k, g in gpu_sinr.items():
                errs[k].append(np.abs(g[:, sl] - ref) / np.abs(ref))
        done += J * (sl.stop - sl.start)
        start = sl.stop
        if start >= w.K:
            start, passes = 0, passes + 1
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    base = {"value": done / wall, "unit": METRIC, "cores": max(1, round(cpu / wall)),
            "kind": "oracle",
            "sample": f"FP64 NumPy oracle, svd SINR of the same system in slices of "
                      f"{kslice} subcarriers, repeated for {wall:.1f} s wall ({done} "
                      f"subcarrier-SINRs; {os.cpu_count()} host cores visible)"}
    out = {}
    for k, lst in errs.items():
        if not lst:
            continue
        e = np.concatenate([x.ravel() for x in lst])
        out[k] = {"max_rel": float(e.max()), "p99_rel": float(np.percentile(e, 99)),
                  "median_rel": float(np.median(e)), "n": int(e.size),
                  "vs": "FP64 oracle on the cpu_baseline subcarriers"}
    return base, out


# ------------------------------------------------------------ batch workload
def batch_systems(count: int, seed: int = 0):
    """Instances of the batching workload: N in {64,128,256,512}, M in {2,4,8},
    K uniform in 256..3300, J uniform in 2..16, m = M, n in {16,32,64} (<= N),
    p in {8,16,32}, P = 64, L = m; path-form coefficients; Tucker form drawn
    directly; SVD precoding."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        M = int(rng.choice([2, 4, 8]))
        N = int(rng.choice([64, 128, 256, 512]))
        n = int(min(N, rng.choice([16, 32, 64])))
        out.append(synth.Workload(f"batch{j}", J=int(rng.integers(2, 17)), M=M, N=N, P=64,
                                  K=int(rng.integers(256, 3301)), m=M, n=n, p=int(rng.choice([8, 16, 32])),
                                  L=M, n_los=2, pdp_decay_s=300e-9, sigma2=None, seed=1000 + j))
    return out


def run_batch(args):
    import torch

    from paper_2401_09792_gb300 import tuckersinr as ts
    import __graft_entry__
    __graft_entry__.build()
    ts.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    systems = batch_systems(args.batch_instances)
    keep, insts, host = [], [], []
    for w in systems:
        # the Tucker form drawn on the device (seeded; thousands of systems);
        # the oracle check below reads back the ones it samples
        tk = synth.direct_tucker_device(w, device=dev)
        alpha, tau = synth.path_gains_delays(w)
        s2 = synth.noise_powers(w)
        d = ts.Dims.of(w)
        G = tk["G"]
        C = tk["C"]
        al = ts.factor_to_device(alpha.reshape(w.J * w.J, w.P), dev)
        ta = ts.real_to_device(tau.reshape(w.J * w.J, w.P), dev)
        sig = ts.real_to_device(s2, dev)
        cs, k = ts.make_coef(alpha=al, tau=ta)
        sinr = torch.empty(w.J, w.K, w.L, device=dev)
        flags = torch.empty(w.J, w.K, dtype=torch.uint8, device=dev)
        insts.append(ts.instance(d, ts.TS_OP_SINR_SVD, cs, G, C, sig, sinr, flags))
        keep.append((G, C, al, ta, sig, sinr, flags, k))
        host.append((w, alpha, tau, s2))
    ws = ts.batch_workspace(insts, dev)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    plan = ts.BatchPlan(insts, ws, autotune=True)
    plan_s = time.perf_counter() - t0
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(args.warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    time.sleep(0.5)
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        plan.launch(stream)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    clocks = sampler.stop()
    bad = sum(int((kp[6] & ts.TS_FLAG_ERRORS).max().item()) for kp in keep)
    assert bad == 0, "numerical flags raised in the batch"
    # the same instances one call after another on one stream, no graph,
    # all on the start of the batch workspace (one at a time)
    maxnb = max(ts.ts_workspace_bytes(ts.Dims.of(w), ts.TS_OP_SINR_SVD) for w in systems)
    slices = [ws[:maxnb]] * len(systems)
    seq_steps = max(1, args.steps // 2)
    seq = 0.0
    for _ in range(seq_steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        for w, x, kp, wsi in zip(systems, insts, keep, slices):
            ts.ts_sinr_svd(ts.Dims.of(w), x.coef, kp[0], kp[1], kp[4], kp[5], kp[6], wsi, stream)
        b.record(stream)
        b.synchronize()
        seq += a.elapsed_time(b)
    units = sum(w.J * w.K for w in systems)
    # CPU oracle on a bounded sample: the first instances, 64-subcarrier slices
    from oracle import sinr as S
    c0, t1, done = time.process_time(), time.perf_counter(), 0
    errs = []
    for (w, alpha, tau, s2), kp in zip(host, keep):
        if time.perf_counter() - t1 > 12.0:
            break
        J = w.J
        Gh = kp[0].cpu().numpy().astype(np.complex128).reshape(J, J, w.p, w.m, w.n).transpose(0, 1, 3, 4, 2)
        Ch = kp[1].cpu().numpy().astype(np.complex128).reshape(J, J, w.P, w.p)
        coef = S.coefficients(alpha, tau, min(w.K, 64), w.delta_f_hz)
        ref = S.tucker_sinr(Gh, Ch, coef, s2, w.L, "svd")
        got = kp[5][:, :coef.shape[2]].cpu().numpy().astype(np.float64)
        errs.append((np.abs(got - ref) / np.abs(ref)).ravel())
        done += w.J * coef.shape[2]
    wall = time.perf_counter() - t1
    e = np.concatenate(errs)
    line = {
        "metric": METRIC, "value": units * args.steps / (total * 1e-3), "unit": METRIC, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batch: {len(systems)} systems, N in {{64..512}}, M in {{2,4,8}}, "
                               "K in 256..3300, J in 2..16, ranks up to (8,64,32), P=64, L=m; "
                               "svd-precoded MMSE SINR; one CUDA-graph launch per step",
                   "units_per_step": units, "l2": "flushed before every timed step (256 MiB write)",
                   "plan_seconds_incl_autotune": round(plan_s, 2),
                   "workspace_gib": round(ws.numel() / 2**30, 2)},
        "sequential_calls": {"ms_per_step": seq / seq_steps,
                             "what": "the same systems as one ts_sinr_svd call each on one stream"},
        "gpu_launches": sum(svd_launches(w) for w in systems) * args.steps, "clocks": clocks,
        "cpu_baseline": {"value": done / wall, "unit": METRIC,
                         "cores": max(1, round((time.process_time() - c0) / wall)), "kind": "oracle",
                         "sample": f"FP64 NumPy oracle on the first 64 subcarriers of the first "
                                   f"{len(errs)} systems ({done} subcarrier-SINRs)"},
        "sinr_err": {"max_rel": float(e.max()), "p99_rel": float(np.percentile(e, 99)),
                     "median_rel": float(np.median(e)), "n": int(e.size)},
    }
    print(json.dumps(line), flush=True)
    plan.close()


def run_multiuser(args):
    """The paper's own system sizes (Section 4): J = 21 cells, U UEs per
    cell with first-UE inter-cell interference, (M, N, P) = (8, 256, 401)
    and the paper's compressed sizes; Tucker form drawn directly (fitting
    ~15 GB of channels per UE group is an offline step the paper does once).
    Reports the compressed-path throughput, the wide-core link kernel
    against the FP32 roofline, the dense-channel comparator on the
    reconstructed channels X^ (the same SINR up to rounding: A and B cancel)
    as the speedup R_t = t_dense / t_compressed, and R_s of eq. (29)."""
    import torch

    from oracle import tucker as T
    from paper_2401_09792_gb300 import tuckersinr as ts
    import __graft_entry__
    __graft_entry__.build()
    ts.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = WORKLOAD
    U, J, K, L, P, M, N, m, n, p = w.U, w.J, w.K, w.L, w.P, w.M, w.N, w.m, w.n, w.p
    nl = J * J
    d = ts.Dims.of(w)
    t_setup = time.perf_counter()
    c64 = dict(dtype=torch.complex64, device=dev)
    Gd = torch.empty(U * nl, p, m, n, **c64)
    Cd = torch.empty(U * nl, P, p, **c64)
    Ad = torch.empty(U, J, M, m, **c64)
    ad = torch.empty(U * nl, P, **c64)
    td = torch.empty(U * nl, P, dtype=torch.float32, device=dev)
    sd = torch.empty(U * J, dtype=torch.float32, device=dev)
    host = {}                                 # UE groups 0 and 1 for the oracle sample
    # cores of millions of entries per link: drawn on the device
    on_device = m * n * p >= (1 << 20)
    for u in range(U):
        alpha, tau = synth.path_gains_delays(w, ue=u)
        s2 = synth.noise_powers(w, ue=u)
        if on_device:
            td_ = synth.direct_tucker_device(w, ue=u, device=dev)
            Gd[u * nl:(u + 1) * nl] = td_["G"]
            Cd[u * nl:(u + 1) * nl] = td_["C"]
            Ad[u] = td_["A"]
            if u == 0:
                Bd = td_["B"]
            tk = None                      # no host copy: no oracle sample at these sizes
            del td_
        else:
            tk = synth.direct_tucker(w, ue=u)
            Gd[u * nl:(u + 1) * nl] = ts.core_to_device(tk["G"], dev)
            Cd[u * nl:(u + 1) * nl] = ts.factor_to_device(tk["C"].reshape(nl, P, p), dev)
            Ad[u] = ts.factor_to_device(tk["A"], dev)
        ad[u * nl:(u + 1) * nl] = ts.factor_to_device(alpha.reshape(nl, P), dev)
        td[u * nl:(u + 1) * nl] = ts.real_to_device(tau.reshape(nl, P), dev)
        sd[u * J:(u + 1) * J] = ts.real_to_device(s2, dev)
        if u == 0 and not on_device:
            Bd = ts.factor_to_device(tk["B"], dev)
        if u < 2 and tk is not None:
            host[u] = (tk["G"], tk["C"], alpha, tau, s2)
        del tk
    cs, keep = ts.make_coef(alpha=ad, tau=td)
    sinr = torch.empty(U, J, K, L, device=dev)
    flags = torch.empty(U, J, K, dtype=torch.uint8, device=dev)
    # one single-UE workspace per group: the groups after the first run
    # concurrently on the library's side streams
    single = ts.ts_workspace_bytes(d, ts.TS_OP_SINR_SVD_MULTIUSER) // 2
    ws = torch.empty(max(2, U) * single, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    setup_s = time.perf_counter() - t_setup

    def step():
        ts.ts_sinr_svd_multiuser(d, U, cs, Gd, Cd, sd, sinr, flags, ws, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    time.sleep(0.5)
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    clocks = sampler.stop()
    # the link pass of one UE group alone (the groups overlap in the step)
    link_ms = []
    for _ in range(5):
        flush.zero_()
        k0, k1 = ev(), ev()
        k0.record(stream)
        k1.record(stream)
        ts.ts_set_timing_events(k0, k1)
        ts.ts_sinr_svd_multiuser(d, 1, cs, Gd, Cd, sd, sinr, flags, ws, stream)
        ts.ts_set_timing_events(None, None)
        k1.synchronize()
        link_ms.append(k0.elapsed_time(k1))
    assert int((flags & ts.TS_FLAG_ERRORS).max().item()) == 0, "numerical flags raised"
    units = U * J * K
    value = units * args.steps / (total * 1e-3)
    if args.step_only:
        print(json.dumps({"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": total / args.steps, "higher_is_better": True,
                          "link_ms": float(np.mean(link_ms)), "clocks": clocks,
                          "config": {"workload": WORKLOAD_NAME, "U": U}}), flush=True)
        del keep
        return

    # dense comparator on X^ (exact Tucker form, so the same SINR up to
    # rounding); when X^ of every group would not fit comfortably (the
    # (64, 512, 401) channels: 46 GB per group), on the first UE group only,
    # against the compressed path on that group alone
    ud = U if U * nl * P * M * N * 8 <= 64 << 30 else 1
    t_comp_ms = total / args.steps
    if ud < U:
        t_comp_ms = 0.0
        for _ in range(3):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            ts.ts_sinr_svd_multiuser(d, 1, cs, Gd, Cd, sd, sinr, flags, ws, stream)
            b.record(stream)
            b.synchronize()
            t_comp_ms += a.elapsed_time(b) / 3
    Xh = torch.empty(ud * nl, P, M, N, **c64)
    wsr = ts.workspace(d, ts.TS_OP_RECONSTRUCT, dev)
    for u in range(ud):
        ts.ts_tucker_reconstruct(d, ts.TS_MODEL_GROUPWISE, Ad[u], Bd, Cd[u * nl:(u + 1) * nl],
                                 Gd[u * nl:(u + 1) * nl], Xh[u * nl:(u + 1) * nl], wsr, stream)
    del wsr
    sinr_d = torch.empty(ud, J, K, L, device=dev)
    flags_d = torch.empty(ud, J, K, dtype=torch.uint8, device=dev)
    wsd = torch.empty(max(2, ud) * (ts.ts_workspace_bytes(d, ts.TS_OP_DENSE_SVD_MULTIUSER) // 2),
                      dtype=torch.uint8, device=dev)             # concurrent groups, as above

    def dense_step():
        ts.ts_dense_sinr_svd_multiuser(d, ud, cs, Xh, sd, sinr_d, flags_d, wsd, stream)

    dense_step()
    torch.cuda.synchronize()
    dsteps = max(3, args.steps // 10)
    dense_ms = 0.0
    for _ in range(dsteps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        dense_step()
        b.record(stream)
        b.synchronize()
        dense_ms += a.elapsed_time(b)
    step()
    torch.cuda.synchronize()
    st, sdn = sinr[:ud].double(), sinr_d.double()
    agree = float(((st - sdn).abs() / sdn.abs()).max().item())
    del Xh, wsd

    # the FP64 oracle on UE groups 0 and 1 (their SINRs depend on no other
    # group) and slices of 2 subcarriers, about 12 s (not at sizes whose
    # Tucker form is drawn on the device: no host copy)
    from oracle import sinr as S
    cpu_base, sinr_err = None, None
    if len(host) == min(U, 2):
        G2 = np.stack([host[u][0] for u in range(min(U, 2))])
        C2 = np.stack([host[u][1] for u in range(min(U, 2))])
        s22 = np.stack([host[u][4] for u in range(min(U, 2))])
        got = sinr[:min(U, 2)].cpu().numpy().astype(np.float64)
        coef_all = np.stack([S.coefficients(host[u][2], host[u][3], K, w.delta_f_hz)
                             for u in range(min(U, 2))])
        kslice, start, done, errs = 2, 0, 0, []
        c0, t1 = time.process_time(), time.perf_counter()
        while time.perf_counter() - t1 < 12.0:
            ks = [(start + j) % K for j in range(kslice)]
            coef = coef_all[:, :, :, ks]
            ref = S.tucker_sinr_multiuser(G2, C2, coef, s22, L)
            if len(errs) < 4:
                errs.append((np.abs(got[:, :, ks] - ref) / np.abs(ref)).ravel())
            done += min(U, 2) * J * kslice
            start += kslice
        wall = time.perf_counter() - t1
        e = np.concatenate(errs)
        cpu_base = {"value": done / wall, "unit": METRIC,
                    "cores": max(1, round((time.process_time() - c0) / wall)), "kind": "oracle",
                    "sample": f"FP64 NumPy oracle, UE groups 0-{min(U, 2) - 1} on slices of "
                              f"{kslice} subcarriers for 12 s ({done} subcarrier-SINRs)"}
        sinr_err = {"max_rel": float(e.max()), "median_rel": float(np.median(e)), "n": int(e.size)}
    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    lf = link_flops(w, "svd")
    lmean = float(np.mean(link_ms))
    achieved = lf / (lmean * 1e-3) / 1e12
    traffic, traffic_basis = wide_link_traffic(w)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"{WORKLOAD_NAME}: J={J} cells x U={U} UEs, first-UE inter-cell "
                                f"interference, M={M}, N={N}, P={P}, K={K} subcarriers, ranks "
                                f"(m,n,p)=({m},{n},{p}), L={L}; svd-precoded MMSE SINR; path-form "
                                "coefficients; Tucker form drawn directly"),
                   "units_per_step": units, "l2": "flushed before every timed step (256 MiB write)",
                   "setup_seconds": round(setup_s, 1)},
        "roofline": {"kernel": "k_sinr_link_wide (svd)", "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak, 4),
                     "traffic": traffic, "traffic_basis": traffic_basis,
                     "flops_per_launch": lf, "kernel_ms": round(lmean, 4),
                     "peak_basis": f"FP32 FFMA: {sms} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz",
                     "launch": "one UE group (J(J-1) interfering links x K subcarriers)"},
        "gpu_launches": svd_launches(w) * U * args.steps,
        "clocks": clocks,
        "dense_comparator": {"value": ud * J * K * dsteps / (dense_ms * 1e-3), "unit": METRIC,
                             "ms_per_step": dense_ms / dsteps, "ue_groups": ud,
                             "what": f"the same SINR from X^ = G x1 A x2 B x3 C (M={M}, N={N}, "
                                     f"P={P}) on the same GPU kernels"
                                     + ("" if ud == U else "; the first UE group only, R_t against "
                                        "the compressed path on that group alone"),
                             "max_rel_diff_vs_compressed": agree},
        "R_t": (dense_ms / dsteps) / t_comp_ms,
        "R_s": T.storage_ratio(J, U, M, N, P, m, n, p, "groupwise"),
        "cpu_baseline": cpu_base,
        "sinr_err": sinr_err,
    }
    print(json.dumps(line), flush=True)
    del keep


def run_paper_method(args):
    """e_c (eq. 30) at the paper's sizes: the groupwise form fitted on the GPU
    (Algorithm 2, `sweeps` sweeps, 8 inner iterations per large eigensolve)
    from synthetic channels of the first UE of every cell (J = 21, (M, N, P)
    and the workload's ranks; spatially correlated NLOS submatrices), then
    the SVD-precoded SINR from the fitted form against the dense-channel
    SINR on the same channels, both on the GPU; with the fit's time per
    sweep and the storage ratio of eq. (29)."""
    import torch

    from oracle import tucker as T
    from paper_2401_09792_gb300 import tuckersinr as ts
    import __graft_entry__
    __graft_entry__.build()
    ts.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = dataclasses.replace(WORKLOAD, U=1, nlos_corr=synth.MID_CORR.nlos_corr)
    J, K, L, M, N, P, m, n, p = w.J, w.K, w.L, w.M, w.N, w.P, w.m, w.n, w.p
    sweeps = 3
    t0 = time.perf_counter()
    Xd = ts.channels_to_device(synth.channel_submatrices(w), dev)
    gen_s = time.perf_counter() - t0
    alpha, tau = synth.path_gains_delays(w)
    s2 = synth.noise_powers(w)
    al = ts.factor_to_device(alpha.reshape(J * J, P), dev)
    ta = ts.real_to_device(tau.reshape(J * J, P), dev)
    sig = ts.real_to_device(s2, dev)
    cs, keep = ts.make_coef(alpha=al, tau=ta)
    d = ts.Dims.of(w)
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    c64 = dict(dtype=torch.complex64, device=dev)
    A = torch.empty(J, M, m, **c64)
    B = torch.empty(J, N, n, **c64)
    C = torch.empty(J * J, P, p, **c64)
    G = torch.empty(J * J, p, m, n, **c64)
    g = torch.empty(3 * sweeps + 1, dtype=torch.float64, device=dev)
    wsf = ts.workspace(d, ts.TS_OP_TUCKER_FIT, dev)
    ts.ts_set_fit_iterations(8)
    a, b = ev(), ev()
    a.record(stream)
    ts.ts_tucker_fit(d, Xd, sweeps, 0, A, B, C, G, g, wsf, stream)
    b.record(stream)
    b.synchronize()
    ts.ts_set_fit_iterations(0)
    fit_ms = a.elapsed_time(b)
    del wsf
    s_t = torch.empty(J, K, L, device=dev)
    s_d = torch.empty_like(s_t)
    ts.ts_sinr_svd(d, cs, G, C, sig, s_t, None, ts.workspace(d, ts.TS_OP_SINR_SVD, dev), stream)
    ts.ts_dense_sinr_svd(d, cs, Xd, sig, s_d, None, ts.workspace(d, ts.TS_OP_DENSE_SVD, dev), stream)
    torch.cuda.synchronize()
    st, sd = s_t.double(), s_d.double()
    x2 = float((Xd.abs() ** 2).sum().item())
    line = {"metric": "e_c at the paper's sizes (eq. 30)",
            "workload": (f"{WORKLOAD_NAME} first UEs: J={J}, M={M}, N={N}, P={P}, K={K} subcarriers, "
                         f"ranks ({m},{n},{p}), L={L}; NLOS correlation {w.nlos_corr}"),
            "e_c": float(((st - sd).abs() / sd.abs()).mean().item()),
            "g_over_x2": float(g[-1].item()) / x2, "g_history": [float(v) / x2 for v in g.cpu().tolist()],
            "fit_ms": round(fit_ms, 1), "fit_ms_per_sweep": round(fit_ms / sweeps, 1),
            "fit_sweeps": sweeps, "fit_inner_iterations": 8,
            "R_s_one_ue_per_cell": T.storage_ratio(J, 1, M, N, P, m, n, p, "groupwise"),
            "channel_generation_s": round(gen_s, 1),
            "what": "Tucker form fitted on the GPU from the synthetic channels; both SINRs on the GPU"}
    print(json.dumps(line), flush=True)
    del keep


def run_rank_sweep(args):
    """Fig. 5 of the paper on synthetic channels: vary the compressed column
    count n with (m, p) fixed, then p with (m, n) fixed, and report for
    every point the storage ratio R_s (eq. 29), the GPU speedup
    R_t = t_dense / t_compressed of the SVD-precoded SINR, and e_c (eq. 30)
    of the groupwise form fitted on the GPU (Algorithm 2, 10 sweeps)."""
    import torch

    from oracle import tucker as T
    from paper_2401_09792_gb300 import tuckersinr as ts
    import __graft_entry__
    __graft_entry__.build()
    ts.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = WORKLOAD
    J, K, L, M, N, P = w.J, w.K, w.L, w.M, w.N, w.P
    alpha, tau = synth.path_gains_delays(w)
    s2 = synth.noise_powers(w)
    al = ts.factor_to_device(alpha.reshape(J * J, P), dev)
    ta = ts.real_to_device(tau.reshape(J * J, P), dev)
    sig = ts.real_to_device(s2, dev)
    cs, keep = ts.make_coef(alpha=al, tau=ta)
    Xd = ts.channels_to_device(synth.channel_submatrices(w), dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    d0 = ts.Dims.of(w)
    s_d = torch.empty(J, K, L, device=dev)
    wsd = ts.workspace(d0, ts.TS_OP_DENSE_SVD, dev)
    t_dense = timed(lambda: ts.ts_dense_sinr_svd(d0, cs, Xd, sig, s_d, None, wsd, stream))
    sd = s_d.double()
    del wsd
    m0, n0, p0 = w.m, w.n, w.p
    if n0 >= 64:
        # the paper's sizes: coarser grid, 3 sweeps with 8 inner iterations
        # per large eigensolve (the fit costs ~14 s per sweep here)
        points = [(m0, n, p0) for n in (32, 64, n0, 200) if n <= N and L <= n] + \
                 [(m0, n0, p) for p in (30, 60, 90) if p <= P and p != p0]
        sweeps = 3
        ts.ts_set_fit_iterations(8)
    else:
        points = [(m0, n, p0) for n in (8, 16, 24, 32, 48, 64) if n <= N and L <= n] + \
                 [(m0, n0, p) for p in (2, 4, 8, 16, 24, 32) if p <= P and p != p0]
        sweeps = 10
    rows = []
    for (m, n, p) in points:
        d = ts.Dims(J, M, N, P, m, n, p, K, L)
        A = torch.empty(J, M, m, dtype=torch.complex64, device=dev)
        B = torch.empty(J, N, n, dtype=torch.complex64, device=dev)
        C = torch.empty(J * J, P, p, dtype=torch.complex64, device=dev)
        G = torch.empty(J * J, p, m, n, dtype=torch.complex64, device=dev)
        g = torch.empty(3 * sweeps + 1, dtype=torch.float64, device=dev)
        wsf = ts.workspace(d, ts.TS_OP_TUCKER_FIT, dev)
        t0 = time.perf_counter()
        ts.ts_tucker_fit(d, Xd, sweeps, 0, A, B, C, G, g, wsf, stream)
        torch.cuda.synchronize()
        fit_s = time.perf_counter() - t0
        del wsf
        s_t = torch.empty(J, K, L, device=dev)
        wss = ts.workspace(d, ts.TS_OP_SINR_SVD, dev)
        t_t = timed(lambda: ts.ts_sinr_svd(d, cs, G, C, sig, s_t, None, wss, stream))
        st = s_t.double()
        rows.append({"m": m, "n": n, "p": p,
                     "R_s": T.storage_ratio(J, 1, M, N, P, m, n, p, "groupwise"),
                     "R_t": t_dense / t_t, "sinr_ms": round(t_t, 4),
                     "e_c": float(((st - sd).abs() / sd.abs()).mean().item()),
                     "g_over_x2": float(g[-1].item()) / float((Xd.abs() ** 2).sum().item()),
                     "fit_s": round(fit_s, 2)})
        del A, B, C, G, wss
    ts.ts_set_fit_iterations(0)
    line = {"metric": "rank sweep (Fig. 5 analogue)", "workload": workload_config(w)["workload"],
            "fit_sweeps": sweeps, "nlos_corr": w.nlos_corr,
            "dense_sinr_ms": round(t_dense, 4), "points": rows,
            "what": "n swept with (m, p) fixed, then p with (m, n) fixed; Tucker form fitted on the "
                    "GPU from the synthetic channels; R_t and e_c against the dense-channel SINR "
                    "on the same GPU kernels"}
    print(json.dumps(line), flush=True)
    del keep


# ------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import sinr as S
    w = WORKLOAD
    if w.U > 1:
        # UE groups 0 and 1 (the SINRs of group u depend on groups 0 and u only)
        groups = [synth.direct_tucker(w, ue=u) for u in range(2)]
        pg = [synth.path_gains_delays(w, ue=u) for u in range(2)]
        Gm = np.stack([t["G"] for t in groups])
        Cm = np.stack([t["C"] for t in groups])
        s2m = np.stack([synth.noise_powers(w, ue=u) for u in range(2)])
        coefm = np.stack([S.coefficients(a, t, w.K, w.delta_f_hz) for a, t in pg])
        kslice = 2

        def one(start):
            sl = slice(start % w.K, start % w.K + kslice)
            S.tucker_sinr_multiuser(Gm, Cm, coefm[:, :, :, sl], s2m, w.L)
        units_per = 2 * w.J * kslice
    else:
        tk = synth.direct_tucker(w)
        alpha, tau = synth.path_gains_delays(w)
        s2 = synth.noise_powers(w)
        coef = S.coefficients(alpha, tau, w.K, w.delta_f_hz)
        kslice = 128

        def one(start):
            sl = slice(start % w.K, start % w.K + kslice)
            S.tucker_sinr(tk["G"], tk["C"], coef[:, :, sl], s2, w.L, "svd")
        units_per = w.J * kslice

    for s in range(args.warmup):
        one(s * kslice)
    c0 = time.process_time()
    t0 = time.perf_counter()
    for s in range(args.steps):
        one(s * kslice)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    units = units_per * args.steps
    value = units / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w), "parallelism": "none (host CPU)",
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": max(1, round(cpu / wall)),
                         "kind": "oracle",
                         "sample": f"each step: FP64 NumPy oracle on {kslice} of the {w.K} "
                                   f"subcarriers ({units_per} subcarrier-SINRs"
                                   f"{', UE groups 0 and 1' if w.U > 1 else ''}); "
                                   f"{os.cpu_count()} host cores visible"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--step-only", action="store_true",
                    help="time only the SVD step (no end-to-end, variant or comparator runs)")
    ap.add_argument("--workload", default="diff", choices=sorted(synth.WORKLOADS) + ["batch"],
                    help="synthetic system of the timed step (default: diff, the largest "
                         "single-GPU workload, the headline)")
    ap.add_argument("--batch-instances", type=int, default=4096,
                    help="systems of the batch workload")
    ap.add_argument("--ue-groups", type=int, default=None,
                    help="UEs per cell of a several-UE workload (default: the workload's)")
    ap.add_argument("--paper-method", action="store_true",
                    help="paper-scale workloads: fit the first UEs' channels on the GPU and report e_c")
    ap.add_argument("--rank-sweep", action="store_true",
                    help="sweep the compressed sizes n, then p, on the workload (default mid_corr): "
                         "R_s, R_t and e_c per point")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the timing of the SVD-SINR adjoint (dSINR -> dG, dC) on the workload")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32", "bf16x2", "tf32x3"],
                    help="arithmetic of the interfering links' core contraction in the timed step "
                         "(fp32: FMA pipe; tf32, bf16x2, tf32x3: tensor cores; default tf32x3, "
                         "which keeps every SINR within 1e-5 of the FP64 oracle)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch":
        run_batch(args)
        return
    if args.rank_sweep:
        select_workload("mid_corr" if args.workload in ("mid", "diff") else args.workload)
        if WORKLOAD.U > 1:
            # the first UE of every cell, spatially correlated NLOS
            set_ue_groups(1)
            set_nlos_corr(synth.MID_CORR.nlos_corr)
        run_rank_sweep(args)
        return
    select_workload(args.workload)
    several = WORKLOAD.U > 1
    if args.ue_groups is not None:
        set_ue_groups(args.ue_groups)
    if args.impl == "reference":
        run_reference(args)
    elif several and args.paper_method:
        run_paper_method(args)
    elif several:
        run_multiuser(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
