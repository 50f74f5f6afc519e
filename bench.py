#!/usr/bin/env python
"""Benchmark: nodal DG Maxwell right-hand-side throughput on GB300.

Workload (default): the unit cube cut into 24^3 hexahedra x 6 = 82,944
tetrahedra, interior vertices jittered by +-10% of h (seed 1), polynomial
order N=5 (Np=56), eps = mu = 1, PEC walls, upwind flux, initial data the
closed-form (1,1,1) cavity eigenmode, FP32 fields [6][K][Np_pad], LSERK4 with
dt = 0.5 h / N^2. One benchmark step is one LSERK4 time step = five fused
right-hand-side stages. The metric is GDOF/s per right-hand-side evaluation:
5 * DOF * steps / time, DOF = 6 Np K.

Arms:
  default           the CUDA library through the C ABI (device-resident inputs,
                    CUDA-event timing), plus an end-to-end number with the
                    host<->device copies of every step inside the timed region.
                    The line also carries the precision comparison (24^3 N=5 and
                    32^3 N=7, FP32 / BF16x3 / FP16x3 with their errors against
                    stored FP64 samples) and the adjoint block (20^3 N=4, 400
                    steps: adjoint/forward time with checkpoints every 20 steps
                    and with automatic segments, two finite-difference checks).
  --impl reference  the FP64 CPU oracle, timed on the host cores on a bounded
                    sample of the same workload (5 right-hand-side evaluations
                    on a fixed sample of elements per step).
Multi-GPU (torchrun): independent replicas, one per GPU; value = all ranks'
units / max-over-ranks time (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Maxwell DG RHS GDOF/s at N=5/7, TC split vs FP32 at equal error; adjoint cost"
UNIT = "GDOF/s"
STAGES = 5
NUM_SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def flops_per_element(N: int) -> float:
    """Algorithmic flops of one fused stage per element (see the design notes)."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    volume = 2 * 3 * 6 * Np * Np          # Dr, Ds, Dt on six fields
    chain = Np * (6 * 2 * 3 * 2 + 6)      # two physical derivatives per field (3 FMA each) + curls
    flux = 4 * Nfp * 60                   # jumps, cross products, weights per face node
    lift = 2 * 6 * Np * 4 * Nfp           # LIFT on six fields
    update = 6 * Np * (1 + 4)             # material scale + LSERK update
    return float(volume + chain + flux + lift + update)


def bytes_per_element(N: int, Npad: int) -> float:
    """Algorithmic DRAM bytes of one fused LSERK stage per element, averaged
    over the five stages of a step: read u and res, write res and u_out (FP32),
    except that the first stage (a_1 = 0) does not read res; plus the
    per-element geometry (64 B), face geometry (64 B) and face connectivity (32 B)."""
    return (4 * 4 + 3) / 5 * 6 * Npad * 4 + 64 + 64 + 32


# DRAM bytes (read + write) per launch of the stage kernel, the mean over the
# five stages of one step, from an ncu capture of the current kernel;
# keyed by (precision, N, hexahedra per edge, element order); absent where no
# capture of the current kernel exists. The N=7 32^3 entries are the 16^3
# captures scaled by the element count (x8).
NCU_TRAFFIC = {
    ("fp16x3", 5, 24, "hilbert"): 391.75e6, ("bf16x3", 5, 24, "hilbert"): 391.77e6,
    ("fp32", 5, 24, "hilbert"): 394.45e6,
    ("fp16x3", 7, 16, "hilbert"): 220.23e6, ("bf16x3", 7, 16, "hilbert"): 219.47e6,
    ("fp32", 7, 16, "hilbert"): 221.75e6,
    ("fp16x3", 7, 32, "hilbert"): 8 * 220.23e6, ("bf16x3", 7, 32, "hilbert"): 8 * 219.47e6,
    ("fp32", 7, 32, "hilbert"): 8 * 221.75e6,
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(device_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], None, set()
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, p[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_max_ms(ms_local: float, dist, device) -> float:
    """The job's time: the maximum over the replicas of each one's measured
    time (a single process returns its own)."""
    if dist is None:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gdof_s(world: int, dof: int, steps: int, ms: float) -> float:
    """Whole-job throughput: every replica advances its own copy of the
    workload, so the job's units are world x 5 stages x DOF x steps."""
    return world * STAGES * dof * steps / (ms * 1e-3) / 1e9


def make_workload(N: int, n: int, order: str = "hilbert"):
    import workloads as W
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1, order=order)
    return VX, VY, VZ, EToV


def cpu_oracle_rate(N: int, n: int, sample_elems: int, reps: int = 1, order: str = "hilbert"):
    """Oracle (FP64, single thread) right-hand side on a fixed element sample of
    the same mesh: returns (GDOF/s per RHS, seconds, elements)."""
    import numpy as np

    import oracle as O
    import workloads as W
    VX, VY, VZ, EToV = make_workload(N, n, order)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    x, y, z = m.coords()
    u = W.cavity_mode(x, y, z, 0.0)
    elems = np.sort(np.unique((W.uniform(31, sample_elems) * m.K).astype(np.int64)))
    t0 = time.perf_counter()
    for _ in range(reps):
        m.rhs_subset(u, elems)
    dt = time.perf_counter() - t0
    dof = 6 * m.Np * elems.size * reps
    return dof / dt / 1e9, dt, int(elems.size), m, u, elems


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O
    N, n = args.order, args.n
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    # size the per-step sample so that one step (5 RHS evaluations) takes about a second
    _, t1, e1, m, u, _ = cpu_oracle_rate(N, n, 256, order=args.element_order)
    per_elem = t1 / e1
    sample = int(max(64, min(m.K, 1.0 / (STAGES * per_elem))))
    import numpy as np
    import workloads as W
    elems = np.sort(np.unique((W.uniform(31, sample) * m.K).astype(np.int64)))
    for _ in range(args.warmup):
        for _ in range(STAGES):
            m.rhs_subset(u, elems)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(STAGES):
            m.rhs_subset(u, elems)
    dt = time.perf_counter() - t0
    dof = 6 * Np * elems.size
    value = STAGES * dof * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, m.K, Np),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{STAGES} oracle RHS evaluations per step on {elems.size} of {m.K} elements"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, K, Np):
    return {"workload": f"PEC cube cavity, {args.n}^3x6 jittered tets, N={args.order}, upwind, LSERK4",
            "K": int(K), "N": args.order, "Np": Np, "dof": 6 * Np * int(K), "rhs_per_step": STAGES,
            "precision": args.precision, "element_order": args.element_order,
            "l2": "inputs larger than L2 (u, res, u_out: 3 x 6 K Np_pad x 4 B per stage)",
            "parallelism": f"replicas x{args.gpus}"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1211_0582_gb300 as dg
    import workloads as W

    world, rank, local = dist_setup()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    N, n = args.order, args.n
    VX, VY, VZ, EToV = make_workload(N, n, args.element_order)
    K = EToV.shape[0]
    s = dg.Solver(N, precision=args.precision, stream=stream).upload(VX, VY, VZ, EToV)
    x, y, z = s.node_coords()
    u0_host = W.cavity_mode(x, y, z, 0.0)
    h = 1.0 / n
    dt = 0.5 * h / N ** 2
    Np, Npad = s.Np, s.Npad
    dof = 6 * Np * K
    u = s.to_device(u0_host, device)
    res = s.zeros(device)

    # ---- warm-up
    s.step(u, res, dt, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    # ---- device-resident timed region
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0.record(stream)
    s.step(u, res, dt, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = replica_max_ms(ev0.elapsed_time(ev1), dist, device)
    value = job_gdof_s(world, dof, args.steps, ms)
    launches = STAGES * args.steps
    launch_ms = ms / launches

    # sanity: the run must stay finite and bounded (upwind: energy does not grow)
    energy = s.energy(u)

    # ---- end to end: every step takes its input state from pinned host memory
    # and returns its result to host memory (the residual is scratch: the first
    # LSERK4 stage overwrites it without reading it). Consecutive steps are
    # independent problems; they alternate between contexts on their own
    # streams, so one step's copies overlap another step's compute (all inside
    # the timed region).
    # its own step count (not --steps): the pipeline over the streams needs a
    # few steps to fill and drain, which a short run would mostly measure
    e2e_steps = max(1, args.e2e_steps)
    u_h = torch.empty((6, K, Npad), dtype=torch.float32).pin_memory()
    u_h.copy_(u.cpu())
    ns = max(1, args.e2e_streams)
    out_h = [torch.empty_like(u_h).pin_memory() for _ in range(ns)]
    streams = [stream] + [torch.cuda.Stream(device) for _ in range(ns - 1)]
    solvers = [s] + [dg.Solver(N, precision=args.precision, stream=streams[j]).upload(VX, VY, VZ, EToV)
                     for j in range(1, ns)]
    ud = [torch.empty_like(u) for _ in range(ns)]
    rd = [torch.empty_like(res) for _ in range(ns)]
    for j in range(ns):  # warm-up of every context
        with torch.cuda.stream(streams[j]):
            ud[j].copy_(u_h, non_blocking=True)
            solvers[j].step(ud[j], rd[j], dt, 1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # three repetitions of the timed pipeline; the median is reported (the
    # figure has varied between runs on boxes with equal host-link rates)
    e2e_reps = []
    for _rep in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        for j in range(1, ns):
            streams[j].wait_event(e0)
        for i in range(e2e_steps):
            j = i % ns
            with torch.cuda.stream(streams[j]):
                ud[j].copy_(u_h, non_blocking=True)
                solvers[j].step(ud[j], rd[j], dt, 1)
                out_h[j].copy_(ud[j], non_blocking=True)
        for j in range(1, ns):
            streams[0].wait_stream(streams[j])
        e1.record(streams[0])
        torch.cuda.synchronize()
        e2e_reps.append(replica_max_ms(e0.elapsed_time(e1), dist, device))
    e2e_ms = statistics.median(e2e_reps)
    field_bytes = 6 * K * Npad * 4
    e2e_value = job_gdof_s(world, dof, e2e_steps, e2e_ms)
    # the host link's own rate on this machine (the end-to-end number is bounded by
    # max(copy in, copy out, step) per step when the streams overlap them)
    h2d_ms = _timed(lambda: [ud[0].copy_(u_h, non_blocking=True) for _ in range(5)], streams[0]) / 5
    d2h_ms = _timed(lambda: [out_h[0].copy_(ud[0], non_blocking=True) for _ in range(5)], streams[0]) / 5

    # ---- roofline of the dominant kernel (the fused stage kernel)
    peaks, peak_kind = measured_peaks()
    if args.precision == "fp32":
        peak_tf = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        achieved = flops_per_element(N) * K / (launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": args.traffic or NCU_TRAFFIC.get((args.precision, N, n, args.element_order)),
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"}
    else:
        peak = peaks["hbm_gbs"]
        achieved = bytes_per_element(N, Npad) * K / (launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": args.traffic or NCU_TRAFFIC.get((args.precision, N, n, args.element_order)),
                "algorithmic_bytes": bytes_per_element(N, Npad) * K, "peak_source": f"hbm_gbs ({peak_kind})"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
        "data": "synthetic", "config": config_dict(args, K, Np),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": field_bytes,
                "d2h_bytes_per_step": field_bytes, "steps": e2e_steps,
                "how": "each step: u from pinned host memory, 1 LSERK4 step, u back to pinned host memory (res is "
                       "scratch: stage 1 overwrites it unread); the steps are independent problems (the same "
                       "state advanced by one step each time, not one time-marching run), alternating over "
                       f"{ns} contexts/streams so that copies overlap compute",
                "h2d_gbs": field_bytes / (h2d_ms * 1e-3) / 1e9, "d2h_gbs": field_bytes / (d2h_ms * 1e-3) / 1e9,
                "repeats_ms": e2e_reps, "statistic": "median of 3 repetitions"},
        "gpu_launches": launches, "roofline": roof, "clocks": clk,
        "kernel_ms_per_launch": launch_ms, "energy_after": energy,
    }
    if rank == 0 and world == 1 and not args.no_precisions:
        line["precisions"] = precision_legs(args, stream, headline=(s, args.precision))
    if rank == 0 and world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_leg(stream, steps=400, fd_dirs=2)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, ne, *_ = cpu_oracle_rate(N, n, args.cpu_sample, order=args.element_order)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"1 oracle RHS on {ne} of {K} elements ({secs:.1f} s, FP64, 1 thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def precision_legs(args, stream, headline=None):
    """The metric's comparison on its two workloads, each in FP32 (CUDA cores),
    BF16x3 and FP16x3 (tensor cores): throughput over args.steps LSERK4 steps
    (device-resident, CUDA events) and the relative l2 error against the FP64
    oracle after the workload's full run (500 steps at N=5, 200 at N=7), over
    the 65,536 node values stored by tests/golden/make_precision_refs.py (a
    data file written by the oracle; nothing of the oracle runs here).
    `headline` = (solver, precision) reuses the headline context for its precision."""
    import numpy as np

    import paper_1211_0582_gb300 as dg
    import workloads as W
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_precision_refs as R
    peaks, peak_kind = measured_peaks()
    out = {}
    for name in ("cavity_n5_24cube_500steps", "precision_n7_32cube_200steps"):
        c, mesh, eps, dt = R.setup(name, args.element_order)
        try:
            ref = R.load(name)
        except OSError:
            ref = None
        N, K = c["N"], mesh[3].shape[0]
        leg = {"workload": f"{c['n']}^3x6 = {K} jittered tets, N={N}, "
                           f"{'eps U[1,4] per element' if eps is not None else 'eps=mu=1'}, cavity-mode start, "
                           f"upwind, LSERK4 dt=0.5h/N^2, {args.element_order} element order",
               "error_reference": None if ref is None else str(ref["source"]),
               "error_steps": c["steps"], "error_samples": None if ref is None else int(ref["idx"].size)}
        u0_host = None
        for prec in ("fp32", "bf16x3", "fp16x3"):
            if headline is not None and headline[1] == prec and N == args.order and c["n"] == args.n \
                    and eps is None:
                sv = headline[0]
            else:
                sv = dg.Solver(N, precision=prec, stream=stream).upload(*mesh, eps=eps)
            if u0_host is None:
                x, y, z = sv.node_coords()
                u0_host = W.cavity_mode(x, y, z, 0.0)
                del x, y, z
            u, r = sv.to_device(u0_host), sv.zeros()
            sv.step(u, r, dt, args.warmup)
            ms = _timed(lambda: sv.step(u, r, dt, args.steps), stream)
            dof = 6 * sv.Np * K
            launch_ms = ms / (STAGES * args.steps)
            e = {"gdof_s": STAGES * dof * args.steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / args.steps}
            if prec == "fp32":
                peak_tf = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
                e["alu_frac"] = flops_per_element(N) * K / (launch_ms * 1e-3) / 1e12 / peak_tf
            else:
                e["hbm_frac"] = bytes_per_element(N, sv.Npad) * K / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
                e["traffic"] = NCU_TRAFFIC.get((prec, N, c["n"], args.element_order))
            if ref is not None:
                u, r = sv.to_device(u0_host), sv.zeros()
                sv.step(u, r, dt, c["steps"])
                sv.sync()
                idx = R.renumber_samples(ref["idx"], c["n"], args.element_order, sv.Np)
                got = u[:, :, :sv.Np].reshape(-1)[torch_index(idx, u.device)].double().cpu().numpy()
                e["rel_l2_vs_fp64"] = float(np.linalg.norm(got - ref["ref"]) / np.linalg.norm(ref["ref"]))
                e["max_abs_err_rel_to_max"] = float(np.abs(got - ref["ref"]).max() / float(ref["max_full"]))
            leg[prec] = e
            del u, r
            if sv is not (headline[0] if headline else None):
                del sv
        leg["speedup_vs_fp32"] = {p: leg[p]["gdof_s"] / leg["fp32"]["gdof_s"] for p in ("bf16x3", "fp16x3")}
        out[f"N{N}_{c['n']}cube"] = leg
    return out


def torch_index(idx, device):
    import torch
    return torch.as_tensor(idx, dtype=torch.int64, device=device)


def _timed(fn, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_precision(args):
    """Split-precision tensor-core forms vs the FP32 CUDA-core form: speed on
    the workload mesh and relative l2 error against the FP64 oracle on a small
    version of it (same N, same materials rule, fewer steps)."""
    import numpy as np
    import torch

    import oracle as O
    import paper_1211_0582_gb300 as dg
    import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    N, n = args.order, args.n
    eps_rule = args.order >= 7
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2) if eps_rule else None
    # error reference: the same setup on a 6^3 mesh, 20 steps, against the oracle
    ne_ref, steps_ref = 6, 20
    sVX, sVY, sVZ, sE = W.kuhn_cube(ne_ref, jitter=0.1, seed=1)
    seps = W.element_eps(sE.shape[0], seed=2) if eps_rule else None
    m = O.Mesh(N, sVX, sVY, sVZ, sE, eps=None if seps is None else seps.astype(np.float64))
    x, y, z = m.coords()
    su0 = W.cavity_mode(x, y, z, 0.0)
    sdt = 0.5 / ne_ref / N ** 2
    ref, _ = m.lserk(su0, sdt, steps_ref)
    out = {}
    for prec in ("fp32", "bf16x3", "fp16x3"):
        try:
            s = dg.Solver(N, precision=prec, stream=stream).upload(VX, VY, VZ, EToV, eps=eps)
        except dg.DGError as e:
            out[prec] = {"unsupported": str(e)}
            continue
        xx, yy, zz = s.node_coords()
        u = s.to_device(W.cavity_mode(xx, yy, zz, 0.0))
        res = s.zeros()
        dt = 0.5 / n / N ** 2
        s.step(u, res, dt, args.warmup)
        ms = _timed(lambda: s.step(u, res, dt, args.steps), stream)
        ss = dg.Solver(N, precision=prec, stream=stream).upload(sVX, sVY, sVZ, sE, eps=seps)
        su, sr = ss.to_device(su0), ss.zeros()
        ss.step(su, sr, sdt, steps_ref)
        err = float(np.linalg.norm(ss.from_device(su) - ref) / np.linalg.norm(ref))
        dof = 6 * s.Np * K
        out[prec] = {"gdof_s": STAGES * dof * args.steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / args.steps,
                     "rel_l2_vs_fp64": err}
    fp32 = out["fp32"]["gdof_s"]
    best = max((v["gdof_s"], k) for k, v in out.items() if "gdof_s" in v)
    line = {"metric": METRIC, "value": best[0], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": best[1], "data": "synthetic",
            "config": {"workload": f"precision form, {n}^3x6 jittered tets, N={N}, "
                                   f"{'eps U[1,4] per element' if eps_rule else 'eps=mu=1'}, LSERK4",
                       "K": K, "error_reference": f"FP64 oracle, {ne_ref}^3x6 version, {steps_ref} steps"},
            "precisions": out, "speedup_vs_fp32": {k: v["gdof_s"] / fp32 for k, v in out.items() if "gdof_s" in v}}
    print(json.dumps(line), flush=True)


def run_ensemble(args):
    """64 meshes (n^3 x 6, n uniform in {8..20}), N=4, own eps and dt each,
    Gaussian-pulse initial data: one persistent launch per call from a CUDA
    graph vs one dg_step per mesh (FP32), and the same persistent launch with
    the FP16x3 tensor-core stage (FP32 fields)."""
    import numpy as np
    import torch

    import paper_1211_0582_gb300 as dg
    import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    N = 4
    ns = W.ensemble_sizes(args.ens_meshes, seed=3)
    meshes, epss, dts = [], [], []
    for i, n in enumerate(ns):
        VX, VY, VZ, EToV = W.kuhn_cube(int(n), jitter=0.1, seed=10 + i)
        meshes.append((VX, VY, VZ, EToV))
        epss.append(W.element_eps(EToV.shape[0], seed=100 + i))
        dts.append(0.5 / int(n) / N ** 2)
    ens = dg.Solver(N, stream=stream).upload_ensemble(meshes, epss, dts)
    off = ens.ensemble_layout()
    Ktot = int(off[-1])
    u = torch.zeros((6, Ktot, ens.Npad), dtype=torch.float32, device="cuda")
    singles = []
    for i, mesh in enumerate(meshes):
        sgl = dg.Solver(N, stream=stream).upload(*mesh, eps=epss[i])
        x, y, z = sgl.node_coords()
        u[:, off[i]:off[i + 1]] = sgl.to_device(W.gaussian_pulse(x, y, z, seed=7, index=i))
        singles.append(sgl)
    res = torch.zeros_like(u)
    u_init = u.clone()
    ens.ensemble_tune(force=True)
    best, ebs, tms = ens.ensemble_tuning()
    gbest, geb, gbps, gms = ens.ensemble_tuning_grid()
    steps, warm = args.steps, max(3, args.warmup)
    ens.ensemble_step(u, res, warm)
    ms = _timed(lambda: ens.ensemble_step(u, res, steps), stream)
    graph = ens.ensemble_graph_used()
    dof = 6 * ens.Np * Ktot
    value = STAGES * dof * steps / (ms * 1e-3) / 1e9
    # per-mesh launches of the ordinary stage kernel, same total work
    us = [u[:, off[i]:off[i + 1]].contiguous() for i in range(len(meshes))]
    rs = [torch.zeros_like(x) for x in us]
    def per_mesh(nst):
        for i, sgl in enumerate(singles):
            sgl.step(us[i], rs[i], dts[i], nst)
    per_mesh(warm)
    ms2 = _timed(lambda: per_mesh(steps), stream)
    # the FP16x3 tensor-core form of the same persistent launch, and its
    # difference from the FP32 form after 10 steps
    ens16 = dg.Solver(N, precision="fp16x3", stream=stream).upload_ensemble(meshes, epss, dts)
    u16, r16 = u_init.clone(), torch.zeros_like(u)
    ens16.ensemble_step(u16, r16, warm)
    ms16 = _timed(lambda: ens16.ensemble_step(u16, r16, steps), stream)
    ua, ub = u_init.clone(), u_init.clone()
    ens.ensemble_step(ua, res, 10)
    ens16.ensemble_step(ub, r16, 10)
    torch.cuda.synchronize()
    diff16 = float((ub - ua).norm() / ua.norm())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ensemble of {len(meshes)} jittered cube meshes, n^3x6 with n in {{8..20}}, N=4, "
                                   "eps U[1,4] per element, Gaussian pulse, LSERK4 with per-mesh dt",
                       "meshes": len(meshes), "K_total": Ktot, "dof": dof},
            "persistent_graph": {"gdof_s": value, "ms_per_step": ms / steps, "graph_replay": graph,
                                 "launches_per_call": 1},
            "per_mesh_launches": {"gdof_s": STAGES * dof * steps / (ms2 * 1e-3) / 1e9, "ms_per_step": ms2 / steps,
                                  "launches_per_step": 5 * len(meshes)},
            "autotune": {"elements_per_block": ebs, "ms_per_step": tms, "chosen": best,
                         "grid": {"elements_per_block": geb, "blocks_per_sm": gbps, "ms_per_step": gms,
                                  "chosen_candidate": gbest}},
            "fp16x3_persistent": {"gdof_s": STAGES * dof * steps / (ms16 * 1e-3) / 1e9, "ms_per_step": ms16 / steps,
                                  "graph_replay": ens16.ensemble_graph_used(), "tile_elements": 20,
                                  "rel_l2_vs_fp32_after_10_steps": diff16}}
    print(json.dumps(line), flush=True)


def adjoint_leg(stream, steps: int = 400, fd_dirs: int = 16, precision: str = "fp32") -> dict:
    """Adjoint workload: 20^3 x 6 jittered tets, N=4, FP32, 256 receivers, `steps`
    steps; adjoint-to-forward cost with checkpoints every 20 steps and with the
    segment length the library picks from the free device memory (the whole run
    in one stored segment when it fits), and a finite-difference check of the
    eps gradient along `fd_dirs` random directions."""
    import torch

    import paper_1211_0582_gb300 as dg
    import workloads as W
    N, n, ck = 4, 20, 0
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2)
    s = dg.Solver(N, precision=precision, stream=stream).upload(VX, VY, VZ, EToV, eps=eps)
    x, y, z = s.node_coords()
    u0 = s.to_device(W.gaussian_pulse(x, y, z, seed=7))
    recv = torch.as_tensor(W.receivers(K, s.Np, 256, seed=4), device="cuda")
    dt = 0.5 / n / N ** 2
    epsd = torch.as_tensor(eps, device="cuda")
    Eref = s.receiver_traces(u0, recv, dt, steps, eps=torch.as_tensor(W.element_eps(K, seed=6), device="cuda"))
    s.set_eps(epsd)
    uf, rf = u0.clone(), s.zeros()
    s.step(uf, rf, dt, 3)
    uf, rf = u0.clone(), s.zeros()
    fwd_ms = _timed(lambda: s.step(uf, rf, dt, steps), stream)
    out = {}
    s.adjoint(u0, recv, Eref, dt, steps, ck, eps=epsd)  # warm-up: the work buffers stay in the context
    adj_ms = _timed(lambda: out.setdefault("r", s.adjoint(u0, recv, Eref, dt, steps, ck, eps=epsd)), stream)
    J, g_eps, g_u0 = out["r"]
    seg = s.adjoint_segment_steps()
    # the same gradient with checkpoints every 20 steps (the last two segments
    # stored by the forward sweep, the other 360 of 400 steps recomputed)
    s.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd)
    adj20_ms = _timed(lambda: s.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd), stream)
    form = s.adjoint_form()
    # the same with the reverse stage's contractions on the CUDA cores
    s.set_adjoint_form("cuda")
    s.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd)
    adj20c_ms = _timed(lambda: s.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd), stream)
    if form == "tensor":
        s.set_adjoint_form("tensor")
    # the same gradient in an FP16x3 context: the forward sweeps and the
    # forward it is compared with run the tensor-core stage
    s16 = s if precision == "fp16x3" else \
        dg.Solver(N, precision="fp16x3", stream=stream).upload(VX, VY, VZ, EToV, eps=eps)
    uf16, rf16 = u0.clone(), s16.zeros()
    s16.step(uf16, rf16, dt, 3)
    uf16, rf16 = u0.clone(), s16.zeros()
    fwd16_ms = _timed(lambda: s16.step(uf16, rf16, dt, steps), stream)
    s16.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd)
    adj16_20_ms = _timed(lambda: s16.adjoint(u0, recv, Eref, dt, steps, 20, eps=epsd), stream)
    if s16 is not s:
        del s16
    h = 1e-3
    dirs = 2.0 * W.uniform(5, 16 * K).reshape(16, K)[:fd_dirs] - 1.0
    rels = []
    for d in dirs:
        dd = torch.as_tensor(d, dtype=torch.float64, device="cuda")
        ep, em = (epsd.double() + h * dd).float(), (epsd.double() - h * dd).float()
        Jp = float(((s.receiver_traces(u0, recv, dt, steps, eps=ep).double() - Eref.double()) ** 2).sum())
        Jm = float(((s.receiver_traces(u0, recv, dt, steps, eps=em).double() - Eref.double()) ** 2).sum())
        fd, ad = Jp - Jm, float((g_eps * (ep.double() - em.double())).sum())
        rels.append(abs(fd - ad) / abs(fd))
    dof = 6 * s.Np * K
    return {"workload": f"adjoint, 20^3x6 jittered tets, N=4, {precision} context, 256 receivers, {steps} steps",
            "K": K, "dof": dof, "steps": steps, "forward_ms": fwd_ms,
            "forward_gdof_s": STAGES * dof * steps / (fwd_ms * 1e-3) / 1e9, "J": J,
            "reverse_stage": form + (" cores: FP16x3 tcgen05 transposed contractions, face loop on the CUDA cores"
                                     if form == "tensor" else " cores"),
            "checkpoints_every_20": {"adjoint_ms": adj20_ms, "ratio": adj20_ms / fwd_ms,
                                     "recomputed_steps": max(0, steps - 40),
                                     "cuda_core_reverse": {"adjoint_ms": adj20c_ms, "ratio": adj20c_ms / fwd_ms}},
            "automatic_segments": {"adjoint_ms": adj_ms, "ratio": adj_ms / fwd_ms, "segment_steps": seg,
                                   "recomputed_steps": steps - seg,
                                   "segment_bytes": int(seg * 5 * 1.5 * 6 * K * ((s.Np + 3) // 4 * 4) * 4)},
            "fp16x3_context": {"forward_ms": fwd16_ms, "adjoint_ms_checkpoints_every_20": adj16_20_ms,
                               "ratio": adj16_20_ms / fwd16_ms,
                               "note": "forward sweeps and the forward compared with on the tensor cores: faster "
                                       "gradients than in FP32, against a 2.5x faster forward"},
            "timing": "second call of each (warm-up first; adjoint work buffers kept in the context)",
            "fd_check": {"step": h, "directions": len(rels), "rel_diff": rels, "max_rel_diff": max(rels),
                         "median_rel_diff": statistics.median(rels),
                         "abs_bar": "the tests check |fd - adjoint| <= 1e-6 J (FP32 round-off of the two runs)"}}


def run_adjoint(args):
    """The adjoint workload alone (ratio of the automatic segments as the value;
    16 finite-difference directions)."""
    import torch
    torch.cuda.set_device(0)
    leg = adjoint_leg(torch.cuda.current_stream(), steps=args.steps, fd_dirs=16, precision=args.adjoint_precision)
    line = {"metric": METRIC, "value": leg["automatic_segments"]["ratio"], "unit": "adjoint/forward time",
            "n_gpus": 1, "steps": args.steps, "warmup": 3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.adjoint_precision == "fp32" else args.adjoint_precision,
            "data": "synthetic",
            "config": {"workload": leg["workload"] + " (value: automatic segments)", "K": leg["K"],
                       "dof": leg["dof"]}, "adjoint": leg}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3", "fp16x3"], default="fp16x3")
    ap.add_argument("--order", type=int, default=5)
    ap.add_argument("--n", type=int, default=24, help="hexahedra per cube edge")
    ap.add_argument("--element-order", choices=["hilbert", "lexicographic"], default="hilbert",
                    help="element numbering of the cube mesh (hexahedra along a 3D Hilbert curve, or x fastest)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--e2e-streams", type=int, default=4, help="contexts/streams the end-to-end steps alternate over")
    ap.add_argument("--cpu-sample", type=int, default=50000, help="elements in the oracle CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-precision", choices=["fp32", "bf16x3", "fp16x3"], default="fp32",
                    help="context precision of the adjoint workload (the configuration's is fp32)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="leave the adjoint block (20^3 N=4, 400 steps, cost ratios) out of the default line")
    ap.add_argument("--no-precisions", action="store_true",
                    help="skip the FP32 / BF16x3 / FP16x3 comparison at N=5 (24^3) and N=7 (32^3)")
    ap.add_argument("--workload", choices=["cavity", "precision", "ensemble", "adjoint"], default="cavity",
                    help="cavity: 24^3 N=5 LSERK4 (headline); precision: split vs FP32 error and speed; "
                         "ensemble: 64 meshes in one persistent launch; adjoint: gradient cost and check")
    ap.add_argument("--ens-meshes", type=int, default=64, help="meshes in the ensemble workload")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the stage kernel (from a capture), if known")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cavity":
        run_ours(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    else:
        run_adjoint(args)


if __name__ == "__main__":
    main()
