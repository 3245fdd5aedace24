"""Benchmark of the axisymmetric phase-field MRT-LB step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
                [--workload batched|oscillating|static] [--precision mix_fp16|fp32|...]

Default workload: the batched case set (512 independent static and
oscillating droplet cases, grids drawn from seed 20181022 between 64 x 128 and
256 x 512, density ratios 10/100/1000) advancing together, one kernel launch
per time step, FP32 populations and arithmetic (FP64 mass ledger and
reductions).  The same line reports the 16-bit deviation-stored form.
Per-step inputs (~2.5-4.5 GB of populations) are far larger than L2 (129 MB),
so no flush is needed between steps.  The same JSON line also reports the
plain FP32 single-case path on the 128 x 256 oscillating drop (L2 flushed
between timed steps) and the FP64 path.

One step = one pass of the whole hot path over every case: phi recovery,
stencils, macroscopic recovery, both MRT collisions, streaming with the
boundary rules.  MLUPS = lattice nodes x steps / seconds / 1e6.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline: FP64/FP32 vs mixed-precision/batched at stated error"
# Algorithmic bytes per node update (populations read + written, f_0 -- FP64,
# the double-float ledger of FP32 and bfloat16, or FP16's single FP32 word --,
# chi^{n-1} read + written; the lagged-p array is not touched).
BYTES_PER_NODE = {
    "fp64": 2 * (9 * 8 + 9 * 8 + 2 * 8),       # 320
    "fp32": 2 * (8 + 8 * 4 + 9 * 4 + 2 * 4),    # 168
    "mix_fp16": 2 * (4 + 8 * 2 + 9 * 2 + 2 * 4),  # 92
    "mix_bf16": 2 * (8 + 8 * 2 + 9 * 2 + 2 * 4),  # 100
}
# The wider per-node byte count that also charges the p^{n-1} plane (read and
# written; FP64 also phi once each way); reported beside the count above.
BYTES_PER_NODE_WITH_P = {"fp64": 352, "fp32": 176, "mix_fp16": 100, "mix_bf16": 108}
# The benchmark's cost model per node update: the 36 population values, phi
# written and read once and chi^{n-1}, p^{n-1} read and written (44 values),
# 8 B each in FP64, 4 B in FP32, and with 16-bit storage 4 B for f_0, phi and
# the auxiliary values and 2 B for the other 34 populations.
BYTES_PER_NODE_MODEL = {"fp64": 352, "fp32": 176, "mix_fp16": 108, "mix_bf16": 108}
DTYPE = {"fp64": "f64", "fp32": "f32", "mix_fp16": "f32 (fp16 storage)", "mix_bf16": "f32 (bf16 storage)"}
# DRAM bytes per node update of the step kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the nodes of the captured
# launch), keyed by precision, launch variant and collision basis:
# profiles/step_kernel_seq2_fp32_batched64cases.md (variant 5, the shape the
# autotuner picks for FP32, re-captured on the current build).  Scaled to a
# full launch by the node count.  Kept only for the kernel builds captured
# (another variant reports null).
TRAFFIC_B_PER_NODE = {("fp32", 5, "orthogonal"): 163.88}
# The FP64 step is bound by the FP64 pipe, not by HBM: FP64-pipe thread
# instructions (DADD + DFMA + DMUL) per node update from one ncu capture
# (profiles/step_kernel_fp64_batched64cases.md), against the pipe's rate
# measured in the same run (lbm_measure_fp64_rate: dependent FP64 FMA chains
# timed with CUDA events).
FP64_OPS_PER_NODE = 383.3
# What the GPU parity tests hold each precision to against the FP64 oracle.
PARITY_TOL = {
    "fp64": "phi, rho, u, p within 1e-11 (relative max-norm) of the FP64 oracle",
    "fp32": "static drop, 2000 steps: phi max err < 2e-3, rms < 1e-4; mass drift < 1e-6",
    "mix_fp16": "static drop, 2000 steps: phi max err < 2e-2, rms < 5e-4; mass drift < 1e-6",
    "mix_bf16": "static drop, 2000 steps: phi max err < 0.2, rms < 1e-2; mass drift < 1e-6",
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d.get("hbm_gbs")), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"axilbm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a few hundred ms to print its first sample: wait
            # for it so that the samples cover the whole timed region
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_cases(workload: str, precision: str, rank: int, ncases: int = 512):
    from paper_1810_09299_gb300 import workloads as W
    if workload == "batched":
        cases = W.batched_cases(ncases, seed=20181022 + rank, precision=precision)
    elif workload == "oscillating":
        cases = [dict(W.oscillating_drop(), precision=precision)]
    elif workload == "static":
        cases = [dict(W.static_drop(), precision=precision)]
    else:
        raise ValueError(workload)
    return cases


def time_steps(sim, torch, steps: int, flush=None):
    """Per-step CUDA-event timing on the handle's (torch's current) stream."""
    st = torch.cuda.current_stream()
    times = []
    if flush is None:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(st)
        for i in range(steps):
            sim.step(1)
            ev[i + 1].record(st)
        torch.cuda.synchronize()
        times = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        return times
    for i in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.step(1)
        b.record(st)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return times


def cpu_baseline(case: dict, budget_s: float = 15.0):
    """The FP64 oracle (as it stands) on the host cores, on one case of the
    workload for a bounded number of steps."""
    import oracle
    from paper_1810_09299_gb300 import workloads as W
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    c = dict(case, precision="fp64")
    o = oracle.Oracle(c).init(W.initial_phi(c))
    nodes = c["nr"] * c["nz"]
    t0 = time.perf_counter()
    o.step(2)
    dt = time.perf_counter() - t0
    steps = max(2, int(budget_s / max(dt / 2, 1e-6)))
    steps = min(steps, 5000)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, one {c['nr']}x{c['nz']} case of the workload, {steps} steps "
                      f"({dt:.1f} s, OpenMP over {cores} host threads)"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_cpu_table(args):
    """The FP64 oracle as it stands on this host, single-threaded and on every
    core, on the 64 x 128 static drop and the 128 x 256 oscillating drop
    (2000 steps each): one JSON line per run."""
    import oracle
    from paper_1810_09299_gb300 import workloads as W
    cores = os.cpu_count() or 1
    model = cpu_model()
    for name, case in (("static drop 64x128", W.static_drop()), ("oscillating drop 128x256", W.oscillating_drop())):
        for threads in (1, cores):
            oracle.set_threads(threads)
            o = oracle.Oracle(dict(case, precision="fp64")).init(W.initial_phi(case))
            steps = args.cpu_steps
            t0 = time.perf_counter()
            o.step(steps)
            dt = time.perf_counter() - t0
            print(json.dumps({"workload": name, "steps": steps, "threads": threads, "nproc": cores,
                              "cpu": model, "seconds": dt,
                              "mlups": case["nr"] * case["nz"] * steps / dt / 1e6}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cases = build_cases(args.workload, "fp64", 0)
    c = cases[0]
    nodes = c["nr"] * c["nz"]
    import oracle
    from paper_1810_09299_gb300 import workloads as W
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    o = oracle.Oracle(c).init(W.initial_phi(c))
    # size each step so that warm-up + timed steps stay within a few minutes
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    inner = max(1, int(4.0 / max(per, 1e-6)))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(inner)
    dt = time.perf_counter() - t0
    value = nodes * inner * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.workload}: FP64 CPU oracle on case 0 ({c['nr']}x{c['nz']})",
                       "steps_per_timed_step": inner},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"case 0 of the {args.workload} workload, {inner} oracle steps per "
                                       f"timed step"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cuda(args):
    import torch
    import torch.distributed as dist

    from paper_1810_09299_gb300 import lbm, shard
    from paper_1810_09299_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = args.precision
    cases = build_cases(args.workload, prec, rank, args.cases)
    if args.collision == "raw":
        from paper_1810_09299_gb300 import workloads as W
        cases = [W.with_raw_collision(c) for c in cases]
    nodes = sum(c["nr"] * c["nz"] for c in cases)
    sim = lbm.Simulation(cases)
    for i, c in enumerate(cases):
        sim.init_phase(i, c["shape"], c["shape_args"])
    mass0 = sim.diagnostics(0)["mass"]
    if args.variant is None:
        variant = sim.autotune(reps=2)
    else:
        variant = args.variant
        sim.set_variant(variant)
    flush_buf = None
    if nodes * BYTES_PER_NODE[prec] < 4 * 129e6:
        flush_buf = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")

        def flush():
            flush_buf.fill_(1.0)
    else:
        flush = None
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.kernel_launches
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        times = time_steps(sim, torch, args.steps, flush if flush_buf is not None else None)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    launches = sim.kernel_launches - launches0
    # weak scaling: every rank advances its own case set; the job's throughput
    # is all ranks' nodes over the slowest rank's device time
    value, ms, total_nodes = shard.job_throughput(nodes, args.steps, float(np.sum(times)),
                                                  dist if world > 1 else None, torch.device("cuda", local))
    d = sim.diagnostics(0)
    peak, peak_kind = measured_peaks()
    per_launch_ms = float(np.mean(times))
    achieved = BYTES_PER_NODE[prec] * nodes / (per_launch_ms * 1e-3) / 1e9
    ach_with_p = BYTES_PER_NODE_WITH_P[prec] * nodes / (per_launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": {"batched": f"{len(cases)} batched static/oscillating droplet cases (seed 20181022), "
                                           "grids 64x128..256x512, one launch per step",
                                "oscillating": "oscillating P2 drop, 128x256, R0=32",
                                "static": "static drop, 64x128, R=16"}[args.workload],
                   "precision": prec, "nodes_per_gpu": nodes, "cases_per_gpu": len(cases),
                   "collision": "raw moments" if args.collision == "raw" else "orthogonal (paper)",
                   "l2": "flushed between timed steps" if flush_buf is not None else
                         "inputs larger than L2 (no flush)",
                   "variant": variant, "parallelism": f"independent cases per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (TRAFFIC_B_PER_NODE[(prec, variant, args.collision)] * nodes
                                 if (prec, variant, args.collision) in TRAFFIC_B_PER_NODE else None),
                     "traffic_unit": "bytes per launch (ncu capture of 64 cases scaled by node count)",
                     "note": f"peak {peak_kind}; algorithmic bytes {BYTES_PER_NODE[prec]} B/node x {nodes} nodes "
                             f"per launch / mean CUDA-event launch duration",
                     "bytes_per_node_with_p": BYTES_PER_NODE_WITH_P[prec], "achieved_with_p": ach_with_p,
                     "frac_with_p": ach_with_p / peak, "bytes_per_node_model": BYTES_PER_NODE_MODEL[prec],
                     "frac_model": BYTES_PER_NODE_MODEL[prec] * nodes / (per_launch_ms * 1e-3) / 1e9 / peak},
        "gpu_launches": int(launches),
        # the autotuner restores the state it started from, so d["step"] counts
        # the warm-up and timed steps only
        "stated_error": dict(case_error_vs_fp64(sim, cases[0], int(d["step"]), prec),
                             case0_rel_mass_drift=abs(d["mass"] - mass0) / mass0, case0_steps=d["step"],
                             parity_tolerance=PARITY_TOL[prec]),
    }
    if rank == 0 and not args.no_extra:
        line["graph"] = graph_leg(sim, torch, nodes, args)
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    # ---- end to end through the C ABI with host buffers
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e(cases, args, torch)
    if rank == 0 and not args.no_extra:
        sim.close()
        if args.workload == "batched":
            for other in ("fp32", "mix_fp16", "mix_bf16", "fp64"):
                if other != prec:
                    line[f"batched_{other}"] = batched_other(torch, args, other, steps=min(args.steps, 50)
                                                             if other != "fp64" else 5)
            for other in ("fp32", "mix_fp16"):
                line[f"batched_{other}_raw_collision"] = batched_other(torch, args, other, min(args.steps, 50),
                                                                      raw=True)
        line["single_case_fp32"] = single_case(torch, "oscillating", "fp32", min(args.steps, 50))
        line["single_case_fp64"] = single_case(torch, "oscillating", "fp64", min(max(4, args.steps // 4), 20))
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(cases[0], budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def case_error_vs_fp64(sim, case, steps, prec):
    """Max and L2 (rms over nodes) errors of phi, u_z, u_r and p of the timed
    case 0 against the FP64 GPU path run from the same initial shape for the
    same number of steps (the FP64 path matches the FP64 oracle to 1e-11 in
    the parity tests)."""
    from paper_1810_09299_gb300 import lbm
    got = sim.fields(0)
    ref_sim = lbm.Simulation(dict(case, precision="fp64"))
    ref_sim.init_phase(0, case["shape"], case["shape_args"])
    ref_sim.step(steps)
    ref = ref_sim.fields(0)
    ref_sim.close()
    out = {"against": f"FP64 GPU path, case 0 ({case['nr']}x{case['nz']}), {steps} steps"}
    for k in ("phi", "uz", "ur", "p"):
        e = got[k] - ref[k]
        out[k] = {"max": float(np.max(np.abs(e))), "l2": float(np.sqrt(np.mean(e * e))),
                  "scale": float(np.max(np.abs(ref[k])))}
    return out


def graph_leg(sim, torch, nodes, args):
    """The same handle stepped by lbm_step(n) with n a multiple of the 32-step
    captured CUDA graph: one graph launch per 32 steps, timed with CUDA events
    around the whole call."""
    n = 64
    sim.step(n)  # captures the graph (first use) and warms up
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, min(4, args.steps // n))
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        sim.step(n)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * n)
    return {"value": nodes / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": reps * n,
            "launch": "lbm_step(64): two replays of the captured 32-step graph per call"}


def e2e(cases, args, torch):
    """Same metric through the public API with host buffers: every case's phi0
    uploaded from pinned host memory at the start, then every step one
    lbm_step and one diagnostics record read back to the host.  The headline
    loop uploads all cases with one lbm_init_phase_all and pipelines the
    read-back (lbm_case_diagnostics_enqueue / lbm_diagnostics_wait, two pinned
    record slots): record n is waited for after step n + 1 is enqueued, and
    every record is checked.  The synchronous loop (one lbm_case_init_phase
    per case, lbm_case_diagnostics after every step) is reported beside it."""
    from paper_1810_09299_gb300 import lbm
    from paper_1810_09299_gb300 import workloads as W
    phi_all = torch.from_numpy(np.concatenate([W.initial_phi(c).ravel() for c in cases])).pin_memory()
    phi_np = phi_all.numpy()
    slots = [torch.zeros(11, dtype=torch.float64).pin_memory() for _ in range(2)]
    recs = [lbm.LbmDiag.from_address(t.data_ptr()) for t in slots]
    nodes = sum(c["nr"] * c["nz"] for c in cases)
    offs = np.cumsum([0] + [c["nr"] * c["nz"] for c in cases])
    sim = lbm.Simulation(cases)
    sim.init_all(phi_np)
    sim.step(args.warmup)
    torch.cuda.synchronize()

    def pipelined():
        t0 = time.perf_counter()
        sim.init_all(phi_np)
        for n in range(args.steps):
            sim.step(1)
            sim.diagnostics_enqueue(0, recs[n % 2], n % 2)
            if n > 0:
                if sim.diagnostics_wait((n - 1) % 2) != lbm.LBM_OK or recs[(n - 1) % 2].step != n:
                    raise RuntimeError("pipelined diagnostics record %d" % n)
        if sim.diagnostics_wait((args.steps - 1) % 2) != lbm.LBM_OK:
            raise RuntimeError("pipelined diagnostics: last record")
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def synchronous():
        t0 = time.perf_counter()
        for i in range(len(cases)):
            sim.init_phase(i, "host_array", phi=phi_np[offs[i]:offs[i + 1]].reshape(cases[i]["nz"], cases[i]["nr"]))
        for _ in range(args.steps):
            sim.step(1)
            sim.diagnostics(0)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    dt = pipelined()
    dt_sync = synchronous()
    sim.close()
    h2d = phi_np.nbytes / args.steps
    return {"value": nodes * args.steps / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 88 + 4,
            "read_back": "diagnostics record + status word every step, pipelined one step behind",
            "synchronous": {"value": nodes * args.steps / dt_sync / 1e6, "unit": "MLUPS",
                            "read_back": "lbm_case_init_phase per case; lbm_case_diagnostics after every step"}}


def batched_other(torch, args, prec, steps, raw=False):
    """The same batched case set in another precision (same timing method);
    raw: with the raw-moment collision option instead of the paper's."""
    from paper_1810_09299_gb300 import lbm, workloads as W
    cases = build_cases("batched", prec, 0, args.cases)
    if raw:
        cases = [W.with_raw_collision(c) for c in cases]
    nodes = sum(c["nr"] * c["nz"] for c in cases)
    sim = lbm.Simulation(cases)
    for i, c in enumerate(cases):
        sim.init_phase(i, c["shape"], c["shape_args"])
    variant = sim.autotune(reps=2)
    for _ in range(args.warmup):
        sim.step(1)
    times = time_steps(sim, torch, steps)
    ms = float(np.mean(times))
    peak, kind = measured_peaks()
    ach = BYTES_PER_NODE[prec] * nodes / (ms * 1e-3) / 1e9
    sim.close()
    ach_p = BYTES_PER_NODE_WITH_P[prec] * nodes / (ms * 1e-3) / 1e9
    out = {"precision": prec, "collision": "raw moments" if raw else "orthogonal (paper)",
           "value": nodes / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
           "variant": variant, "achieved_gbs": ach, "frac": ach / peak,
           "bytes_per_node": BYTES_PER_NODE[prec], "frac_with_p": ach_p / peak,
           "bytes_per_node_with_p": BYTES_PER_NODE_WITH_P[prec],
           "bytes_per_node_model": BYTES_PER_NODE_MODEL[prec],
           "frac_model": BYTES_PER_NODE_MODEL[prec] * nodes / (ms * 1e-3) / 1e9 / peak}
    if prec == "fp64":
        gops = FP64_OPS_PER_NODE * nodes / (ms * 1e-3) / 1e9
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            peak = lbm.measure_fp64_rate(iters=20000) / 1e9
        out["alu_roofline"] = {"bound": "alu", "achieved": gops, "peak": peak,
                               "unit": "G FP64-pipe instructions/s", "frac": gops / peak,
                               "peak_kind": "measured: lbm_measure_fp64_rate (dependent FP64 FMA chains, "
                                            "CUDA events)", "peak_clocks": clk.summary(),
                               "note": f"{FP64_OPS_PER_NODE} DADD+DFMA+DMUL per node (ncu)"}
    return out


def single_case(torch, workload, prec, steps):
    from paper_1810_09299_gb300 import lbm
    cases = build_cases(workload, prec, 0)
    c = cases[0]
    sim = lbm.Simulation(c)
    sim.init_phase(0, c["shape"], c["shape_args"])
    sim.autotune(reps=3)
    for _ in range(3):
        sim.step(1)
    buf = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")
    times = time_steps(sim, torch, steps, lambda: buf.fill_(1.0))
    nodes = c["nr"] * c["nz"]
    ms = float(np.mean(times))
    peak, kind = measured_peaks()
    ach = BYTES_PER_NODE[prec] * nodes / (ms * 1e-3) / 1e9
    sim.close()
    return {"workload": f"{workload} {c['nr']}x{c['nz']}", "precision": prec, "value": nodes / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "ms_per_step": ms, "l2": "flushed between timed steps",
            "achieved_gbs": ach, "frac": ach / peak}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "oscillating", "static"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "mix_fp16", "mix_bf16"])
    ap.add_argument("--collision", default="orthogonal", choices=["orthogonal", "raw"],
                    help="moment basis of both collisions (raw: the raw-moment option)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--variant", type=int, default=None, help="step-kernel launch shape (default: autotuned)")
    ap.add_argument("--cases", type=int, default=512, help="number of batched cases")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the FP64 oracle on the host (1 thread and all cores) and exit")
    ap.add_argument("--cpu-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_table:
        run_cpu_table(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
