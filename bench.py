#!/usr/bin/env python
"""Benchmark of the R -> K -> Omega hot path: energy-solves per second.

One step = every energy of the workload through near-pole check, channel
functions, R formation, matching solve, T and Omega accumulation (one
partial wave, 64 channels, 1920 poles, 20000 energies per GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32|bf16x3]
  python bench.py --impl reference ...     # the oracle on the host cores

Under torchrun (N > 1) each rank solves its own 20000 energies of an
N*20000-point grid, taken with stride N (the paper's interleaved energy
assignment); no collective is needed on the data path (weak scaling).
Prints one JSON line on rank 0.
"""
import argparse
import json
import multiprocessing as mproc
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("R→K→Ω energy-solves/sec vs plain FP64 GPU path at stated "
          "Ω error; p50/p99 latency")
UNIT = "energy-solves/s"
WORKLOAD = ("one partial wave: 64 channels (thresholds 0-2 Ry, l 0-8, z=2), 1920 poles "
            "on [-2,60] Ry, w~N(0,0.05^2), a=15, 20000 energies on 0.01-2.5 Ry per GPU")
N_E = 20000
# FP64 rate of a GB300 SM: the nominal 1.25 TFLOP/s at the 2070 MHz maximum SM
# clock over 152 SMs is 4 FP64 flops per clock per SM (2 DFMA).
FP64_FLOPS_PER_CLK_SM = 4.0
N_SM = 152
PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------
# oracle legs (CPU)

def _oracle_chunk(args):
    import oracle  # noqa: F401  (oracle is test infrastructure; used only in this leg)
    from paper_1909_07321_gb300 import synth
    lo, hi, stride, offset = args
    pws, E = synth.workload_64ch(N_E * stride)
    Es = E[offset::stride][lo:hi]
    t = time.perf_counter()
    res = oracle.solve_energies(pws[0], Es)
    return hi - lo, time.perf_counter() - t, int((res["status"] == 0).sum())


def oracle_throughput(pool, n_cores, per_core):
    """Energy-solves/s of the oracle over a bounded sample, energy-parallel on
    n_cores processes. Returns (value, sample description)."""
    chunks = [(c * per_core * 37 % (N_E - per_core), c * per_core * 37 % (N_E - per_core) + per_core, 1, 0)
              for c in range(n_cores)]
    t = time.perf_counter()
    out = pool.map(_oracle_chunk, chunks)
    wall = time.perf_counter() - t
    n = sum(o[0] for o in out)
    cpu = sum(o[1] for o in out)
    return n / wall, ("%d energies (%d processes x %d contiguous energies) of the 64-channel "
                      "workload, %.1f s CPU" % (n, n_cores, per_core, cpu))


# --------------------------------------------------------------------------
# clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    n_cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    per_core = 6
    with ctx.Pool(n_cores) as pool:
        for _ in range(args.warmup):
            oracle_throughput(pool, n_cores, per_core)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, sample = oracle_throughput(pool, n_cores, per_core)
            vals.append(v)
        wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    pool = None
    n_cores = os.cpu_count() or 1
    if rank == 0 and not args.no_cpu_baseline:
        pool = mproc.get_context("spawn").Pool(n_cores)   # before the first GPU call

    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_07321_gb300 import rmgb, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    pws, Eall = synth.workload_64ch(args.energies * world)
    pw = pws[0]
    E = np.ascontiguousarray(Eall[rank::world])
    n, N = pw["W"].shape
    prec = PREC[args.precision]
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    ctx = rmgb.Context(precision=prec, stream=stream.cuda_stream, device=local_rank)
    ctx.load_pw(0, pw)
    Ed = torch.tensor(E, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            ctx.solve_energies(0, Ed)
            ctx.reset_omega()
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        props = torch.cuda.get_device_properties(dev)
        clk = ClockSampler("GPU-%s" % props.uuid if getattr(props, "uuid", None) else local_rank)
        clk.start()
        time.sleep(0.3)
        ctx.profile_enable(True)
        l0 = ctx.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            ctx.reset_omega()
            ctx.solve_energies(0, Ed)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        launches = ctx.launch_count() - l0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        phase = {p: ctx.profile_get(p) for p in range(rmgb.RM_PH_COUNT)}
        ctx.profile_enable(False)
        clocks = clk.stop()
        t_step = sum(step_ms) / len(step_ms)
        if dist:
            t = torch.tensor([t_step], device=dev)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            t_step = float(t.item())
        value = world * E.size / (t_step * 1e-3)

        # end to end through the public API with host buffers
        E_pin = torch.tensor(E, dtype=torch.float64).pin_memory()
        n_tri = pw["n_levels"] * (pw["n_levels"] + 1) // 2
        om_pin = torch.empty((E.size, n_tri), dtype=torch.float64).pin_memory()
        ctx.collision_strengths(reset=True)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        k2 = max(2, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(k2):
            ctx.solve_energies(0, E_pin.numpy())
            ctx.collision_strengths(om_pin.numpy(), reset=True)
        e2e_s = (time.perf_counter() - t0) / k2
        if dist:
            t = torch.tensor([e2e_s], device=dev)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            e2e_s = float(t.item())
    ctx.close()

    if rank != 0:
        return
    peaks, peak_src = _peaks()
    # dominant kernel: R formation. Algorithmic work n(n+1)/2 MACs per pole
    # per energy = n(n+1) N flops per energy.
    form_n, form_ms = phase[rmgb.RM_PH_FORM]
    flops_per_launch = n * (n + 1) * N * (E.size / max(1, form_n / args.steps))
    achieved = flops_per_launch / (form_ms / max(form_n, 1) * 1e-3) / 1e12
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if prec == 0:
        peak = N_SM * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "form_r_tiled (FP64)",
                "peak_source": "FP64 4 flop/clk/SM x 152 SMs at the sampled SM clock"}
    else:
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "formation",
                "peak_source": "bf16 burst (%s)" % peak_src}
    total_phase_ms = sum(v[1] for v in phase.values())
    cpu = None
    if pool is not None:
        v, sample = oracle_throughput(pool, n_cores, 24)
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": n_cores, "kind": "oracle", "sample": sample}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_channels": n, "n_poles": N,
                       "energies_per_gpu": int(E.size), "formation": args.precision,
                       "mode": "direct", "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "energy-interleaved dp%d" % world},
            "roofline": roof,
            "phases_ms_per_step": {name: phase[p][1] / args.steps for name, p in
                                   [("nearpole", rmgb.RM_PH_NEARPOLE), ("chanfn", rmgb.RM_PH_CHANFN),
                                    ("form", rmgb.RM_PH_FORM), ("fixup", rmgb.RM_PH_FIXUP),
                                    ("solve", rmgb.RM_PH_SOLVE)]},
            "phase_share": {k: (phase[p][1] / total_phase_ms if total_phase_ms else None)
                            for k, p in [("form", rmgb.RM_PH_FORM), ("solve", rmgb.RM_PH_SOLVE),
                                         ("chanfn", rmgb.RM_PH_CHANFN)]},
            "cpu_baseline": cpu,
            "e2e": {"value": world * E.size / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(E.size * 8),
                    "d2h_bytes_per_step": int(E.size * n_tri * 8)},
            "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=list(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--energies", type=int, default=N_E,
                    help="energies per GPU (smaller only for profiler captures)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
