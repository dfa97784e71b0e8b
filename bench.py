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
PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2}   # fp32 = 3xTF32 on tensor cores


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
    """nvidia-smi clocks and throttle reasons every 20 ms, each sample stamped
    with the host clock, so that stop() can keep the samples taken inside a
    timed window (window(t0, t1)); the window's neighbours are used only when
    the window is shorter than the sampling interval."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.win = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=3.0):
        """Waits until nvidia-smi has printed its first sample."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def window(self, t0, t1):
        self.win = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        lines = self.lines
        in_window = None
        if self.win is not None:
            t0, t1 = self.win
            inside = [x for x in lines if t0 <= x[0] <= t1]
            in_window = len(inside)
            if not inside:   # window shorter than the interval: the samples next to it
                before = [x for x in lines if x[0] < t0][-1:]
                after = [x for x in lines if x[0] > t1][:1]
                inside = before + after
            lines = inside
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
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
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": in_window,
                "interval_ms": self.INTERVAL_MS}


# --------------------------------------------------------------------------

def _one_blas_thread():
    """Oracle processes each use one BLAS thread (set before they import numpy)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _table_sample(cfg, n_energies, part, parts):
    """(partial waves, energies) of a bounded, evenly strided sample of
    configuration cfg: n_energies energies per wave (all 40 waves of the
    batched workload; 8 requests of the serving workload with their own
    energies), part `part` of `parts` for the parallel run."""
    from paper_1909_07321_gb300 import synth
    if cfg == 0:
        pws, E = synth.workload_small(2000)
    elif cfg == 1:
        pws, E = synth.workload_64ch(20000)
    elif cfg == 2:
        pws, E = synth.workload_batched()
    elif cfg == 3:
        pws, E = synth.workload_1000ch()
    else:
        specs = synth.serving_requests(8, 1.0, n_range=(50, 1500), ne_range=(256, 8192), n_sets=64)
        out = []
        for sp in specs:
            Es = sp["E"][np.linspace(0, sp["E"].size - 1, n_energies).round().astype(int)]
            out.append((synth.serving_pole_set(sp["set_id"], sp["n"]), Es[part::parts], sp["mode"]))
        return out
    idx = np.linspace(0, E.size - 1, n_energies).round().astype(int)
    Es = E[idx][part::parts]
    return [(pw, Es, 0) for pw in pws]


def _table_chunk(args):
    import oracle  # noqa: F401  (test infrastructure; this leg only times it)
    cfg, n_energies, part, parts = args
    t = time.perf_counter()
    n = 0
    for pw, Es, mode in _table_sample(cfg, n_energies, part, parts):
        if Es.size:
            oracle.solve_energies(pw, Es, mode=mode)
            n += Es.size
    return n, time.perf_counter() - t


# energies per wave (per request for the serving workload) of each timed
# sample, and the energy-solves of the whole configuration
CPU_TABLE = {0: (2000, 2000), 1: (48, 20000), 2: (2, 40 * 10000), 3: (3, 5000), 4: (2, None)}


def run_cpu_table(args):
    """The oracle on the host cores for every configuration: one process with
    one BLAS thread, and energy-parallel processes over all cores (one BLAS
    thread each), on bounded samples; the whole-configuration time is
    extrapolated linearly in the energy count where the sample is smaller."""
    _one_blas_thread()
    n_cores = os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    rows = {}
    from paper_1909_07321_gb300 import synth
    specs = synth.serving_requests(200, 1.0, n_range=(50, 1500), ne_range=(256, 8192), n_sets=64)
    total4 = sum(sp["E"].size for sp in specs)
    with ctx.Pool(n_cores) as pool:
        for cfg, (ne, total) in CPU_TABLE.items():
            total = total if total is not None else total4
            n1, t1 = pool.apply(_table_chunk, ((cfg, ne, 0, 1),))
            ne_par = max(ne, n_cores)     # at least one energy (per wave / request) per process
            t0 = time.perf_counter()
            res = pool.map(_table_chunk, [(cfg, ne_par, k, n_cores) for k in range(n_cores)])
            tp = time.perf_counter() - t0
            npar = sum(r[0] for r in res)
            rows[str(cfg)] = {"sample_energy_solves": n1, "one_core_energy_solves_per_s": n1 / t1,
                              "all_cores_energy_solves_per_s": npar / tp, "parallel_sample": npar,
                              "config_energy_solves": total,
                              "one_core_s_for_config": total * t1 / n1,
                              "all_cores_s_for_config": total * tp / npar,
                              "extrapolated": total != n1}
    line = {"impl": "reference", "cpu_table": rows, "cores": n_cores, "cpu_model": _cpu_model(),
            "note": ("oracle (plain FP64, numpy/LAPACK with one BLAS thread per process, Coulomb functions in "
                     "binary128 C); configuration 4 = the 200-request serving stream")}
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.cpu_table:
        run_cpu_table(args)
        return
    _one_blas_thread()
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


def _time_steps(ctx, Ed, stream, flush, steps, rmgb, torch):
    """Times `steps` full steps (reset + solve of every energy) with CUDA events
    on the library's stream, flushing L2 before each; returns (ms per step,
    per-phase (launches, ms), kernel launches)."""
    ctx.profile_enable(True)
    l0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
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
    return sum(step_ms) / len(step_ms), phase, launches


def _solve_flops(n, n_open, f32):
    """Algorithmic flops of steps (c)+(d) for the energies given, as the
    shared-memory solver takes them, split (FP64, FP32): elimination of the
    n x (n + n_o) system (2/3 n^3 + n^2 n_o) and back-substitution of the n_o
    trailing rows (n_o^3); then FP64: M = 1 + K^2 (upper triangle, n_o^3),
    M^{-1} by the symmetric sweep (n_o^3), X = K M^{-1} for the upper triangle
    (n_o^3); or, when f32, everything in FP32 with the T step as the complex
    symmetric sweep of 1 - iK (upper triangle, n_o^3 / 2 complex FMAs =
    4 n_o^3 flops)."""
    no = n_open.astype(np.float64)
    elim = float(np.sum(2.0 / 3.0 * n**3 + n * n * no + no**3))
    if f32:
        return 0.0, elim + float(np.sum(4.0 * no**3))
    return elim + float(np.sum(3.0 * no**3)), 0.0


# FP64 operations (FMA, multiply, add, compare: one each; the reciprocal of
# the continued fractions: 4; an IEEE division or square root counted as 8)
# per iteration of the channel-function recurrences (Wallis forms, with the
# rescaling and convergence test of every 8th step spread over 8 steps),
# counted from the kernel.
CHANFN_OPS = {"cf1": 17, "cf2_fwd": 28, "cf2_bwd": 15, "open_l": 90, "open_fixed": 130,
              "closed_fwd": 14, "closed_bwd": 10, "ladder": 36, "closed_fixed": 70,
              "thr_interp": 16 * 10 + 40, "open_table": 4 * 2 * 11 + 60, "closed_table": 2 * 2 * 11 + 50}
CF2_FAST_DEPTH = 32   # CF2 settling within this many forward steps has no backward pass


def _chanfn_ops(work):
    """FP64 operations of step (b) from the per-(energy, channel) iteration
    counts {kind, CF1 iterations n1, CF2 forward iterations n2, l steps}."""
    w = work.reshape(-1, 4).astype(np.float64)
    op, cl = w[:, 0] == 0, w[:, 0] == 1
    c = CHANFN_OPS
    o = w[op]
    slow_o = o[:, 2] > CF2_FAST_DEPTH
    ops_open = (c["cf1"] * o[:, 1] + c["cf2_fwd"] * (o[:, 2] - 1)
                + c["cf2_bwd"] * (2 * o[:, 2] + 20) * slow_o + c["open_l"] * o[:, 3] + c["open_fixed"])
    k = w[cl]
    slow_c = k[:, 2] > CF2_FAST_DEPTH
    ops_closed = (c["closed_fwd"] * (k[:, 2] - 1) + c["closed_bwd"] * (2 * k[:, 2] + 19) * slow_c
                  + c["ladder"] * k[:, 3] + c["closed_fixed"])
    # near-threshold pairs: barycentric interpolation over the 16 nodes of the
    # channel's table (a reciprocal and 5 FMAs per node) and A(eps, l)
    ti = w[w[:, 0] == 3]
    ops_thr = c["thr_interp"] * ti.shape[0] + 2.0 * ti[:, 3].sum()
    # open pairs from the channel's Chebyshev table: Clenshaw for four
    # 12-term series, the segment and A(eps, l)
    to = w[w[:, 0] == 4]
    ops_tab = c["open_table"] * to.shape[0] + 2.0 * to[:, 3].sum()
    # closed pairs from the channel's direction table: Clenshaw for two
    # 12-term series and the normalisation
    tc = w[w[:, 0] == 5]
    ops_ctab = c["closed_table"] * tc.shape[0]
    return float(ops_open.sum() + ops_closed.sum() + ops_thr + ops_tab + ops_ctab)


def run_serving(args, prec):
    """The serving workload: a stream of partial-wave x energy-batch requests
    (50-1500 channels, 25-35 poles per channel, 256-8192 energies on 0-8 Ry,
    half MQDT; a pool of 64 pole sets) through the continuous-batching server
    with the mixed-precision path (bf16x3 formation, FP32 matching) and with
    the plain FP64 path. Mixed: first every request at once (capacity), the
    same requests back to back on one lane, then Poisson arrivals at 0.9 x the
    capacity (p50 / p99 latency). FP64: the same
    requests with every args.serving_fp64_stride-th energy (throughput in
    energy-solves/s; the FP64 path is ~10^2 slower), and the Omega error of
    the mixed results on those energies."""
    from paper_1909_07321_gb300 import serving, synth
    nreq = args.serving_requests
    specs = synth.serving_requests(nreq, 1.0, n_range=(50, 1500), ne_range=(256, 8192), n_sets=64)
    pws = {}

    def make(specs_, stride=1, t_scale=0.0):
        out = []
        for sp in specs_:
            if sp["set_id"] not in pws:
                pws[sp["set_id"]] = synth.serving_pole_set(sp["set_id"], sp["n"])
            out.append(serving.Request(sp["id"], sp["set_id"], pws[sp["set_id"]], sp["E"][::stride], sp["mode"],
                                       sp["t_arrival"] * t_scale))
        return out

    def keep_rows(stride):
        # host memory holds only the rows the FP64 comparison reads
        def sink(req, om):
            req.omega = om[::stride].copy() if stride else None
        return sink

    def serve(precision, sp_, reqs, keep, n_slots=4):
        srv = serving.Server(n_slots=n_slots, precision=precision, solve_precision=sp_, mem_budget=120 << 30,
                             lane_workspace=16 << 30, cache_sets=64, sink=keep_rows(keep))
        try:
            srv.prepare(reqs)
            warm = [serving.Request(-1 - i, r.set_id, r.pw, r.E[:64], r.mode, 0.0) for i, r in enumerate(reqs[:4])]
            srv.run(warm)
            srv.run(reqs)
            loads = srv.loads
        finally:
            srv.close()
        return serving.latency_stats(reqs), loads

    # capacity: every request queued at t = 0
    k = args.serving_fp64_stride
    sat = make(specs)
    st_sat, loads = serve(2, 1, sat, k)
    cap = st_sat["requests"] / st_sat["wall_s"]
    # the same requests back to back: one lane of one context
    st_one, _ = serve(2, 1, make(specs), 0, n_slots=1)
    # Poisson arrivals at 0.9 x capacity (the stream's exponential gaps rescaled)
    rate = 0.9 * cap
    pois = make(specs, t_scale=1.0 / rate)
    st_p, _ = serve(2, 1, pois, 0)
    # FP64 served arm on a strided subsample of every request's energies
    sub = make(specs, stride=k)
    st64, _ = serve(0, 0, sub, 1)
    rel = []
    for a, b in zip(sat, sub):
        om_m = a.omega
        nb = np.linalg.norm(b.omega, axis=1)
        ok = nb > 0
        rel.extend((np.linalg.norm(om_m[ok] - b.omega[ok], axis=1) / nb[ok]).tolist())
    rel = np.array(rel)
    ns = [sp["n"] for sp in specs]
    nes = [sp["E"].size for sp in specs]
    return {"workload": ("%d requests: 50-1500 channels (drawn n %d-%d, mean %.0f), 25-35 poles per channel "
                         "(pool of 64 pole sets), 256-8192 energies on 0-8 Ry (mean %.0f), half MQDT; "
                         "4 lanes of one context" % (nreq, min(ns), max(ns), np.mean(ns), np.mean(nes))),
            "mixed_saturated": {"energy_solves_per_s": st_sat["energy_solves_per_s"],
                                "requests_per_s": cap, "wall_s": st_sat["wall_s"],
                                "energy_solves": st_sat["energy_solves"], "pole_set_loads": loads},
            "mixed_one_lane": {"energy_solves_per_s": st_one["energy_solves_per_s"], "wall_s": st_one["wall_s"],
                               "saturated_over_one_lane": st_sat["energy_solves_per_s"] / st_one["energy_solves_per_s"]},
            "mixed_poisson_0.9": {"rate_per_s": rate, "energy_solves_per_s": st_p["energy_solves_per_s"],
                                  "p50_ms": 1e3 * st_p["p50_s"], "p99_ms": 1e3 * st_p["p99_s"],
                                  "mean_ms": 1e3 * st_p["mean_s"]},
            "fp64_saturated": {"energy_solves_per_s": st64["energy_solves_per_s"], "energy_stride": k,
                               "energy_solves": st64["energy_solves"], "wall_s": st64["wall_s"]},
            "mixed_over_fp64": st_sat["energy_solves_per_s"] / st64["energy_solves_per_s"],
            "omega_rel_err_vs_fp64": {"median": float(np.median(rel)), "p99": float(np.quantile(rel, 0.99)),
                                      "max": float(rel.max()), "energies": int(rel.size)},
            "formation": "bf16x3", "matching": "fp32"}


def run_batched(args):
    """The batched workload: 40 partial waves of 20-400 channels (30 poles per
    channel, z = 3) on 10000 energies over 0-5 Ry, mixed precision (bf16x3
    formation chosen per wave by the autotuner, FP32 matching), solved by
    rm_solve_batch over 4 lanes and replayed as one captured CUDA graph, against
    the same waves one rm_solve_energies call after another on one lane; and
    the FP64 batch on every 200th energy for the Omega error."""
    import torch

    from paper_1909_07321_gb300 import rmgb, synth
    pws, E = synth.workload_batched()
    ns = np.array([pw["W"].shape[0] for pw in pws])
    Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
    ids = list(range(len(pws)))
    out = {"workload": ("%d partial waves, %d-%d channels (sum %d), 30 poles per channel, z = 3, "
                        "%d energies on 0-5 Ry, 100 levels" % (len(pws), ns.min(), ns.max(), ns.sum(), E.size))}
    ctx = rmgb.Context(precision=2, solve_precision=1, lanes=4, autotune=1, mem_budget=8 << 30, stream=0)
    try:
        t0 = time.perf_counter()
        for i, pw in enumerate(pws):
            ctx.load_pw(i, pw)
        load_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        ctx.solve_batch(ids, Ed, 0, True)          # tunes, runs eagerly, captures
        ctx.sync()
        first_s = time.perf_counter() - t0
        st = torch.cuda.Stream()
        reps = 2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ctx.reset_omega()
        torch.cuda.synchronize()
        lane0 = torch.cuda.ExternalStream(ctx.lane_stream(0))
        ev[0].record(lane0)
        for _ in range(reps):
            ctx.solve_batch(ids, Ed, 0, True)      # graph replays
        ev[1].record(lane0)
        torch.cuda.synchronize()
        t_batch = ev[0].elapsed_time(ev[1]) / reps / 1e3
        om_batch = ctx.collision_strengths() / reps
        info = [ctx.autotune_info(i) for i in ids]
        del st
    finally:
        ctx.close()
    choice = {}
    for f, tn, stg, _ in info:
        k = "pairs %dx%d/%d stages" % (128, tn, stg) if f == 1 else "per-energy"
        choice[k] = choice.get(k, 0) + 1
    # the same waves one call after another on one lane (same tuned choices)
    ctx = rmgb.Context(precision=2, solve_precision=1, autotune=1, mem_budget=8 << 30, stream=0)
    try:
        for i, pw in enumerate(pws):
            ctx.load_pw(i, pw)
        for i in ids:
            ctx.solve_energies(i, Ed[:2048])    # the batch's tuner bucket: the same choices
        ctx.collision_strengths(reset=True)
        lane0 = torch.cuda.ExternalStream(ctx.lane_stream(0))
        torch.cuda.synchronize()
        ev[0].record(lane0)
        for i in ids:
            ctx.solve_energies(i, Ed)
        ev[1].record(lane0)
        torch.cuda.synchronize()
        t_seq = ev[0].elapsed_time(ev[1]) / 1e3
        om_seq = ctx.collision_strengths()
    finally:
        ctx.close()
    # FP64 batch on every 200th energy
    sub = np.arange(0, E.size, 200)
    ctx = rmgb.Context(precision=0, lanes=4, mem_budget=8 << 30, stream=0)
    try:
        for i, pw in enumerate(pws):
            ctx.load_pw(i, pw)
        Es = torch.tensor(E[sub], dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_batch(ids, Es, 0, False)
        om64 = ctx.collision_strengths()
        t64 = time.perf_counter() - t0
    finally:
        ctx.close()
    nrm = np.linalg.norm(om64, axis=1)
    ok = nrm > 0
    rel = np.linalg.norm(om_batch[sub][ok] - om64[ok], axis=1) / nrm[ok]
    n_es = len(pws) * E.size
    out.update({"batched_graph": {"energy_solves_per_s": n_es / t_batch, "s": t_batch,
                                  "timing": "CUDA events on lane 0 around %d graph replays" % reps},
                "one_call_per_wave": {"energy_solves_per_s": n_es / t_seq, "s": t_seq},
                "speedup": t_seq / t_batch,
                "omega_batch_vs_sequential_rel": _dist(np.linalg.norm(om_batch - om_seq, axis=1) /
                                                       np.maximum(np.linalg.norm(om_seq, axis=1), 1e-300)),
                "first_call_s": first_s, "load_s": load_s,
                "autotune_choices": choice,
                "fp64_batch": {"energy_solves_per_s": len(pws) * sub.size / t64, "energies": int(sub.size)},
                "omega_rel_err_vs_fp64": _dist(rel),
                "worst_energy_vs_fp64": {"E_ry": float(E[sub][ok][int(np.argmax(rel))]),
                                         "omega_norm_over_median": float(nrm[ok][int(np.argmax(rel))] /
                                                                         np.median(nrm[ok]))}})
    return out


def _dist(x):
    x = np.asarray(x)
    return {"median": float(np.median(x)), "p99": float(np.quantile(x, 0.99)), "max": float(x.max())}


def _pe_tiles(n):
    """Tiles of 128 rows x 256 columns holding some (i <= j) of an n x n matrix."""
    n_ib, n_jb = -(-n // 128), -(-n // 256)
    return sum(min(n_ib, 2 * jb + 2) for jb in range(n_jb))


def run_wide(args, prec, sp, stream, flush, peaks, peak_src):
    """The 1000-channel, 30000-pole workload (the per-energy tensor-core
    formation): a strided sample of its energy grid through the mixed path,
    and every 16th of those through the plain FP64 path, with the Omega error
    of the mixed path on the common energies."""
    import torch

    from paper_1909_07321_gb300 import rmgb, synth
    pws, Eall = synth.workload_1000ch()
    pw = pws[0]
    n, N = pw["W"].shape
    idx = np.linspace(0, Eall.size - 1, args.wide_energies).round().astype(int)
    E = np.ascontiguousarray(Eall[idx])
    sub = np.arange(0, E.size, 16)
    out = {"workload": ("one partial wave: 1000 channels (250 levels x 4 on 0-8 Ry, l 0-8, z=2), "
                        "30000 poles on [-5,200] Ry, w~N(0,0.02^2), a=20; %d of its 5000 energies on "
                        "0-10 Ry (evenly strided)" % E.size)}
    res = {}
    for name, pr, Es, spn in [("mixed", prec, E, sp), ("fp64", 0, E[sub], 0)]:
        ctx = rmgb.Context(precision=pr, stream=stream.cuda_stream, solve_precision=spn)
        ctx.load_pw(0, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            ctx.solve_energies(0, Ed)
            ctx.reset_omega()
            t, ph, launches = _time_steps(ctx, Ed, stream, flush, 2, rmgb, torch)
            om = ctx.collision_strengths()
        ctx.close()
        res[name] = (t, ph, om, Es.size)
    t, ph, om, ne = res["mixed"]
    names = {rmgb.RM_PH_CHANFN: "chanfn", rmgb.RM_PH_FORM: "form", rmgb.RM_PH_FIXUP: "reduce+nearpole",
             rmgb.RM_PH_SOLVE: "solve", rmgb.RM_PH_SPLIT: "d(E)"}
    form_ms = ph[rmgb.RM_PH_FORM][1] / 2
    alg = n * (n + 1) * N * ne / (form_ms * 1e-3) / 1e12
    tpk = peaks["bf16_tflops"] if prec == 2 else peaks["bf16_tflops"] / 2.0
    t64, _, om64, ne64 = res["fp64"]
    rel = np.linalg.norm(om[sub] - om64, axis=1) / np.maximum(np.linalg.norm(om64, axis=1), 1e-300)
    out.update({
        "mixed": {"energy_solves_per_s": ne / (t * 1e-3), "ms_per_step": t, "energies": ne,
                  "phases_ms_per_step": {v: ph[k][1] / 2 for k, v in names.items()}},
        "fp64_path": {"energy_solves_per_s": ne64 / (t64 * 1e-3), "ms_per_step": t64, "energies": ne64},
        "omega_rel_err_vs_fp64": {"median": float(np.median(rel)), "max": float(rel.max())},
        "formation_roofline": {
            "bound": "tensor", "achieved": alg, "peak": tpk, "unit": "TFLOP/s", "frac": alg / tpk,
            "issued_frac": 3.0 * alg / tpk,
            "executed_frac": 3.0 * alg * _pe_tiles(n) * 128 * 256 / (n * (n + 1) / 2) / tpk,
            "traffic": None, "kernel": "form_r_pe_kernel (%s, one GEMM per energy)" % args.precision,
            "note": ("algorithmic n(n+1)N flops per energy; issued x3 (hi/lo products); executed "
                     "counts the tiles of 128 x 256 that cover the upper triangle"),
            "peak_source": ("bf16 dense burst, %s" % peak_src) if prec == 2 else
            ("tf32 = bf16 dense burst (%s) x nominal ratio 1/2" % peak_src)}})
    return out


def run_qdt(args, prec, sp):
    """MQDT coarse-mesh interpolation on the 64-channel workload: the full
    per-energy MQDT solve of every energy against K_u solved at the nodes and
    S_u interpolated to the fine energies, for node spacings ieq = -2 .. -25
    (every |ieq|-th fine energy a node); the speed-up is reported at the
    sparsest spacing whose per-energy Omega difference from the full solve
    stays within 1e-3 at the 99th percentile."""
    import torch

    from paper_1909_07321_gb300 import rmgb, synth
    pws, E = synth.workload_64ch(args.energies)
    pw = pws[0]

    def timed(fn, ctx, st):
        best = None
        for rep in range(3):
            if rep:
                ctx.reset_omega()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            ctx.sync()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best, ctx.collision_strengths(), st.cpu().numpy()

    ctx = rmgb.Context(precision=prec)
    ctx.load_pw(0, pw)
    st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
    tf, omf, stf = timed(lambda: ctx.solve_energies(0, E, 1, None, None, st), ctx, st)
    ctx.close()
    sweep = []
    for ieq in (-2, -3, -5, -8, -12, -25):
        ctx = rmgb.Context(precision=prec)
        ctx.load_pw(0, pw)
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ti, omi, sti = timed(lambda: ctx.solve_energies_qdt(0, E, ieq, 0.0, 1, None, st), ctx, st)
        ctx.close()
        ok = (stf == 0) & (sti == 0)
        rel = np.linalg.norm(omi[ok] - omf[ok], axis=1) / np.maximum(np.linalg.norm(omf[ok], axis=1), 1e-300)
        sweep.append({"ieq": ieq, "speedup": tf / ti, "s": ti, "p99": float(np.quantile(rel, 0.99)),
                      "median": float(np.median(rel)), "max": float(rel.max())})
    good = [r for r in sweep if r["p99"] <= 1e-3]
    at = min(good, key=lambda r: r["ieq"]) if good else None
    return {"workload": "64-channel workload in MQDT mode, %d energies; S_u interpolation (iqdt = 1)" % E.size,
            "full_mqdt": {"energy_solves_per_s": E.size / tf, "s": tf},
            "at_p99_1e-3": at,
            "sweep": sweep,
            "timing": "host wall clock around each call, best of 3 (the interpolated call synchronises once "
                      "after its node solves)"}


def run_propagation(args, prec, sp, fp64_peak, stream):
    """Outer-region propagation with the multipole potential (32 channels,
    lambda_max = 2, a = 15 -> r1 = 35 in 2000 Numerov steps): the whole solve of
    args.prop_energies energies with propagation, the same solve without it,
    and the propagation kernel against the FP64 pipe."""
    import torch

    from paper_1909_07321_gb300 import rmgb, synth
    pw, A, r1, steps, E = synth.workload_multipole(args.prop_energies)
    n = pw["W"].shape[0]
    lmax = A.shape[0]
    out = {"workload": "%d channels, lambda_max = %d, a = %g -> r1 = %g in %d Numerov steps, %d energies "
                       "(0.01-2.5 Ry), formation %s" % (n, lmax, pw["a"], r1, steps, E.size, args.precision)}
    Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
    res = {}
    for name in ("propagated", "unpropagated"):
        ctx = rmgb.Context(precision=prec, stream=stream.cuda_stream, solve_precision=sp)
        ctx.load_pw(0, pw)
        if name == "propagated":
            ctx.set_multipoles(0, A, r1, steps)
        with torch.cuda.stream(stream):
            ctx.solve_energies(0, Ed)
            ctx.reset_omega()
            ctx.profile_enable(True)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            reps = 2
            torch.cuda.synchronize()
            t0.record(stream)
            for _ in range(reps):
                ctx.solve_energies(0, Ed)
                ctx.reset_omega()
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / reps
            pl, pms = ctx.profile_get(rmgb.RM_PH_PROPAGATE)
        ctx.close()
        res[name] = (ms, pl, pms / reps)
    # truncation: Omega with twice the steps
    om2 = {}
    for k, st_ in (("1x", steps), ("2x", 2 * steps)):
        ctx = rmgb.Context(precision=prec, stream=stream.cuda_stream, solve_precision=sp)
        ctx.load_pw(0, pw)
        ctx.set_multipoles(0, A, r1, st_)
        with torch.cuda.stream(stream):
            ctx.solve_energies(0, Ed)
            om2[k] = ctx.collision_strengths()
        ctx.close()
    dn = np.abs(om2["1x"] - om2["2x"]).max(axis=1) / np.maximum(np.abs(om2["2x"]).max(axis=1), 1e-300)
    ms_p, pl, prop_ms = res["propagated"]
    ms_u = res["unpropagated"][0]
    # per energy and Numerov step: two products T X (2 n^3 flops each), the
    # summed-form updates (12 flops per element) and one build of T (lambda_max
    # FMA and a scaling per element); the Runge-Kutta start and the basis
    # renormalisations are not counted
    flops = E.size * steps * (4.0 * n ** 3 + (14.0 + 2.0 * lmax) * n * n)
    ach = flops / (prop_ms * 1e-3) / 1e12
    out.update({"propagated": {"energy_solves_per_s": E.size / (ms_p * 1e-3), "ms": ms_p},
                "unpropagated": {"energy_solves_per_s": E.size / (ms_u * 1e-3), "ms": ms_u},
                "propagate_ms": prop_ms, "propagate_launches_per_solve": pl / 2,
                "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": ach / fp64_peak, "traffic": None,
                             "kernel": "propagate_kernel (FP64 Numerov, one CTA per energy)",
                             "flops_per_launch": flops,
                             "peak_source": "FP64 4 flop/clk/SM x 152 SMs at the sampled SM clock"},
                "omega_rel_change_with_2x_steps": {"median": float(np.median(dn)), "max": float(dn.max())},
                "timing": "CUDA events on the context stream around 2 solves after one warm-up"})
    # 64 channels (the 512-thread kernel; lambda_max = 2) on the same energies
    pw6, A6, r16, steps6, _ = synth.workload_multipole(args.prop_energies, n=64)
    ctx = rmgb.Context(precision=prec, stream=stream.cuda_stream, solve_precision=sp)
    ctx.load_pw(0, pw6)
    ctx.set_multipoles(0, A6, r16, steps6)
    with torch.cuda.stream(stream):
        ctx.solve_energies(0, Ed)
        ctx.reset_omega()
        ctx.profile_enable(True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        ctx.solve_energies(0, Ed)
        t1.record(stream)
        torch.cuda.synchronize()
        ms6 = t0.elapsed_time(t1)
        _, pms6 = ctx.profile_get(rmgb.RM_PH_PROPAGATE)
    ctx.close()
    f6 = E.size * steps6 * (4.0 * 64 ** 3 + (14.0 + 2.0 * A6.shape[0]) * 64 * 64)
    a6 = f6 / (pms6 * 1e-3) / 1e12
    out["64ch"] = {"energy_solves_per_s": E.size / (ms6 * 1e-3), "ms": ms6, "propagate_ms": pms6,
                   "propagate_tflops": a6, "frac_of_fp64_peak": a6 / fp64_peak,
                   "kernel": "propagate_kernel<512,8,64> (FP64 Numerov, one CTA per energy)"}
    return out


def _leg(fn, *a):
    """Runs one auxiliary leg; a failure there is reported in its slot of the
    JSON line instead of taking the headline measurement down with it."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001
        return {"error": "%s: %s" % (type(e).__name__, e)}


def run_ours(args, rank, world, local_rank):
    import torch

    pool = None
    n_cores = os.cpu_count() or 1
    if rank == 0 and not args.no_cpu_baseline:
        _one_blas_thread()
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
    n_tri = pw["n_levels"] * (pw["n_levels"] + 1) // 2
    prec = PREC[args.precision]
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        return float(t.item())

    Ed = torch.tensor(E, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    sp = 1 if (prec != 0 and args.matching == "fp32") else 0
    ctx = rmgb.Context(precision=prec, stream=stream.cuda_stream, device=local_rank, solve_precision=sp)
    ctx.load_pw(0, pw)
    n_open = torch.zeros(E.size, dtype=torch.int32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            ctx.solve_energies(0, Ed, 0, None, n_open)
            ctx.reset_omega()
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        props = torch.cuda.get_device_properties(dev)
        clk = ClockSampler("GPU-%s" % props.uuid if getattr(props, "uuid", None) else local_rank)
        clk.start()
        clk.wait_first()
        tw0 = time.perf_counter()
        t_step, phase, launches = _time_steps(ctx, Ed, stream, flush, args.steps, rmgb, torch)
        clk.window(tw0, time.perf_counter())
        clocks = clk.stop()
        t_step = max_over_ranks(t_step)
        value = world * E.size / (t_step * 1e-3)
        om_main = ctx.collision_strengths()      # Omega of the last timed step
        work = torch.zeros((E.size, n, 4), dtype=torch.int32, device=dev)
        ctx.channel_work(0, Ed, work)
        torch.cuda.synchronize()
        chan_ops = _chanfn_ops(work.cpu().numpy())

        # end to end through the public API with host buffers: pinned
        # energies in, the full Omega out every step. Streamed: each step's
        # read-out drains (rm_collision_strengths_async, two host buffers in
        # turn) while the next step computes; the clock stops after the last
        # copy has landed. Also the blocking form (read-out, then the next
        # step).
        E_pin = torch.tensor(E, dtype=torch.float64).pin_memory()
        om_pin = [torch.empty((E.size, n_tri), dtype=torch.float64).pin_memory() for _ in range(2)]
        ctx.collision_strengths(reset=True)
        k2 = max(2, args.steps)
        e2e = {}
        for form in ("blocking", "streamed"):
            # one untimed step of the same form first (the streamed form's
            # second Omega buffer is allocated by its first read-out)
            ctx.solve_energies(0, E_pin.numpy())
            if form == "streamed":
                ctx.collision_strengths_async(om_pin[1].numpy(), reset=True)
            else:
                ctx.collision_strengths(om_pin[1].numpy(), reset=True)
            ctx.sync()
            torch.cuda.synchronize()
            if dist:
                tdist.barrier()
            t0 = time.perf_counter()
            for i in range(k2):
                ctx.solve_energies(0, E_pin.numpy())
                if form == "streamed":
                    ctx.collision_strengths_async(om_pin[i % 2].numpy(), reset=True)
                else:
                    ctx.collision_strengths(om_pin[i % 2].numpy(), reset=True)
            ctx.sync()
            e2e[form] = max_over_ranks((time.perf_counter() - t0) / k2)
        om_e2e = om_pin[(k2 - 1) % 2].numpy().copy()
        e2e_ok = bool(np.array_equal(om_e2e, om_main))
        e2e_s = e2e["streamed"]
    ctx.close()

    # the plain FP64 GPU path on the same workload (the metric's comparison)
    fp64 = None
    if prec != 0 and not args.no_fp64_compare:
        ctx64 = rmgb.Context(precision=0, stream=stream.cuda_stream, device=local_rank)
        ctx64.load_pw(0, pw)
        with torch.cuda.stream(stream):
            ctx64.solve_energies(0, Ed)
            ctx64.reset_omega()
            t64, ph64, _ = _time_steps(ctx64, Ed, stream, flush, max(2, args.steps // 3), rmgb, torch)
            om64 = ctx64.collision_strengths()
        ctx64.close()
        t64 = max_over_ranks(t64)
        rel = np.linalg.norm(om_main - om64, axis=1) / np.maximum(np.linalg.norm(om64, axis=1), 1e-300)
        fp64 = {"value": world * E.size / (t64 * 1e-3), "ms_per_step": t64,
                "mixed_over_fp64": (world * E.size / (t_step * 1e-3)) / (world * E.size / (t64 * 1e-3)),
                "omega_rel_err_vs_fp64": {"median": float(np.median(rel)),
                                          "p99": float(np.quantile(rel, 0.99)),
                                          "max": float(rel.max())}}

    serving_line = None
    if rank == 0 and world == 1 and args.serving_requests > 0:
        serving_line = _leg(run_serving, args, 2)

    if rank != 0:
        return
    peaks, peak_src = _peaks()
    wide = None
    if world == 1 and args.wide_energies > 0:
        wide = _leg(run_wide, args, prec if prec != 0 else 2, sp, stream, flush, peaks, peak_src)
    batched_line = None
    if world == 1 and args.batched:
        batched_line = _leg(run_batched, args)
    qdt_line = None
    if world == 1 and args.qdt_ieq != 0:
        qdt_line = _leg(run_qdt, args, prec, sp)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = N_SM * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
    prop_line = None
    if world == 1 and args.prop_energies > 0:
        prop_line = _leg(run_propagation, args, prec, sp, fp64_peak, stream)
    names = {rmgb.RM_PH_NEARPOLE: "nearpole", rmgb.RM_PH_CHANFN: "chanfn", rmgb.RM_PH_FORM: "form",
             rmgb.RM_PH_FIXUP: "fixup", rmgb.RM_PH_SOLVE: "solve", rmgb.RM_PH_SPLIT: "split"}
    total_phase_ms = sum(v[1] for v in phase.values())
    share = {names[p]: (phase[p][1] / total_phase_ms if total_phase_ms else None) for p in names}

    def per_launch_ms(p):
        return phase[p][1] / max(phase[p][0], 1)

    # formation kernel: algorithmic n(n+1)/2 MACs per pole per energy
    form_flops = n * (n + 1) * N * (E.size / max(1, phase[rmgb.RM_PH_FORM][0] / args.steps))
    form_ach = form_flops / (per_launch_ms(rmgb.RM_PH_FORM) * 1e-3) / 1e12
    if prec == 0:
        form_roof = {"bound": "alu", "achieved": form_ach, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": form_ach / fp64_peak, "traffic": None, "kernel": "form_r_tiled (FP64)",
                     "peak_source": "FP64 4 flop/clk/SM x 152 SMs at the sampled SM clock"}
    else:
        tpk = peaks["bf16_tflops"] if prec == 2 else peaks["bf16_tflops"] / 2.0
        issued = 3.0 * form_ach
        form_roof = {"bound": "tensor", "achieved": form_ach, "peak": tpk, "unit": "TFLOP/s",
                     "frac": form_ach / tpk, "issued_frac": issued / tpk, "traffic": None,
                     "kernel": "form_r_tc_kernel (%s)" % args.precision,
                     "peak_source": ("bf16 dense burst, %s" % peak_src) if prec == 2 else
                     ("tf32 = bf16 dense burst (%s) x nominal ratio 1/2" % peak_src)}
    # channel functions: FP64 operations counted from the recurrence depths
    fp64_op_peak = N_SM * FP64_FLOPS_PER_CLK_SM / 2.0 * sm_mhz * 1e6 / 1e12
    chan_ach = chan_ops / (phase[rmgb.RM_PH_CHANFN][1] / args.steps * 1e-3) / 1e12
    chan_roof = {"bound": "alu", "achieved": chan_ach, "peak": fp64_op_peak, "unit": "TFP64op/s",
                 "frac": chan_ach / fp64_op_peak, "traffic": None,
                 "kernel": "chanfn_kernel (channel tables + FP64 continued fractions)",
                 "ops_per_step": chan_ops,
                 "peak_source": "FP64 pipe 2 op/clk/SM x 152 SMs at the sampled SM clock"}
    # matching + T + Omega
    f32 = sp == 1
    fl64, fl32 = _solve_flops(n, n_open.cpu().numpy(), f32)
    t_solve = phase[rmgb.RM_PH_SOLVE][1] / args.steps * 1e-3
    if f32:
        fp32_peak = N_SM * 256.0 * sm_mhz * 1e6 / 1e12
        ach = fl32 / t_solve / 1e12
        # DRAM bytes per launch from one ncu capture of this kernel on 2000
        # energies of the same workload (58.20 MB read, 6 KB written: Omega
        # stays in L2 at that size), scaled to the launch's energies
        traffic = (58.20e6 + 0.006e6) * (E.size / 2000.0) if n == 64 else None
        solve_roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                      "frac": ach / fp32_peak, "traffic": traffic,
                      "kernel": "solve_f32_kernel (FP32 Gauss-Jordan, FP32 complex T sweep, register tiles)",
                      "peak_source": "FP32 128 FMA/clk/SM x 152 SMs at the sampled SM clock",
                      "note": "one CTA per energy, four per SM; pivots in blocks factored by one warp "
                              "(n/4 + n_o/2 barrier pairs); ncu: barrier stalls (the block's serial pivot "
                              "chain) dominate, FMA pipe 22% busy, issue 52% (bound by the pivot chain's "
                              "latency and the energies resident per SM, not by a pipe)"}
    else:
        ach = fl64 / t_solve / 1e12
        solve_roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                      "frac": ach / fp64_peak, "traffic": None,
                      "kernel": "solve_small_kernel (FP64 elimination, FP64 T step)",
                      "peak_source": "FP64 4 flop/clk/SM x 152 SMs at the sampled SM clock"}
    # dominant kernel by device time
    dom = max((rmgb.RM_PH_FORM, rmgb.RM_PH_SOLVE, rmgb.RM_PH_CHANFN), key=lambda p: phase[p][1])
    roof = {rmgb.RM_PH_FORM: form_roof, rmgb.RM_PH_SOLVE: solve_roof, rmgb.RM_PH_CHANFN: chan_roof}[dom]
    cpu = None
    if pool is not None:
        v, sample = oracle_throughput(pool, n_cores, 24)
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": n_cores, "kind": "oracle", "sample": sample}
    dtype = ("bf16x3+fp32/fp64" if prec == 2 else "tf32x3+fp32/fp64") if prec != 0 else "f64"
    if prec != 0 and sp == 0:
        dtype = dtype.replace("+fp32/", "/")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_channels": n, "n_poles": N,
                       "energies_per_gpu": int(E.size), "formation": args.precision,
                       "matching": args.matching if prec != 0 else "fp64",
                       "near_pole_delta_ry": 1e-3, "mode": "direct",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "energy-interleaved dp%d" % world,
                       "arithmetic": ("formation bf16 hi/lo x3 products, FP32 accumulation, near-pole terms "
                                      "FP64; matching and T step FP32; channel functions and Omega FP64")},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * E.size / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(E.size * 8),
                    "d2h_bytes_per_step": int(E.size * n_tri * 8),
                    "form": "streamed read-out (rm_collision_strengths_async, two pinned host buffers)",
                    "blocking_value": world * E.size / e2e["blocking"],
                    "omega_equals_device_step": e2e_ok},
            "clocks": clocks, "gpu_launches": int(launches),
            "rooflines": {"chanfn": chan_roof, "solve": solve_roof, "formation": form_roof},
            "phases_ms_per_step": {names[p]: phase[p][1] / args.steps for p in names},
            "phase_share": share,
            "mqdt_interpolation": qdt_line,
            "multipole_propagation": prop_line,
            # the workloads of the other configurations, and the FP64 path the
            # metric compares against, last (the end of the line is what a
            # truncated log keeps)
            "wide_1000ch": wide,
            "batched_40pw": batched_line,
            "serving": serving_line,
            "fp64_path": fp64}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PREC))
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 path beside the chosen precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-table", action="store_true",
                    help="with --impl reference: time the oracle on samples of every configuration")
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests in the serving leg (0 to skip)")
    ap.add_argument("--serving-fp64-stride", type=int, default=128,
                    help="the FP64 served arm solves every k-th energy of each request")
    ap.add_argument("--matching", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the matching elimination on the mixed path")
    ap.add_argument("--qdt-ieq", type=int, default=-25,
                    help="node spacing of the MQDT interpolation leg (0 to skip)")
    ap.add_argument("--wide-energies", type=int, default=256,
                    help="energies of the 1000-channel leg (0 to skip)")
    ap.add_argument("--batched", type=int, default=1, help="run the batched 40-wave leg (0 to skip)")
    ap.add_argument("--prop-energies", type=int, default=1024,
                    help="energies of the multipole-propagation leg (0 to skip)")
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
