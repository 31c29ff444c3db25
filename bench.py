"""Benchmark of the TSBTS hot path on GB300: G pair-interactions/s.

Workload (one "step"): a Plummer sphere of n = 16384 equal-mass bodies in
standard N-body units, eps = 1/256, eta = 0.01, dt = 2^-k (k = 3..20),
dynamic era (Alg. 3), three passes per era, integrated over t = 0..1 from
its initial conditions, mixed precision (FP32 pair terms, FP64 state).
Interactions = sum over all block steps of all passes of n_act * n.

JSON line keys beyond the driver contract:
  peaks         the FP32 / FP64 / rsqrt pipe rates measured on this GPU by
                the library's probe (tsbts_pipe_peak), with the SM clock
  roofline      the force kernel against the FP32 FMA-pipe bound (20
                FMA-pipe ops per interaction), timed with CUDA events on a
                sample of the timed steps (every 8th chunk of steps)
  accuracy      relative energy errors at t = 1 of the mixed and the plain
                FP64 GPU paths and of the FP64 oracle (stored by the script
                in tests/golden), and how the schedules compare
  fp64          the plain FP64 GPU path over the same t = 0..1, timed the
                same way, and the mixed path's speed-up over it
  configs       compact results of the other configurations (Plummer 256
                FP64 latency; force sweep and one full era at n = 131072;
                the 512-cluster ensemble; the adjoint at n = 8192)
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the workload
Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
     [--quick] (skip fp64, configs and cpu_baseline)
Other modes: --force-sweep (force kernel alone), --ensemble (512 clusters),
--adjoint (gradient through a frozen block schedule, Plummer n = 8192),
--study (the paper's Sec. 3-4 era / iteration study, long spans).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BODIES = 16384
EPS = 1.0 / 256.0
ETA = 0.01
DT_MAX = 1.0 / 8.0
T_END = 1.0
N_ITER = 3
SEED = 0
SAMPLE_T = 2.0 ** -6        # oracle sample interval (~16 s of oracle work)
TIMING_PERIOD = 8           # force launches timed: every 8th chunk of steps
OPS_PER_INTERACTION = 20    # FMA-pipe ops of the algorithmic pair term
SM_COUNT = 152              # GB300; replaced by the device's own count
FP32_LANES_PER_SM = 128
NOMINAL_SM_MHZ = 2070.0
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_plummer16384_t1.json")
# DRAM bytes (read + write) per force launch from one ncu capture of this
# workload's first 2^-7 time units (cold cache, 1153 launches averaged);
# the algorithmic bytes of a launch are the j records, n x 48 B
FORCE_TRAFFIC_BYTES = 861313
FORCE_ALGORITHMIC_BYTES = N_BODIES * 48
METRIC = ("G pair-interactions/s, mixed vs FP64 on same GB300 at "
          "|dE/E|<=2x oracle; steps/s")
WORKLOAD = "plummer16384_eps1-256_eta0.01_dynamic_era_3iter_t0-1"


def config_dict(extra=None):
    c = {"workload": WORKLOAD, "n": N_BODIES, "eps": EPS, "eta": ETA,
         "dt_max": DT_MAX, "k_range": [3, 20], "era": "dynamic",
         "n_iter": N_ITER, "t_end": T_END, "seed": SEED,
         "ic": "Plummer (Aarseth-Henon-Wielen), standard units",
         "l2": "256 MiB buffer written between timed steps"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None,
                    "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, its maximum and the throttle reasons seen in
    nvidia-smi CSV lines (noheader, nounits) of ClockSampler.FIELDS."""
    sm, smax, reasons = [], [], set()
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
             "sw_power_cap")
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm.append(float(parts[0]))
            smax.append(float(parts[1]))
        except ValueError:
            continue
        for name, val in zip(names, parts[4:8]):
            if val.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
            "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist:
        dist.barrier()


def reduce_max(dist, x):
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(dist, x):
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(m, r, v, t_end, threads):
    """The FP64 oracle on [0, t_end]: (interactions, seconds, dE/E)."""
    import oracle
    oracle.set_threads(threads)
    s = oracle.Sim(m, r, v, eps=EPS, eta=ETA, dt_max=DT_MAX, n_iter=N_ITER,
                   era_mode=1, era_log2=3, k_max=20)
    e0 = sum(s.energy())
    t0 = time.perf_counter()
    s.run(t_end)
    sec = time.perf_counter() - t0
    de = abs(sum(s.energy()) / e0 - 1.0)
    st = s.stats()
    s.close()
    return st["interactions"], sec, de, st["block_steps"]


def measure_peaks(local):
    """Pipe rates of this GPU (tsbts_pipe_peak), each probe ~0.3 s, with the
    SM clock sampled meanwhile: FP32 FMA lane-ops/s (the larger of scalar
    and packed f32x2), FP64 FMA lane-ops/s, FP32 rsqrt/s."""
    import torch

    from paper_1205_2288_gb300 import tsbts

    sampler = ClockSampler(local)
    sampler.start()
    out = {}
    for kind, name, iters in ((0, "fp32_fma", 1 << 22), (1, "fp32x2_fma", 1 << 21),
                              (2, "fp64_fma", 1 << 16), (3, "rsqrt", 1 << 20)):
        ops, ms = tsbts.tsbts_pipe_peak(kind, iters)
        out[name] = {"lane_ops_per_s": ops, "ms": ms}
    clocks = sampler.stop()
    props = torch.cuda.get_device_properties(local)
    fp32 = max(out["fp32_fma"]["lane_ops_per_s"],
               out["fp32x2_fma"]["lane_ops_per_s"])
    return {"probe": out, "sm_count": props.multi_processor_count,
            "clocks": clocks, "fp32_lane_ops_per_s": fp32,
            "fp64_lane_ops_per_s": out["fp64_fma"]["lane_ops_per_s"],
            "fp32_peak_Ginteractions_s": fp32 / OPS_PER_INTERACTION / 1e9,
            "fp64_peak_Ginteractions_s":
                out["fp64_fma"]["lane_ops_per_s"] / OPS_PER_INTERACTION / 1e9,
            "nominal_fp32_peak_Ginteractions_s":
                props.multi_processor_count * FP32_LANES_PER_SM
                * NOMINAL_SM_MHZ * 1e6 / OPS_PER_INTERACTION / 1e9}


def timed_integration(m, r, v, t_end, stream, **kw):
    """One integration from t = 0 on the given stream, timed with CUDA
    events: (seconds, stats, dE/E at t_end)."""
    import torch

    from paper_1205_2288_gb300 import tsbts

    sim = tsbts.Simulation(m, r, v, stream=stream.cuda_stream, **kw)
    e0 = sum(sim.energy())
    e_a = torch.cuda.Event(enable_timing=True)
    e_b = torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    sim.step_era(t_end)
    e_b.record(stream)
    e_b.synchronize()
    sec = e_a.elapsed_time(e_b) / 1e3
    st = sim.stats()
    de = abs(sum(sim.energy()) / e0 - 1.0)
    sim.close()
    return sec, st, de


def config_results(local, stream, peak_g):
    """Compact results of the other configurations, each one run."""
    import numpy as np
    import torch

    from paper_1205_2288_gb300 import inputs, tsbts

    out = {}
    # config 1: Plummer 256, FP64, fixed era 1/8, t = 0..1 (latency-bound)
    m, r, v = inputs.plummer(256, SEED)
    kw = dict(eps=0.01, eta=0.01, dt_max=1 / 8, n_iter=3, era_mode=0,
              era_log2=3, k_max=20, precision=tsbts.TSBTS_FP64)
    timed_integration(m, r, v, 0.125, stream, **kw)
    sec, st, de = timed_integration(m, r, v, 1.0, stream, **kw)
    out["plummer256_fp64_fixed_era_t0-1"] = {
        "us_per_block_step": 1e6 * sec / st["block_steps"],
        "block_steps_per_s": st["block_steps"] / sec,
        "Ginteractions_s": st["interactions"] / sec / 1e9,
        "block_steps": st["block_steps"], "dE_E": de,
        "note": "FP64 ascending-j sums, bit-identical to the oracle "
                "(tests/test_gpu_integrator.py)"}
    # config 3: force sweep and one full era at n = 131072, eps = 1/512
    n, eps = 131072, 1.0 / 512.0
    m, r, v = inputs.plummer(n, SEED)
    dm, dr, dv = (torch.from_numpy(x).to(f"cuda:{local}") for x in (m, r, v))
    sweep = {}
    with torch.cuda.stream(stream):
        for na in (1, 32, 1024, 32768, n):
            idx = torch.from_numpy(inputs.active_subset(n, na, 1000 + na)).to(
                f"cuda:{local}")
            a = torch.empty(na, 3, dtype=torch.float64, device=dm.device)
            phi = torch.empty(na, dtype=torch.float64, device=dm.device)
            q = torch.empty(na, dtype=torch.float64, device=dm.device)
            call = lambda: tsbts.tsbts_force(  # noqa: E731
                tsbts.TSBTS_MIXED, dm, dr, dv, eps, idx, a, phi, q,
                stream=stream.cuda_stream)
            call()
            reps = 20 if na >= 32768 else 200
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            for _ in range(reps):
                call()
            e_b.record(stream)
            e_b.synchronize()
            ms = e_a.elapsed_time(e_b) / reps
            g = na * n / (ms / 1e3) / 1e9
            sweep[str(na)] = {"us_per_call": 1e3 * ms, "Ginteractions_s": g,
                              "frac_of_fp32_peak": g / peak_g}
    out["plummer131072_force_sweep"] = {
        "results": sweep,
        "note": "tsbts_force per call (packing, force, partial-sum "
                "finalize); small sets are latency-bound: one call streams "
                "n x 48 B of j records (6.3 MB)"}
    kw = dict(eps=eps, eta=ETA, dt_max=DT_MAX, n_iter=N_ITER, era_mode=1,
              precision=tsbts.TSBTS_MIXED)
    sec, st, de = timed_integration(m, r, v, 0.125, stream, **kw)
    out["plummer131072_mixed_era_t0-0.125"] = {
        "Ginteractions_s": st["interactions"] / sec / 1e9,
        "block_steps_per_s": st["block_steps"] / sec, "seconds": sec,
        "block_steps": st["block_steps"], "dE_E_mixed": de}
    short = 2.0 ** -9
    _, _, de_m = timed_integration(m, r, v, short, stream, **kw)
    _, _, de_f = timed_integration(m, r, v, short, stream,
                                   **dict(kw, precision=tsbts.TSBTS_FP64))
    out["plummer131072_mixed_era_t0-0.125"].update(
        {"t_compare": short, "dE_E_mixed_t_compare": de_m,
         "dE_E_fp64_gpu_t_compare": de_f})
    # config 4: 512-cluster ensemble, one integration over t = 0..1/2
    off, m, r, v, eps = inputs.ensemble(512, seed=SEED)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, eta=ETA, dt_max=DT_MAX,
                       precision=tsbts.TSBTS_MIXED, n_iter=N_ITER, era_log2=3,
                       stream=stream.cuda_stream)
    e_a = torch.cuda.Event(enable_timing=True)
    e_b = torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    g.step_era(0.5)
    e_b.record(stream)
    e_b.synchronize()
    sec = e_a.elapsed_time(e_b) / 1e3
    st = g.stats()
    g.close()
    out["ensemble512_salpeter_t0-0.5"] = {
        "Ginteractions_s": st["interactions"] / sec / 1e9,
        "global_block_steps_per_s": st["block_steps"] / sec,
        "kernel_launches_per_global_step":
            st["kernel_launches"] / max(st["block_steps"], 1),
        "bodies": int(off[-1]), "seconds": sec}
    # config 5: adjoint of one era's final pass, n = 8192, one gradient
    n, eps, t_era = 8192, 0.01, 0.25
    m, r, v = inputs.plummer(n, SEED)
    sim = tsbts.Simulation(m, r, v, eps=eps, eta=ETA, dt_max=DT_MAX,
                           n_iter=N_ITER, era_mode=0, era_log2=2,
                           precision=tsbts.TSBTS_MIXED)
    sim.schedule_log(40_000_000)
    sim.step_era(t_era)
    log = sim.schedule()
    sim.close()
    dm, dr, dv = (torch.from_numpy(x).to(f"cuda:{local}") for x in (m, r, v))
    loss = torch.empty(1, dtype=torch.float64, device=dm.device)
    gr = [torch.empty((n, 3), dtype=torch.float64, device=dm.device),
          torch.empty((n, 3), dtype=torch.float64, device=dm.device),
          torch.empty((n,), dtype=torch.float64, device=dm.device)]

    def one_gradient(**which):
        adj = tsbts.Adjoint(n, eps, precision=tsbts.TSBTS_MIXED,
                            stream=stream.cuda_stream, **which)
        with torch.cuda.stream(stream):
            tsbts.tsbts_adjoint_loss_grad(adj.ctx, dm, dr, dv, loss, *gr,
                                          device=True)
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            tsbts.tsbts_adjoint_loss_grad(adj.ctx, dm, dr, dv, loss, *gr,
                                          device=True)
            e_b.record(stream)
            e_b.synchronize()
        st = adj.stats()
        adj.close()
        ms = e_a.elapsed_time(e_b)
        E = st["entries"]
        return {"ms_per_gradient": ms, "gradients_s": 1e3 / ms,
                "Gpairs_s": 3 * (E + n) * n / (ms / 1e3) / 1e9,
                "schedule_entries": E, "passes": st["passes"],
                "precision": "mixed, taped"}
    # the final pass alone, and every pass of the era (the previous pass's
    # records carry part of the gradient)
    out["adjoint_plummer8192_era0-0.25"] = one_gradient(
        schedule=tsbts.final_pass_schedule(log, 0))
    out["adjoint_plummer8192_era0-0.25_all_passes"] = one_gradient(
        passes=tsbts.era_pass_schedules(log, 0))
    return out


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle, timed as it stands."""
    if rank != 0:
        return 0
    from paper_1205_2288_gb300 import inputs
    threads = os.cpu_count() or 1
    m, r, v = inputs.plummer(N_BODIES, SEED)
    tstep = 2.0 ** -9
    for _ in range(args.warmup):
        oracle_sample(m, r, v, tstep, threads)
    tot_i, tot_s, steps = 0, 0.0, 0
    for _ in range(args.steps):
        i, s, de, bs = oracle_sample(m, r, v, tstep, threads)
        tot_i += i
        tot_s += s
        steps += bs
    value = tot_i / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "Ginteractions/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": config_dict({"t_end": tstep, "precision": "fp64",
                               "sample": f"t=0..{tstep} per step"}),
        "block_steps_per_s": steps / tot_s,
        "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value,
                         "unit": "Ginteractions/s",
                         "sample": f"t=0..2^-9 of the workload per step"},
        "e2e": {"value": value, "unit": "Ginteractions/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def force_sweep(args):
    """Force kernel alone (tsbts_force, device pointers): Plummer n = 131072,
    eps = 1/512, seeded random active sets of the given sizes."""
    import numpy as np
    import torch

    from paper_1205_2288_gb300 import inputs, tsbts

    n, eps = 131072, 1.0 / 512.0
    dev = torch.device("cuda", 0)
    m, r, v = inputs.plummer(n, SEED)
    dm = torch.from_numpy(m).to(dev)
    dr = torch.from_numpy(r).to(dev)
    dv = torch.from_numpy(v).to(dev)
    sizes = [int(x) for x in args.n_act.split(",")] if args.n_act else \
        [1, 32, 1024, 32768, n]
    precs = [tsbts.TSBTS_MIXED] + ([] if args.no_fp64 else [tsbts.TSBTS_FP64])
    out = {}
    peak = measure_peaks(0)["fp32_peak_Ginteractions_s"] * 1e9
    for prec in precs:
        for na in sizes:
            idx = torch.from_numpy(inputs.active_subset(n, na, 1000 + na)).to(dev)
            a = torch.empty(na, 3, dtype=torch.float64, device=dev)
            phi = torch.empty(na, dtype=torch.float64, device=dev)
            q = torch.empty(na, dtype=torch.float64, device=dev)
            reps = args.steps if prec == tsbts.TSBTS_MIXED else 1
            for _ in range(args.warmup if prec == tsbts.TSBTS_MIXED else 1):
                tsbts.tsbts_force(prec, dm, dr, dv, eps, idx, a, phi, q)
            torch.cuda.synchronize()
            if args.profile_range:
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
                tsbts.tsbts_force(prec, dm, dr, dv, eps, idx, a, phi, q)
                torch.cuda.synchronize()
                torch.cuda.profiler.stop()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                tsbts.tsbts_force(prec, dm, dr, dv, eps, idx, a, phi, q)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gint = na * n / (ms / 1e3) / 1e9
            key = ("mixed" if prec else "fp64") + f"_nact{na}"
            out[key] = {"ms_per_call": ms, "Ginteractions_s": gint,
                        "frac_of_fp32_roofline": gint * 1e9 / peak}
    line = {"metric": "force kernel sweep (tsbts_force), Plummer n=131072, "
                      "eps=1/512", "unit": "Ginteractions/s",
            "peak_Ginteractions_s": peak / 1e9, "results": out}
    print(json.dumps(line), flush=True)
    return 0


def ensemble_bench(args):
    """512 independent Plummer clusters (sizes log-uniform in [64, 4096],
    Salpeter masses, eps = 4/N_c) integrated together over t = 0..0.5,
    mixed precision, fixed era 1/8, three passes."""
    import torch

    from paper_1205_2288_gb300 import inputs, tsbts

    off, m, r, v, eps = inputs.ensemble(args.clusters, seed=SEED)
    t_end = args.t_end if args.t_end != T_END else 0.5
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    kw = dict(eps=eps, eta=ETA, dt_max=DT_MAX, precision=tsbts.TSBTS_MIXED,
              n_iter=N_ITER, era_log2=3, stream=stream.cuda_stream)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    tot_s = 0.0
    tot_i = tot_steps = tot_launch = 0
    force_ms = 0.0
    force_n = 0
    for it in range(args.warmup + args.steps):
        g = tsbts.Ensemble(off, m, r, v, **kw)
        g.set_timing(it >= args.warmup)
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step_era(t_end)
        e1.record(stream)
        e1.synchronize()
        st = g.stats()
        if it >= args.warmup:
            tot_s += e0.elapsed_time(e1) / 1e3
            tot_i += st["interactions"]
            tot_steps += st["block_steps"]
            tot_launch += st["kernel_launches"]
            force_ms += st["force_ms"]
            force_n += st["force_launches"]
        g.close()
    peak = measure_peaks(0)["fp32_peak_Ginteractions_s"] * 1e9
    achieved = tot_i / (force_ms / 1e3) if force_ms else 0.0
    line = {
        "metric": "ensemble G pair-interactions/s (512 Plummer clusters)",
        "value": tot_i / tot_s / 1e9, "unit": "Ginteractions/s",
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps,
        "config": {"workload": f"ensemble{args.clusters}_plummer_salpeter_"
                               f"n64-4096_eps4overN_t0-{t_end}",
                   "clusters": args.clusters, "bodies": int(off[-1]),
                   "eta": ETA, "dt_max": DT_MAX, "era": "fixed 1/8",
                   "n_iter": N_ITER, "precision": "mixed"},
        "global_block_steps_per_s": tot_steps / tot_s,
        "kernel_launches_per_global_step": tot_launch / max(tot_steps, 1),
        "gpu_launches": tot_launch,
        "interactions_per_step": tot_i / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9,
                     "peak": peak / 1e9, "unit": "Ginteractions/s",
                     "frac": achieved / peak, "kernel": "ens_force_mixed_kernel",
                     "force_launches": force_n,
                     "peak_basis": "FP32 FMA lane-ops/s measured on this GPU "
                                   "by tsbts_pipe_peak / 20 FMA-pipe ops per "
                                   "interaction"},
    }
    print(json.dumps(line), flush=True)
    return 0


def study_job(job, span):
    """One run of the long-integration study: an ensemble of models with a
    fixed era (one cluster per model) or one model with a dynamic era,
    stepped time unit by time unit to `span`; returns each model's largest
    relative energy error over the run and its error at the end."""
    import numpy as np

    from paper_1205_2288_gb300 import inputs, tsbts

    prec = tsbts.TSBTS_MIXED if job["precision"] == "mixed" else \
        tsbts.TSBTS_FP64
    models = [inputs.plummer(job["n"], s) for s in job["seeds"]]
    t0 = time.perf_counter()
    if job["era"] == "dynamic":
        (m, r, v), = models
        g = tsbts.Simulation(m, r, v, eps=job["eps"], eta=job["eta"],
                             dt_max=job["dt_max"], n_iter=job["n_iter"],
                             era_mode=1, precision=prec)

        def energies():
            return np.array([sum(g.energy())])
    else:
        off = np.cumsum([0] + [len(x[0]) for x in models])
        g = tsbts.Ensemble(off, np.concatenate([x[0] for x in models]),
                           np.vstack([x[1] for x in models]),
                           np.vstack([x[2] for x in models]),
                           eps=np.full(len(models), job["eps"]),
                           eta=job["eta"], dt_max=job["dt_max"],
                           n_iter=job["n_iter"], era_log2=job["era_log2"],
                           precision=prec)

        def energies():
            ek, ep = tsbts.tsbts_ensemble_energy(g.ctx, len(models))
            return ek + ep
    try:
        e0 = energies()
        worst = np.zeros(len(models))
        for t in range(1, span + 1):
            g.step_era(float(t))
            err = np.abs(energies() - e0) / np.abs(e0)
            worst = np.maximum(worst, err)
        steps = g.stats()["block_steps"]
    finally:
        g.close()
    return dict(job, worst=worst.tolist(), at_end=err.tolist(),
                block_steps=int(steps), seconds=time.perf_counter() - t0)


def study(args):
    """The paper's long-integration era and iteration study on the GPU
    (Sec. 3: energy error against era size and pass count, 100-body models
    with eta = 0.1 and 500-body models with eta = 0.5, eps = 0.01, dt_max =
    1/64; Sec. 4: dynamic against fixed era of 1/64, three passes), in FP64
    and in mixed precision. Seeded Plummer models stand in for the paper's
    unpublished ones (the 100-body seeds are the oracle reruns' own, so the
    FP64 runs repeat those bit for bit). Every configuration's runs go on
    their own context and stream, many at a time."""
    import concurrent.futures as cf
    import math

    with open(os.path.join(ROOT, "tests", "golden",
                           "sec3_energy_experiment.json")) as f:
        sec3 = json.load(f)
    with open(os.path.join(ROOT, "tests", "golden",
                           "sec4_dynamic_era.json")) as f:
        sec4 = json.load(f)
    span = args.study_span
    precs = ["fp64", "mixed"] if args.study_precision == "both" else \
        [args.study_precision]
    base = dict(eps=sec3["eps_plummer"], dt_max=sec3["dt_max"])
    jobs = []
    for prec in precs:
        # Sec. 3, 100 bodies: five era sizes, three and five passes
        for n_iter in (3, 5):
            for era in sec3["era_sizes_in_figures"]:
                jobs.append(dict(base, study="sec3_n100", precision=prec,
                                 n=sec3["n_bodies"], eta=sec3["eta"],
                                 n_iter=n_iter, era=era,
                                 era_log2=round(-math.log2(era)),
                                 seeds=[1000 + k for k in range(
                                     sec3["n_realisations"])]))
        # Sec. 3, 500 bodies, eta = 0.5: seven era sizes, three passes
        for k in range(7):
            jobs.append(dict(base, study="sec3_n500", precision=prec, n=500,
                             eta=0.5, n_iter=3, era=2.0 ** -k, era_log2=k,
                             seeds=[3000 + j for j in range(5)]))
        # Sec. 4: ten models, fixed era 1/64 against the dynamic era
        for n, eta, s0 in ((sec4["n_bodies"], sec4["eta"], 2000),
                           (500, 0.5, 4000)):
            seeds = [s0 + k for k in range(sec4["n_realisations"])]
            tag = f"sec4_n{n}"
            jobs.append(dict(base, study=tag, precision=prec, n=n, eta=eta,
                             n_iter=sec4["n_iter"], era=sec4["fixed_era"],
                             era_log2=round(-math.log2(sec4["fixed_era"])),
                             seeds=seeds))
            for sd in seeds:
                jobs.append(dict(base, study=tag, precision=prec, n=n,
                                 eta=eta, n_iter=sec4["n_iter"],
                                 era="dynamic", seeds=[sd]))
    if args.study_only:
        keep = set(args.study_only.split(","))
        jobs = [j for j in jobs if j["study"] in keep]
    if args.study_eras:
        eras = {float(x) for x in args.study_eras.split(",")}
        jobs = [j for j in jobs
                if not j["study"].startswith("sec3") or j["era"] in eras]
    # the 500-body and dynamic runs take longest: start them first
    jobs.sort(key=lambda j: (-j["n"], j["era"] != "dynamic"))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=args.study_workers) as ex:
        done = list(ex.map(lambda j: study_job(j, span), jobs))
    wall = time.perf_counter() - t0

    def geo(x):
        return math.exp(sum(math.log(v) for v in x) / len(x))
    out = {}
    for prec in precs:
        res = {}
        for d in done:
            if d["precision"] != prec or not d["study"].startswith("sec3"):
                continue
            res.setdefault(d["study"], {})[
                f"passes{d['n_iter']}_era{d['era']}"] = {
                "worst_max": max(d["worst"]),
                "worst_median": statistics.median(d["worst"]),
                "block_steps": d["block_steps"]}
        for tag in ("sec4_n100", "sec4_n500"):
            if not any(d["study"] == tag for d in done):
                continue
            fixed = [d for d in done if d["precision"] == prec and
                     d["study"] == tag and d["era"] != "dynamic"][0]
            dyn = sorted((d for d in done if d["precision"] == prec and
                          d["study"] == tag and d["era"] == "dynamic"),
                         key=lambda d: d["seeds"][0])
            ratio = [dd["worst"][0] / fw
                     for dd, fw in zip(dyn, fixed["worst"])]
            res[tag] = {"dynamic_at_most_fixed": sum(x <= 1 for x in ratio),
                        "models": len(ratio),
                        "geomean_ratio_dynamic_over_fixed": geo(ratio),
                        "worst_fixed": max(fixed["worst"]),
                        "worst_dynamic": max(dd["worst"][0] for dd in dyn),
                        "block_steps_fixed": fixed["block_steps"],
                        "block_steps_dynamic": sum(dd["block_steps"]
                                                   for dd in dyn)}
        out[prec] = res
    line = {"metric": "long-integration era / iteration study "
                      "(largest relative energy error over the run)",
            "span_time_units": span, "runs": len(done),
            "models": sum(len(d["seeds"]) for d in done),
            "wall_seconds": wall, "results": out,
            "note": "seeded Plummer models stand in for the paper's; energy "
                    "sampled at every time unit"}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_bench(args):
    """Gradient of the mass-weighted mean-square radius at the end of one
    era with respect to the initial positions, velocities and masses,
    through the era's final-pass block schedule (replay with Eq. 2
    prediction, Eq. 3 forces, Eq. 1 correction, then reverse mode).
    Plummer n = 8192, eps = 0.01, eta = 0.01, fixed era 0..1/4, three
    passes; the schedule comes from the mixed integrator. One step = one
    gradient (forward replay + reverse sweep) from device-resident inputs.
    Pair terms counted per gradient: (E + n) n for the forward replay
    (E = schedule entries, n^2 for the initial force) and 2 (E + n) n for
    the two-sided force vector-Jacobian product."""
    import numpy as np
    import torch

    from paper_1205_2288_gb300 import inputs, tsbts

    n, eps, t_era = 8192, 0.01, 0.25
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    m, r, v = inputs.plummer(n, SEED)
    if args.schedule_in:
        # a schedule saved by an earlier run (--schedule-out)
        z = np.load(args.schedule_in)
        sched = (z["tau"], z["off"], z["act"])
    else:
        sim = tsbts.Simulation(m, r, v, eps=eps, eta=ETA, dt_max=DT_MAX,
                               n_iter=N_ITER, era_mode=0, era_log2=2,
                               precision=tsbts.TSBTS_MIXED)
        sim.schedule_log(40_000_000)
        sim.step_era(t_era)
        sched = tsbts.final_pass_schedule(sim.schedule(), 0)
        sim.close()
    if args.schedule_out:
        np.savez(args.schedule_out, tau=sched[0], off=sched[1], act=sched[2])
    if args.adjoint_steps:
        # the first steps of the schedule only (a smaller case for profiling)
        k = min(args.adjoint_steps, len(sched[0]))
        sched = (sched[0][:k], sched[1][:k + 1], sched[2][:sched[1][k]])
    E = int(sched[1][-1])
    S = int(len(sched[0]))
    pairs = 3 * (E + n) * n
    dm, dr, dv = (torch.from_numpy(x).to(dev) for x in (m, r, v))
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    g = [torch.empty((n, 3), dtype=torch.float64, device=dev),
         torch.empty((n, 3), dtype=torch.float64, device=dev),
         torch.empty((n,), dtype=torch.float64, device=dev)]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    variants = [("mixed_taped", tsbts.TSBTS_MIXED, 0),
                ("mixed_checkpoint64", tsbts.TSBTS_MIXED, 64)]
    if not args.no_fp64:
        variants.append(("fp64_taped", tsbts.TSBTS_FP64, 0))
    results = {}
    sampler = ClockSampler(0)
    clocks = None
    for name, prec, K in variants:
        adj = tsbts.Adjoint(n, eps, sched, precision=prec,
                            checkpoint_every=K, exact_order=0,
                            stream=stream.cuda_stream)
        reps = args.steps if prec == tsbts.TSBTS_MIXED else 1
        with torch.cuda.stream(stream):
            for _ in range(args.warmup if prec == tsbts.TSBTS_MIXED else 1):
                tsbts.tsbts_adjoint_loss_grad(adj.ctx, dm, dr, dv, loss, *g,
                                              device=True)
            torch.cuda.synchronize()
            if name == "mixed_taped":
                sampler.start()
            ms = 0.0
            fwd = bwd = 0.0
            launches0 = adj.stats()["kernel_launches"]
            for rep in range(reps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                profiled = (args.profile_range and name == "mixed_taped"
                            and rep == 0)
                if profiled:
                    torch.cuda.synchronize()
                    torch.cuda.profiler.start()
                e0.record(stream)
                tsbts.tsbts_adjoint_loss_grad(adj.ctx, dm, dr, dv, loss, *g,
                                              device=True)
                e1.record(stream)
                e1.synchronize()
                if profiled:
                    torch.cuda.profiler.stop()
                ms += e0.elapsed_time(e1)
                st = adj.stats()
                fwd += st["forward_ms"]
                bwd += st["backward_ms"]
            if name == "mixed_taped":
                clocks = sampler.stop()
        assert torch.isfinite(g[0]).all()
        ms /= reps
        results[name] = {
            "ms_per_gradient": ms, "Gpairs_s": pairs / (ms / 1e3) / 1e9,
            "forward_ms": fwd / reps, "backward_ms": bwd / reps,
            "pairs_backward_counted": st["pairs_backward"],
            "device_bytes": st["device_bytes"],
            "tape_bytes": st["tape_bytes"],
            "checkpoint_bytes": st["checkpoint_bytes"],
            "kernel_launches_per_gradient":
                (st["kernel_launches"] - launches0) // reps}
        adj.close()
    head = results["mixed_taped"]
    # end to end through the host-pointer API (copies in the timed region)
    adj = tsbts.Adjoint(n, eps, sched, precision=tsbts.TSBTS_MIXED)
    pin = [torch.from_numpy(x).pin_memory().numpy() for x in (m, r, v)]
    outs = [np.zeros(1), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)]
    adj.loss_grad(*pin)
    t0 = time.perf_counter()
    e2e_reps = max(1, min(args.steps, 2))
    for _ in range(e2e_reps):
        tsbts.tsbts_adjoint_loss_grad(adj.ctx, *pin, *outs)
    e2e_s = (time.perf_counter() - t0) / e2e_reps
    adj.close()
    peak = measure_peaks(0)["fp32_peak_Ginteractions_s"] * 1e9
    bwd_pairs = 2 * (E + n) * n
    achieved = bwd_pairs / (head["backward_ms"] / 1e3)
    line = {
        "metric": "adjoint: gradients/s of the era-end loss through the "
                  "frozen final-pass schedule (G pair terms/s)",
        "value": 1e3 / head["ms_per_gradient"], "unit": "gradients/s",
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_gradient"], "higher_is_better": True,
        "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "adjoint_plummer8192_eps0.01_eta0.01_era0-0.25"
                               "_3iter_final_pass",
                   "n": n, "eps": eps, "eta": ETA, "dt_max": DT_MAX,
                   "era": "fixed 1/4", "n_iter": N_ITER,
                   "schedule_steps": S, "schedule_entries": E,
                   "schedule_prefix_steps": args.adjoint_steps or None,
                   "loss": "sum m |r_T|^2 / sum m",
                   "l2": "256 MiB buffer written between timed gradients"},
        "pairs_per_gradient": pairs,
        "Gpairs_s": head["Gpairs_s"],
        "variants": results,
        "gpu_launches": head["kernel_launches_per_gradient"] * args.steps,
        "e2e": {"value": 1.0 / e2e_s, "unit": "gradients/s",
                "h2d_bytes_per_step": 7 * 8 * n,
                "d2h_bytes_per_step": (1 + 7 * n) * 8},
        "roofline": {"bound": "alu", "achieved": achieved / 1e9,
                     "peak": peak / 1e9, "unit": "Gpairs/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "reverse sweep (adj_vjp_kernel + "
                               "adj_back_step_kernel)",
                     "peak_basis": "FP32 FMA lane-ops/s measured on this GPU "
                                   "by tsbts_pipe_peak / 20 FMA-pipe ops per "
                                   "pair term"},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        oracle.set_threads(threads)
        tau, off, act = sched
        s_pre = int(np.searchsorted(off, 400_000))
        pre = (tau[:s_pre], off[:s_pre + 1], act[:off[s_pre]])
        e_pre = int(off[s_pre])
        t0 = time.perf_counter()
        oracle.loss_grad(m, r, v, eps, 20, pre)
        osec = time.perf_counter() - t0
        opairs = 3 * (e_pre + n) * n
        line["cpu_baseline"] = {
            "value": opairs / osec / 1e9, "unit": "Gpairs/s", "cores": threads,
            "kind": "oracle",
            "sample": f"first {s_pre} steps ({e_pre} entries) of the "
                      f"schedule, one gradient, {osec:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--t-end", type=float, default=T_END)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed mixed path (no fp64 run, configs "
                         "or cpu_baseline)")
    ap.add_argument("--force-sweep", action="store_true",
                    help="time the force kernel alone on n = 131072")
    ap.add_argument("--n-act", default="",
                    help="comma-separated active-set sizes for --force-sweep")
    ap.add_argument("--ensemble", action="store_true",
                    help="integrate the 512-cluster ensemble instead")
    ap.add_argument("--clusters", type=int, default=512)
    ap.add_argument("--graph-steps", type=int, default=-1,
                    help="block steps per captured graph replay (default: "
                         "the library's)")
    ap.add_argument("--study", action="store_true",
                    help="the paper's long era / iteration study (Sec. 3-4)")
    ap.add_argument("--study-span", type=int, default=100,
                    help="--study: time units per run (the paper: 1000)")
    ap.add_argument("--study-precision", default="both",
                    choices=["both", "fp64", "mixed"])
    ap.add_argument("--study-workers", type=int, default=32,
                    help="--study: runs in flight at once")
    ap.add_argument("--study-only", default="",
                    help="--study: comma list of sec3_n100, sec3_n500, "
                         "sec4_n100, sec4_n500")
    ap.add_argument("--study-eras", default="",
                    help="--study: comma list of the Sec. 3 era sizes to run")
    ap.add_argument("--adjoint", action="store_true",
                    help="gradient through a frozen block schedule")
    ap.add_argument("--schedule-out", default="",
                    help="--adjoint: save the schedule (.npz)")
    ap.add_argument("--schedule-in", default="",
                    help="--adjoint: replay a saved schedule instead of "
                         "integrating the era")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="--adjoint: use the schedule's first N steps")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the first timed step (--adjoint: the "
                         "first timed mixed gradient) with cudaProfilerStart/"
                         "Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.force_sweep:
        return force_sweep(args)
    if args.ensemble:
        return ensemble_bench(args)
    if args.adjoint:
        return adjoint_bench(args)
    if args.study:
        return study(args)
    ws, rank, local = dist_env()
    dist = init_dist(ws)
    if args.impl == "reference":
        rc = run_reference(args, ws, rank)
        if dist:
            dist.destroy_process_group()
        return rc

    import numpy as np
    import torch

    from paper_1205_2288_gb300 import inputs, tsbts

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    t_end = args.t_end
    peaks = measure_peaks(local)
    peak_g = peaks["fp32_peak_Ginteractions_s"]
    m, r, v = inputs.plummer(N_BODIES, SEED + rank)
    dm = torch.from_numpy(m).to(dev)
    dr = torch.from_numpy(r).to(dev)
    dv = torch.from_numpy(v).to(dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    cfg = tsbts.tsbts_config_default()
    cfg.precision = tsbts.TSBTS_MIXED
    cfg.n_iter = N_ITER
    cfg.era_mode = 1
    cfg.k_max = 20
    cfg.device = local
    cfg.stream = stream.cuda_stream
    if args.graph_steps >= 0:
        cfg.graph_steps = args.graph_steps
    ctx = tsbts.tsbts_create(cfg)

    def one_step(timing):
        tsbts.tsbts_init_device(ctx, dm, dr, dv, EPS, ETA, DT_MAX)
        tsbts.tsbts_set_timing(ctx, timing)
        tsbts.tsbts_step_era(ctx, t_end)
        return tsbts.tsbts_get_stats(ctx)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step(0)
        # timed region: K full integrations, inputs resident in HBM
        sampler = ClockSampler(local)
        tot_inter = tot_steps = tot_launch = 0
        force_ms = 0.0
        force_launches = 0
        force_inter = 0
        elapsed_ms = 0.0
        barrier(dist)
        torch.cuda.synchronize()
        sampler.start()
        for k in range(args.steps):
            flush.fill_(1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            if args.profile_range and k == 0:
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
            ev0.record(stream)
            st = one_step(TIMING_PERIOD)
            ev1.record(stream)
            ev1.synchronize()
            if args.profile_range and k == 0:
                torch.cuda.profiler.stop()
            elapsed_ms += ev0.elapsed_time(ev1)
            tot_inter += st["interactions"]
            tot_steps += st["block_steps"]
            tot_launch += st["kernel_launches"]
            force_ms += st["force_ms"]
            force_launches += st["force_launches"]
            force_inter += st["force_interactions"]
        torch.cuda.synchronize()
        barrier(dist)
        clocks = sampler.stop()
        ek, ep, _ = tsbts.tsbts_energy(ctx)
        tsbts.tsbts_init_device(ctx, dm, dr, dv, EPS, ETA, DT_MAX)
        e0 = sum(tsbts.tsbts_energy(ctx)[:2])
        de_mixed_full = abs((ek + ep) / e0 - 1.0)

        # end to end through the public API with host buffers
        e2e_s = 0.0
        e2e_inter = 0
        pin = {k: torch.from_numpy(x).pin_memory() for k, x in
               dict(m=m, r=r, v=v).items()}
        h2d = 7 * 8 * N_BODIES
        d2h = 6 * 8 * N_BODIES
        for _ in range(max(1, min(args.steps, 2))):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tsbts.tsbts_init(ctx, pin["m"].numpy(), pin["r"].numpy(),
                             pin["v"].numpy(), EPS, ETA, DT_MAX)
            tsbts.tsbts_step_era(ctx, t_end)
            out = tsbts.tsbts_state(ctx, N_BODIES)
            e2e_s += time.perf_counter() - t0
            e2e_inter += tsbts.tsbts_get_stats(ctx)["interactions"]
            assert np.isfinite(out["r"]).all()

    sec = elapsed_ms / 1e3
    sec_max = reduce_max(dist, sec)
    inter_all = reduce_sum(dist, tot_inter)
    value = inter_all / sec_max / 1e9
    e2e_value = reduce_sum(dist, e2e_inter) / reduce_max(dist, e2e_s) / 1e9

    line = None
    if rank == 0:
        clk = clocks.get("sm_mhz") or None
        achieved = force_inter / (force_ms / 1e3) if force_ms > 0 else 0.0
        roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_g,
                "unit": "Ginteractions/s", "frac": achieved / 1e9 / peak_g,
                "traffic": FORCE_TRAFFIC_BYTES,
                "traffic_unit": "DRAM bytes per force launch (ncu, cold "
                                "cache; the live j set is L2-resident)",
                "algorithmic_bytes_per_launch": FORCE_ALGORITHMIC_BYTES,
                "kernel": "force_mixed_kernel",
                "peak_basis": "FP32 FMA lane-ops/s measured on this GPU by "
                              "tsbts_pipe_peak / 20 FMA-pipe ops per "
                              "interaction",
                "peak_nominal": peaks["nominal_fp32_peak_Ginteractions_s"],
                "frac_of_nominal": achieved / 1e9
                / peaks["nominal_fp32_peak_Ginteractions_s"],
                "force_launches_timed": force_launches,
                "force_interactions_timed": force_inter,
                "timing_sample": f"every {TIMING_PERIOD}th chunk of block "
                                 "steps carries CUDA events around its "
                                 "force launches",
                "force_us_per_launch": 1e3 * force_ms / max(force_launches, 1)}
        if clk:
            roof["frac_at_measured_clock"] = achieved / (
                peaks["sm_count"] * FP32_LANES_PER_SM * clk * 1e6
                / OPS_PER_INTERACTION)
        line = {
            "metric": METRIC, "value": value, "unit": "Ginteractions/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": config_dict({"precision": "mixed", "t_end": t_end,
                                   "parallelism": f"replicas{ws}"}),
            "block_steps_per_s": tot_steps / sec,
            "us_per_block_step": 1e6 * sec / max(tot_steps, 1),
            "interactions_per_step": tot_inter / args.steps,
            "gpu_launches": tot_launch,
            "e2e": {"value": e2e_value, "unit": "Ginteractions/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "peaks": {k: peaks[k] for k in (
                "sm_count", "fp32_lane_ops_per_s", "fp64_lane_ops_per_s",
                "fp32_peak_Ginteractions_s", "fp64_peak_Ginteractions_s",
                "clocks")},
            "clocks": clocks,
            "accuracy": {"t_end": t_end, "dE_E_mixed_gpu": de_mixed_full},
        }

    tsbts.tsbts_destroy(ctx)

    if rank == 0:
        acc = line["accuracy"]
        per_step = tot_inter / args.steps
        steps_1 = tot_steps / args.steps
        if os.path.exists(GOLDEN) and t_end == T_END:
            with open(GOLDEN) as f:
                gold = json.load(f)
            acc["dE_E_oracle"] = gold["dE_E"]
            acc["oracle_source"] = ("tests/golden/oracle_plummer16384_t1.json "
                                    "(the FP64 oracle over the same "
                                    "t = 0..1)")
            acc["mixed_within_2x_oracle"] = bool(
                de_mixed_full <= 2 * gold["dE_E"])
            acc["schedule_vs_oracle"] = {
                "mixed_block_steps": steps_1,
                "oracle_block_steps": gold["block_steps"],
                "mixed_interactions": per_step,
                "oracle_interactions": gold["interactions"],
                "interactions_rel_diff":
                    per_step / gold["interactions"] - 1.0}
        if not args.no_fp64 and not args.quick:
            # the plain FP64 GPU path over the same span, timed the same way
            sec64, st64, de64 = timed_integration(
                m, r, v, t_end, stream, eps=EPS, eta=ETA, dt_max=DT_MAX,
                precision=tsbts.TSBTS_FP64, n_iter=N_ITER, era_mode=1,
                device=local)
            v64 = st64["interactions"] / sec64 / 1e9
            line["fp64"] = {
                "value": v64, "unit": "Ginteractions/s",
                "span": f"t=0..{t_end}, CUDA events on the stream",
                "seconds": sec64, "block_steps": st64["block_steps"],
                "speedup_mixed_over_fp64": value / v64,
                "roofline": {"bound": "alu", "achieved": v64,
                             "peak": peaks["fp64_peak_Ginteractions_s"],
                             "frac": v64 / peaks["fp64_peak_Ginteractions_s"],
                             "peak_basis": "FP64 FMA lane-ops/s measured by "
                                           "tsbts_pipe_peak / 20 ops per "
                                           "interaction (whole integrator)"}}
            acc["dE_E_fp64_gpu"] = de64
            if "dE_E_oracle" in acc:
                acc["fp64_within_2x_oracle"] = bool(
                    de64 <= 2 * acc["dE_E_oracle"])
                acc["schedule_vs_oracle"]["fp64_block_steps"] = \
                    st64["block_steps"]
        if not args.quick:
            line["configs"] = config_results(local, stream, peak_g)
        if not args.no_cpu_baseline and not args.quick:
            threads = os.cpu_count() or 1
            oi, osec, ode, obs = oracle_sample(m, r, v, SAMPLE_T, threads)
            line["cpu_baseline"] = {
                "value": oi / osec / 1e9, "unit": "Ginteractions/s",
                "cores": threads, "kind": "oracle",
                "sample": f"t=0..{SAMPLE_T} of the workload ({oi} "
                          f"interactions, {osec:.1f} s)"}
        print(json.dumps(line), flush=True)
    if dist:
        barrier(dist)
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
