#!/usr/bin/env python3
"""Benchmark: accepted system-steps per second of the per-thread ODE
integrators on synthetic sweeps shaped like the paper's test cases.

Default workload: Duffing oscillator x'' + k x' + x + x^3 = B cos t on a
512 x 256 grid (k in [0.2, 0.3], B in [0.3, 0.5]), 2^17 systems, binary64
RKCK45 rtol = atol = 1e-10, h0 = 1e-2, local-maximum event y2 = 0 located to
1e-12, 1024 transient + 64 recorded periods of 2 pi.  One benchmark step is
one whole pass: reset the initial conditions from HBM, integrate every system
over all 1088 periods in one launch (the form the library's autotuner picks:
one thread per system or the persistent work queue), write the 64 records.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload duffing_rkck|duffing_rk4|valve|keller_miksis|duffing_lyapunov|
                   keller_miksis_collapse|keller_miksis_dual|valve_paper|serving]
Under torchrun each rank integrates its own sweep (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

# Algorithmic binary64 flops per accepted step, counted from the kernel's
# formulas (add, mul = 1; fma = 2; the transcendental calls are listed
# separately and not counted).  Duffing RKCK45: 6 right-hand sides x 10
# (= 60), stage times 10, stage states 70, update 18, error estimate 20,
# error norm 10, step-size controller 20, time update 1  -> 209 (+ 6 cos).
# Duffing RK4: 4 x 10 + stage times 4 + stage states 14 + update 18 + 1 = 77
# (+ 4 cos).  Valve RKCK45: 6 x 11 + 10 + 105 + 27 + 30 + 15 + 20 + 1 = 274
# (+ 6 sqrt).  Keller-Miksis RKCK45: 6 x 36 + 10 + 70 + 18 + 20 + 10 + 20 + 1
# = 365 (+ 6 pow, 6 sincospi, 12 div).  Duffing with its polar
# linearisation (n = 4): 6 x 23 + 10 + 140 + 36 + 40 + 20 + 20 + 1 = 405
# (+ 6 cos of the forcing, 6 sincos of the angle, credited as cos).
FLOPS_PER_STEP = {"duffing_rkck": 209, "duffing_rk4": 77, "valve": 274, "keller_miksis": 365,
                  "duffing_lyapunov": 405, "keller_miksis_collapse": 365, "keller_miksis_dual": 365,
                  "valve_paper": 274}
# The binary32 right-hand-side form splits those flops: binary64 keeps the
# update (1 fma per component), the error estimate (1 mul per component), the
# error norm, the controller and the time update; the rest (right-hand sides,
# stage times and states, weighted stage sums) is binary32.  Duffing RKCK45:
# 4 + 2 + 10 + 20 + 1 = 37 binary64, 209 - 37 = 172 binary32.  Valve:
# 6 + 3 + 15 + 20 + 1 = 45 binary64, 274 - 45 = 229 binary32.
FLOPS_FP32RHS = {"duffing_rkck": (37, 172), "valve": (45, 229)}
# transcendental calls per accepted step, converted to DFMA equivalents with
# the library's call-cost probe (one DFMA = 2 flops) for the FMA-peak roofline
# (the dual-frequency Keller-Miksis adds sin and cos of the second drive per
# stage: 12 more)
TRANSCENDENTALS = {"duffing_rkck": {"cos": 6}, "duffing_rk4": {"cos": 4}, "valve": {"sqrt": 6},
                   "keller_miksis": {"pow": 6, "cos": 12}, "duffing_lyapunov": {"cos": 12},
                   "keller_miksis_collapse": {"pow": 6, "cos": 12},
                   "keller_miksis_dual": {"pow": 6, "cos": 24}, "valve_paper": {"sqrt": 6}}
METRIC = "accepted system-steps/s (FP64, rtol 1e-10)"
METRIC_FP32RHS = "accepted system-steps/s (binary32 RHS stages, binary64 state and control, rtol 1e-10)"
UNIT = "system-steps/s"


def workload(name, rank=0):
    if name == "duffing_rkck":
        return rank_band(W.duffing_rkck(), rank)
    if name == "duffing_rk4":
        return W.duffing_rk4()
    if name == "valve":
        return W.valve()
    if name == "keller_miksis":
        return W.keller_miksis(n_transient=16, n_record=16)
    if name == "duffing_lyapunov":
        return W.duffing_lyapunov()
    # the paper's own protocols (Sec. 7.2, 7.3), bounded to a few seconds per
    # pass: collapse-to-collapse iterations (16 + 8 instead of 1024 + 64)
    if name == "keller_miksis_collapse":
        return W.keller_miksis_collapse(255, 256, n_transient=16, n_record=8)
    if name == "keller_miksis_dual":
        return W.keller_miksis_dual(128, 128, n_transient=16, n_record=8)
    if name == "valve_paper":
        return dict(W.valve(rtol=1e-10), name="valve_65536_rtol1e-10")
    raise SystemExit("unknown workload %s" % name)


def describe(w, persistent, l2):
    d = {"workload": w["name"], "systems": w["N"], "periods": w["n_transient"] + w["n_record"],
         "recorded_periods": w["n_record"], "scheme": "RKCK45" if w["scheme"] == 1 else "RK4",
         "rtol": w["rtol"], "launch": {0: "one thread per system", 1: "persistent work queue (clustered chunks)",
                    2: "persistent work queue (lane order)"}[persistent],
         "l2": l2}
    if w["events_on"]:
        d["events"] = ("y2=0 (maximum, stop 1) and y1=0 (impact, y2 <- -r y2), tol %g" % w["evt_tol"][0]
                       if w["model"] == W.VALVE else
                       "y2=0 dir %d located to %g, stop %d" % (w["evt_dir"][0], w["evt_tol"][0], w["evt_stop"][0]))
    return d


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# multi-rank aggregation (weak scaling: every rank integrates its own sweep)
# ---------------------------------------------------------------------------
def rank_band(w, rank):
    """Weak scaling: rank r sweeps the base grid of B shifted up by 0.25 r, so
    ranks never integrate the same system."""
    w = dict(w)
    w["p"] = w["p"].copy()
    w["p"][1] += 0.25 * rank
    return w


def kernel_source_digest():
    """sha256 over the sources that define the integrator kernels (headers
    and the per-model kernel units): a DRAM traffic figure measured by ncu
    applies only to the kernel sources it was taken on."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1810_03931_gb300", "csrc")
    files = sorted(f for f in os.listdir(csrc) if f.endswith(".cuh") or f.startswith("kern_"))
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(workload_name, launch, path=None):
    """DRAM bytes (read + write) of one integrator launch of this workload
    and launch form, from the ncu summary committed under profiles/ -- or None
    when it was taken on other kernel sources."""
    path = path or os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    e = table.get(workload_name, {}).get({0: "per_sweep", 1: "persistent", 2: "persistent_lane_order"}[launch])
    if not e or e.get("source_sha256") != kernel_source_digest():
        return None
    return float(e["dram_bytes_per_launch"])


def measured_counter(workload_name, launch, key, path=None):
    """A per-launch ncu counter (e.g. FP64-pipe utilisation) of this workload
    and launch form from the committed summary table, or None when it was
    taken on other kernel sources."""
    path = path or os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    e = table.get(workload_name, {}).get({0: "per_sweep", 1: "persistent", 2: "persistent_lane_order"}[launch])
    if not e or e.get("source_sha256") != kernel_source_digest() or key not in e:
        return None
    return float(e[key])


def credited_calls(trans, eq, per_step, achieved_tflops, peak_tflops, cos_eq, pow_eq, sqrt_eq):
    """Secondary figure: the transcendental calls the algorithm makes (cos of
    the forcing, pow, sqrt) credited at the library's measured call cost.  The
    kernel replaces them by cheaper arithmetic (angle addition, Newton-refined
    roots), so this credits work the kernel does not do; it is reported only
    while it stays below the peak."""
    frac = achieved_tflops / peak_tflops
    return {"transcendentals_per_step": trans,
            "call_cost_dfma_equiv": {"cos": round(cos_eq, 2), "pow": round(pow_eq, 2), "sqrt": round(sqrt_eq, 2)},
            "flops_per_step": per_step,
            "frac": frac if frac <= 1.0 else None,
            "note": "credit for library calls the kernel replaces with cheaper arithmetic; not the roofline"
                    + ("" if frac <= 1.0 else "; above the peak here, so withheld")}


def reduce_over_ranks(steps, ms, e2e_steps, e2e_s, world, device):
    """Whole-job numbers: (sum of accepted steps, max time in ms, end-to-end
    rate = sum of steps / max end-to-end time).  One collective per quantity
    on the timing path only; the integration itself has no collective."""
    e2e_rate = (e2e_steps / e2e_s) if e2e_s > 0 else None
    if world <= 1:
        return steps, ms, e2e_rate
    import torch
    import torch.distributed as dist
    t = torch.tensor([steps, e2e_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    e2e_rate = float(t[1]) / float(m[1]) if float(m[1]) > 0 else None
    return float(t[0]), float(m[0]), e2e_rate


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1810_03931_gb300 import build as B
    from paper_1810_03931_gb300 import odegpu as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    G.load(build_if_missing=False)

    from paper_1810_03931_gb300.sweeps import MODEL_DIMS as DIMS
    from paper_1810_03931_gb300.sweeps import params as sweep_params

    w = workload(args.workload, rank)
    if args.order in ("shuffled", "clustered"):
        # the same systems in a seeded random order: neighbouring lanes no
        # longer share similar parameters (the "clustering" remark of Sec. 7.2)
        perm = np.random.default_rng(W.SEED).permutation(w["N"])
        w = dict(W.subset(w, perm), name=w["name"] + "_shuffled")
    if args.order == "clustered":
        # ... then put back in order by the library's Z-order of the swept
        # parameters
        if w["model"] == W.KELLER_MIKSIS:
            keys = np.vstack([w[k] for k in ("PA", "omega", "PA2", "omega2") if k in w])
        else:
            keys = w["p"][np.ptp(w["p"], axis=1) > 0]
        w = dict(W.subset(w, G.ode_cluster_order(keys)), name=w["name"] + "_clustered")
    if args.systems is not None and args.systems < w["N"]:
        w = dict(W.subset(w, np.arange(args.systems)), name=w["name"] + "_first%d" % args.systems)
    if args.n_transient is not None:
        w["n_transient"] = args.n_transient
    if args.n_record is not None:
        w["n_record"] = args.n_record
    n, P, A, E = DIMS[w["model"]]
    N = w["N"]
    n_tr, n_rec = w["n_transient"], w["n_record"]
    R = A + n + 1
    stream = torch.cuda.current_stream(dev)

    prec = G.ODE_FP32_RHS if args.prec == "fp32rhs" else G.ODE_FP64
    s = G.ode_create(w["model"], w["scheme"], prec, N, local)
    G.ode_set_tolerances(s, np.full(n, w["rtol"]), np.full(n, w["atol"]), w["hmax"], w["hmin"], w["grow"],
                         w["shrink"])
    G.ode_set_events(s, int(w["events_on"]), np.array(w["evt_dir"][:E], dtype=np.int32),
                     np.array(w["evt_tol"][:E]), np.array(w["evt_stop"][:E], dtype=np.int32), w["max_eq"])
    if w["mc"]:
        G.ode_set_model_constants(s, np.array(w["mc"], dtype=np.float64))
    G.ode_set_time_domain_mode(s, w["td_mode"])
    G.ode_set_launch(s, args.block, args.persistent)
    G.ode_set_schedule(s, args.systems_per_thread, args.slices_per_launch, args.warp_sync)

    params = sweep_params(w)
    # resident inputs (HBM) and the records buffer
    d_td = torch.tensor(w["td"], dtype=torch.float64, device=dev)
    d_y0 = torch.tensor(w["y0"], dtype=torch.float64, device=dev)
    d_p = torch.tensor(params, dtype=torch.float64, device=dev)
    d_acc = torch.zeros((A, N), dtype=torch.float64, device=dev)
    d_rec = torch.zeros((n_rec, R, N), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    nacc = np.zeros(N, dtype=np.int64)

    def step():
        G.ode_reset_counters(s, stream)
        G.ode_linear_set(s, 0, 0, N, N, td=d_td, y=d_y0, p=d_p, acc=d_acc, copy_mode=G.ODE_ALL, stream=stream)
        G.ode_run_periods(s, w["h0"], n_tr, n_rec, d_rec, stream=stream)

    tune = None
    if args.autotune:
        # the project's autotuner picks the launch shape on a short trial
        G.ode_linear_set(s, 0, 0, N, N, td=d_td, y=d_y0, p=d_p, acc=d_acc, copy_mode=G.ODE_ALL, stream=stream)
        t = G.ode_autotune(s, w["h0"], args.tune_slices, stream, full=True)
        trials = t["trial_ms"]
        tune = {"block": t["block"], "persistent": t["persistent"],
                "systems_per_thread": t["systems_per_thread"], "slices_per_launch": t["slices_per_launch"],
                "warp_sync": t["warp_sync"],
                "trial_slices": args.tune_slices,
                "trial_ms": {"per_sweep": [round(x, 2) for x in trials[0]],
                             "per_sweep_2_systems_per_thread": [round(x, 2) for x in trials[1]],
                             "persistent": [round(x, 2) for x in trials[2]],
                             "persistent_lane_order": [round(x, 2) for x in trials[3]],
                             "blocks": [64, 96, 128, 160, 192, 256],
                             "schedule_spl1_half_all_warpsync": [round(x, 2) for x in t["split_ms"]],
                             "warp_sync_per_form_at_its_best_block": [round(x, 2) for x in t["warp_sync_ms"]]}}
        args.persistent = t["persistent"]
        args.block = t["block"]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    acc_steps = []
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        G.ode_get_status(s, accepted=nacc, stream=stream)  # host copy: synchronizes
        acc_steps.append(int(nacc.sum()))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = sum(ms) / len(ms)
    steps_per_pass = float(np.mean(acc_steps))

    # end to end through the C ABI with host buffers: H2D of the inputs, the
    # integration, D2H of the records and the per-system step counts
    h_td = torch.tensor(w["td"], dtype=torch.float64).pin_memory()
    h_y0 = torch.tensor(w["y0"], dtype=torch.float64).pin_memory()
    h_p = torch.tensor(params, dtype=torch.float64).pin_memory()
    h_acc = torch.zeros((A, N), dtype=torch.float64).pin_memory()
    h_rec = torch.zeros((n_rec, R, N), dtype=torch.float64).pin_memory()
    h_nacc = torch.zeros(N, dtype=torch.int64).pin_memory()
    e2e_times, e2e_steps = [], []
    for k in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.ode_reset_counters(s, stream)
        G.ode_linear_set(s, 0, 0, N, N, td=h_td, y=h_y0, p=h_p, acc=h_acc, copy_mode=G.ODE_ALL, stream=stream)
        G.ode_run_periods(s, w["h0"], n_tr, n_rec, h_rec, stream=stream)
        G.ode_get_status(s, accepted=h_nacc, stream=stream)
        e2e_times.append(time.perf_counter() - t0)
        e2e_steps.append(int(h_nacc.numpy().sum()))
    h2d = 8 * (2 + n + P + A) * N
    d2h = 8 * n_rec * R * N + 8 * N

    # roofline peak: binary64 FMA units per SM (2, measured by the probe
    # below as FMA per clock per SM) x SMs x maximum SM clock x 2 flops
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    max_mhz = None
    if os.path.exists(peaks_path):
        max_mhz = json.load(open(peaks_path)).get("sm_max_mhz")
    if not max_mhz:
        max_mhz = clk.get("sm_max_mhz") or 2070.0
    dfma, ffma = G.ode_probe_fma_peak(local)
    cos_eq, pow_eq, sqrt_eq = G.ode_probe_call_cost(local)
    peak_tflops = 2 * 2 * sms * max_mhz * 1e6 / 1e12
    peak32_tflops = 128 * 2 * sms * max_mhz * 1e6 / 1e12  # 128 binary32 FMA lanes per SM
    arith = FLOPS_PER_STEP.get(args.workload, 0)
    trans = TRANSCENDENTALS.get(args.workload, {})
    eq = {"cos": cos_eq, "pow": pow_eq, "sqrt": sqrt_eq}
    per_step = arith + sum(2.0 * eq[k] * v for k, v in trans.items())
    fp32_split = None
    if args.prec == "fp32rhs":
        # mixed precision: the fraction of the step time the two FMA pipes
        # need at their peaks; achieved is stated in binary64-equivalent flops
        # (binary32 flops x peak64 / peak32); forcing evaluations not counted
        f64, f32 = FLOPS_FP32RHS.get(args.workload, (arith, 0))
        arith = f64 + f32 * peak_tflops / peak32_tflops
        per_step = arith
        trans = {}
        fp32_split = {"fp64_flops_per_step": f64, "fp32_flops_per_step": f32, "peak_fp32": peak32_tflops}
    achieved_tflops = per_step * steps_per_pass / (ms_step * 1e-3) / 1e12
    achieved_arith = arith * steps_per_pass / (ms_step * 1e-3) / 1e12

    G.ode_destroy(s)

    # aggregate over ranks: total accepted steps / max time
    tot_steps, max_ms, e2e_rate = reduce_over_ranks(
        steps_per_pass, ms_step, float(np.mean(e2e_steps)) if e2e_steps else 0.0,
        float(np.mean(e2e_times)) if e2e_times else 0.0, world, dev)

    line = None
    spl = tune["slices_per_launch"] if tune else args.slices_per_launch
    if rank == 0:
        value = tot_steps / (max_ms * 1e-3)
        line = {
            "metric": METRIC if args.prec == "fp64" else METRIC_FP32RHS, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32 rhs / f64 state",
            "data": "synthetic",
            "config": describe(w, args.persistent, "flushed before every timed step (256 MB write)"),
            "accepted_steps_per_pass": steps_per_pass, "wall_s_timed": wall,
            "e2e": {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "s_per_step": float(np.mean(e2e_times)) if e2e_times else None},
            # integrator launches per step: one, or one per slices_per_launch slices
            "gpu_launches": args.steps * (1 if not spl else -(-(w["n_transient"] + w["n_record"]) // spl)),
            # the roofline leads with the method's own arithmetic: the add /
            # mul / fma of the algorithm per accepted step (FMA = 2 flops)
            # times accepted steps per CUDA-event second, against the binary64
            # FMA peak; the FP64-pipe utilisation ncu measured on the same
            # kernel sources stands beside it
            "roofline": {"bound": "alu", "achieved": achieved_arith, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved_arith / peak_tflops,
                         "traffic": args.traffic if args.traffic is not None
                         else measured_traffic(w["name"], args.persistent),
                         "fp64_pipe_active_ncu": measured_counter(w["name"], args.persistent,
                                                                  "fp64_pipe_active_pct"),
                         "fp64_pipe_inst_per_step_ncu": measured_counter(w["name"], args.persistent,
                                                                         "fp64_pipe_inst_per_step"),
                         "basis": "algorithmic binary64 flops of the method per accepted step x accepted "
                                  "steps / CUDA-event time of the integrator launch",
                         "arith_flops_per_step": arith,
                         "peak_basis": "2 FP64 FMA/clk/SM x %d SMs x %.0f MHz x 2 (derived; live probe %.3f TFLOP/s)"
                                       % (sms, max_mhz, 2 * dfma / 1e12),
                         "credit_for_replaced_calls": credited_calls(trans, eq, per_step, achieved_tflops,
                                                                     peak_tflops, cos_eq, pow_eq, sqrt_eq)},
            # accepted steps differ between forms (the binary32 error estimate
            # carries rounding noise): system-periods/s compares them on work
            "system_periods_per_s": world * w["N"] * (w["n_transient"] + w["n_record"]) / (max_ms * 1e-3),
            "launch": tune if tune else {"block": args.block, "persistent": args.persistent,
                                         "systems_per_thread": args.systems_per_thread,
                                         "slices_per_launch": args.slices_per_launch,
                                         "warp_sync": args.warp_sync},
            "clocks": clk,
        }
        if fp32_split is not None:
            line["roofline"].update(fp32_split, unit="TFLOP/s (binary64-equivalent)")
        if line["roofline"]["traffic"] is not None:
            # HBM is not the bound: its achieved rate, for evidence
            line["roofline"]["hbm_gbs_achieved"] = line["roofline"]["traffic"] / (max_ms * 1e-3) / 1e9
        if not args.no_cpu_baseline and world == 1:  # CPU baseline: rank 0 at N = 1 only
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU oracle: timed on the host cores on a bounded sample of the workload
# ---------------------------------------------------------------------------
def _oracle_rate(w, n_sys, nthreads):
    import oracle
    idx = W.sample_indices(w["N"], n_sys)
    ws = W.subset(w, idx)
    t0 = time.perf_counter()
    r = oracle.run_workload(ws, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return float(r["nacc"].sum()) / dt, dt, len(idx)


def cpu_baseline(w, seconds):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # calibrate on a few systems, then size the sample to ~`seconds` of wall
    rate1, dt1, n1 = _oracle_rate(w, cores, cores)
    per_sys = dt1 / max(1, n1) * cores
    n_sys = int(max(cores, min(w["N"], seconds / max(per_sys, 1e-6) * cores)))
    rate, dt, n = _oracle_rate(w, n_sys, cores)
    # the same oracle on one core, on a smaller sample (~ seconds / 4 of wall)
    n_one = int(max(1, min(n_sys, seconds / 4 / max(per_sys, 1e-6))))
    rate_one, dt_one, n_one = _oracle_rate(w, n_one, 1)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d systems (seeded), all %d periods, %.1f s wall on %d threads"
                      % (n, w["N"], w["n_transient"] + w["n_record"], dt, cores),
            "value_1_core": rate_one,
            "sample_1_core": "%d systems, %.1f s wall on 1 thread" % (n_one, dt_one),
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "CPU part"):
            for line in txt.splitlines():
                if line.startswith(key):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload(args.workload)
    cores = os.cpu_count() or 1
    budget = max(10.0, 150.0 / max(1, args.steps + args.warmup))
    rate1, dt1, n1 = _oracle_rate(w, cores, cores)
    n_sys = int(max(cores, min(w["N"], budget / max(dt1 / n1 * cores, 1e-6) * cores)))
    for _ in range(args.warmup):
        _oracle_rate(w, max(cores, n_sys // 4), cores)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, n = _oracle_rate(w, n_sys, cores)
        rates.append(r)
        times.append(dt)
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, 0, "n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of %d systems (seeded) per step, all periods" % (n_sys, w["N"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Serving mix: continuous batching of sweep requests
# ---------------------------------------------------------------------------
W_NAMES = {0: "duffing", 1: "keller_miksis", 2: "valve", 3: "bounce", 4: "duffing_lyapunov"}


def run_serving(args):
    import torch
    from paper_1810_03931_gb300 import build as B
    from paper_1810_03931_gb300 import odegpu as G
    from paper_1810_03931_gb300.sweeps import MODEL_DIMS as DIMS
    from paper_1810_03931_gb300.sweeps import params as sweep_params
    from paper_1810_03931_gb300.sweeps import settings_for

    B.build()
    G.load(build_if_missing=False)
    torch.cuda.set_device(0)
    caps = {W.DUFFING: 1 << 18, W.VALVE: 1 << 18, W.KELLER_MIKSIS: 1 << 18}
    base = {W.DUFFING: W.duffing_rkck(1, 1, 0, 1), W.VALVE: W.valve(1, 0, 1),
            W.KELLER_MIKSIS: W.keller_miksis(1, 1, 0, 1)}

    def server():
        srv = G.ode_server_create(0, 8 << 30, args.slice_periods)
        for m, w in base.items():
            G.ode_server_add_model(srv, settings_for(w), w["h0"], caps[m])
        return srv

    reqs = W.serving_mix(args.requests, rate=1.0, max_log2_size=args.max_log2_size,
                         max_log2_h=args.max_log2_horizon)
    inputs = []
    for r in reqs:
        w = W.request_inputs(r)
        p = sweep_params(w)
        inputs.append((np.ascontiguousarray(w["td"]), np.ascontiguousarray(w["y0"]), np.ascontiguousarray(p)))

    stats = []

    def drive(arrivals):
        """Server: submit request k at arrivals[k] s; returns (makespan, latencies, steps)."""
        srv = server()
        try:
            t0 = time.perf_counter()
            open_t, lat, steps = {}, [], 0
            k = 0
            while k < len(reqs) or open_t:
                now = time.perf_counter() - t0
                while k < len(reqs) and arrivals[k] <= now:
                    r = reqs[k]
                    td, y0, p = inputs[k]
                    t = G.ode_server_submit(srv, r["model"], r["horizon"], td, y0, p)
                    open_t[t] = k
                    k += 1
                G.ode_server_progress(srv)
                for t in list(open_t):
                    if G.ode_server_poll(srv, t) == 2:
                        j = open_t.pop(t)
                        r = reqs[j]
                        n_sys, _, A, _ = DIMS[r["model"]]
                        res = G.ode_server_result(srv, t, r["size"], n_sys, A)
                        # latency from the scheduled arrival (submit happens at arrival)
                        lat.append(res["latency"])
                        steps += int(res["nacc"].sum())
                if not open_t and k < len(reqs):
                    time.sleep(max(0.0, min(0.01, arrivals[k] - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
            stats.append({m: G.ode_server_stats(srv, m) for m in base})
            return time.perf_counter() - t0, np.array(lat), steps
        finally:
            G.ode_server_destroy(srv)

    service = []  # per-request service times of the plain sequential launches

    def drive_sequential(arrivals):
        """Plain per-sweep FP64 launches, one request at a time in arrival order
        (a queue without batching): its own solver, ode_run_periods, read-back."""
        t0 = time.perf_counter()
        lat, steps = [], 0
        service.clear()
        for k, r in enumerate(reqs):
            now = time.perf_counter() - t0
            if arrivals[k] > now:
                time.sleep(arrivals[k] - now)
            td, y0, p = inputs[k]
            w = base[r["model"]]
            n_sys, P, A, E = DIMS[r["model"]]
            s = G.ode_create(r["model"], w["scheme"], G.ODE_FP64, r["size"], 0)
            try:
                G.ode_set_tolerances(s, np.full(n_sys, w["rtol"]), np.full(n_sys, w["atol"]), w["hmax"],
                                     w["hmin"], w["grow"], w["shrink"])
                G.ode_set_events(s, int(w["events_on"]), np.array(w["evt_dir"][:E], dtype=np.int32),
                                 np.array(w["evt_tol"][:E]), np.array(w["evt_stop"][:E], dtype=np.int32),
                                 w["max_eq"])
                if w["mc"]:
                    G.ode_set_model_constants(s, np.array(w["mc"], dtype=np.float64))
                G.ode_set_time_domain_mode(s, w["td_mode"])
                G.ode_set_launch(s, 128, 0)
                n = r["size"]
                G.ode_linear_set(s, 0, 0, n, n, td=td, y=y0, p=p, acc=np.zeros((A, n)))
                G.ode_run_periods(s, w["h0"], r["horizon"] - 1, 1, None)
                acc_steps = np.zeros(n, dtype=np.int64)
                G.ode_get_status(s, accepted=acc_steps)
                y = np.zeros((n_sys, n))
                G.ode_linear_get(s, 0, 0, n, n, y=y, copy_mode=G.ODE_STATE)
            finally:
                G.ode_destroy(s)
            lat.append(time.perf_counter() - t0 - arrivals[k])
            service.append(time.perf_counter() - t0 - max(arrivals[k], now))
            steps += int(acc_steps.sum())
        return time.perf_counter() - t0, np.array(lat), steps

    def summary(span, lat, steps, lam=None):
        d = {"makespan_s": span, "steps_per_s": steps / span, "p50_latency_s": float(np.percentile(lat, 50)),
             "p99_latency_s": float(np.percentile(lat, 99))}
        if lam is not None:
            d["lambda_req_per_s"] = lam
        return d

    def fifo(arrivals):
        """The plain sequential queue under an arrival process, from the
        measured service times (a single server taking requests in arrival
        order: finish_k = max(arrival_k, finish_k-1) + service_k)."""
        fin, lat = 0.0, []
        for k in range(len(reqs)):
            fin = max(arrivals[k], fin) + svc[k]
            lat.append(fin - arrivals[k])
        return fin, np.array(lat), steps_seq

    def progress(tag, d):
        # partial results on stderr, so that a run cut short still reports
        print("serving %s: %s" % (tag, json.dumps(d)), file=sys.stderr, flush=True)

    # both forms on the whole mix submitted at once
    span_srv, lat_srv, steps_srv = drive([0.0] * len(reqs))
    progress("served closed batch", summary(span_srv, lat_srv, steps_srv))
    span_seq, lat_seq, steps_seq = drive_sequential([0.0] * len(reqs))
    svc = list(service)
    progress("plain closed batch", dict(summary(span_seq, lat_seq, steps_seq), service_s=[round(x, 3) for x in svc]))
    capacity = len(reqs) / (span_srv if args.load_basis == "served" else span_seq)
    out = {"closed_batch": {"plain_sequential": summary(span_seq, lat_seq, steps_seq),
                            "served": summary(span_srv, lat_srv, steps_srv)},
           "capacity_req_per_s": capacity, "load_basis": args.load_basis,
           "plain_sequential_under_load": "measured" if args.plain_measured else
           "FIFO queue of the service times measured in the closed batch"}
    unit_arrivals = np.array([r["arrival"] for r in reqs])  # rate 1 request/s
    for frac in args.load_fracs:
        lam = frac * capacity
        arr = list(unit_arrivals / lam)
        a = summary(*(drive_sequential(arr) if args.plain_measured else fifo(arr)), lam)
        b_ = summary(*drive(arr), lam)
        out["load_%.2f" % frac] = {"plain_sequential": a, "served": b_}
        progress("load %.2f" % frac, out["load_%.2f" % frac])
    line = {"metric": "serving: accepted system-steps/s and p50/p99 request latency",
            "value": steps_srv / span_srv, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "serving mix: Poisson stream over Duffing / Keller-Miksis / valve sweeps",
                       "requests": len(reqs), "sizes": "floor(2^U(0,%d))" % args.max_log2_size,
                       "horizons": "floor(2^U(4,%d)) periods" % args.max_log2_horizon,
                       "residency_quantum_periods": args.slice_periods,
                       "arrival_rates": "fractions of the %s capacity" % args.load_basis,
                       "pool_capacity": {"duffing": caps[W.DUFFING], "valve": caps[W.VALVE],
                                         "keller_miksis": caps[W.KELLER_MIKSIS]}},
            "serving": out,
            "server_counters": [{W_NAMES[m]: v for m, v in st.items()} for st in stats]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="duffing_rkck",
                    choices=["duffing_rkck", "duffing_rk4", "valve", "keller_miksis", "duffing_lyapunov",
                             "keller_miksis_collapse", "keller_miksis_dual", "valve_paper", "serving"])
    ap.add_argument("--requests", type=int, default=40, help="serving: requests per run")
    ap.add_argument("--slice-periods", type=int, default=0,
                    help="serving: residency quantum in periods (0 = a thread keeps a system to its end)")
    # the full mix (sizes to 2^16, horizons to 1024 periods) takes about an
    # hour per pass; the default is a bounded mix that keeps the run to minutes
    ap.add_argument("--max-log2-size", type=int, default=14, help="serving: sizes floor(2^U(0, x))")
    ap.add_argument("--max-log2-horizon", type=int, default=8, help="serving: horizons floor(2^U(4, x))")
    ap.add_argument("--load-fracs", type=float, nargs="*", default=[0.5, 0.8, 1.0])
    ap.add_argument("--load-basis", default="served", choices=["served", "plain"],
                    help="serving: arrival rates as fractions of the served or the plain sequential capacity")
    ap.add_argument("--plain-measured", action="store_true",
                    help="serving: run the plain sequential launches under each load instead of "
                         "queueing their measured service times")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32rhs"])
    ap.add_argument("--persistent", type=int, default=1)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--systems-per-thread", type=int, default=1, help="with --no-autotune (per-sweep launch)")
    ap.add_argument("--slices-per-launch", type=int, default=0, help="with --no-autotune (0 = all in one)")
    ap.add_argument("--warp-sync", type=int, default=0, help="with --no-autotune: warp-synchronous slices")
    ap.add_argument("--tune-slices", type=int, default=None,
                    help="autotuner trial length in slices (default 16 for Duffing sweeps, 4 otherwise)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch from an ncu capture of the same kernel (null if unknown)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--order", default="grid", choices=["grid", "shuffled", "clustered"],
                    help="system order: parameter grid, seeded shuffle, or shuffle then ode_cluster_order")
    ap.add_argument("--n-transient", type=int, default=None, help="override (profiling runs)")
    ap.add_argument("--n-record", type=int, default=None, help="override (profiling runs)")
    ap.add_argument("--systems", type=int, default=None, help="first N systems of the sweep (profiling runs)")
    args = ap.parse_args()
    if args.tune_slices is None:
        # the schedule choices (split, warp-synchronous slices) show over many
        # slices; a Duffing slice is short, the other models' are long
        args.tune_slices = 16 if args.workload in ("duffing_rkck", "duffing_rk4") else 4
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
