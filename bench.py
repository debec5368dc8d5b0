#!/usr/bin/env python
"""Benchmark of the two-phase GPE step (flow TVD-RK3 + Cahn-Hilliard RK4) on GB300.

Workload: the 3D buoyant bubble, 256 x 256 x 512 cells (33.5M), FP32, no-slip
walls, D3Q15 isotropic stencils, RK4 for the CH equation; synthetic, seeded.
A step is one full time step of the method over the whole grid; the metric is
cell-updates/s = cells x steps / time.  The state (about 2.7 GB) is far
larger than L2, so no flush is needed between steps.

Arms:
  default            the CUDA library through its C ABI, inputs resident in HBM
                     (value), plus the end-to-end number through the same
                     API with host buffers copied in and out every step (e2e),
                     the live roofline of the dominant kernel and the CPU
                     oracle timed on a bounded sample (cpu_baseline).
  --impl reference   the CPU FP64 oracle on the host cores, a bounded sample
                     per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
value is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_00814_gb300 import inputs  # noqa: E402

METRIC = "cell-updates/s (RK3 step)"
# the fraction of the HBM roofline the bubble's dominant kernel is aimed at
TARGET_FRAC = 0.70
UNIT = "cell-updates/s"
WORKLOAD = "3D buoyant bubble 256x256x512 FP32 (no-slip walls, D3Q15, RK4 CH)"

# algorithmic words per cell of each launch kind in the 3D FP32 step, reads +
# writes of one pass: flow stage 1 reads p, u, v, w, phi and mu and writes
# p, u, v, w (6 + 4); stages 2 and 3 also read the four fields of q^n (10 + 4),
# and stage 3 writes u^n + u^{n+1} on the three faces (10 + 7); CH stage 1
# reads the three face sums, phi^n and mu and writes uhat, acc and phi_1
# (5 + 5), stages 2 and 3 read uhat, phi^n, acc, the stage phi and mu and write
# acc and phi (7 + 2), stage 4 writes phi only (7 + 1); the mu sweep reads phi
# and writes mu (1 + 1)
WORDS = {"flow_stage1": 10, "flow_stage2": 14, "flow_stage3": 17, "ch_stage": None, "mu": 2}
CH_WORDS_RK4 = [10, 9, 9, 8]  # CH stage 1 (builds uhat from the face sums), 2, 3, 4


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    for f in ("flow.cu", "flow_ops.cuh", "ring3d.cuh", "tma.cuh", "gpe2p_dev.cuh", "gpe2p_launch.h"):
        with open(os.path.join(ROOT, "paper_2011_00814_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "flow_stage_bubble3d_traffic.json")
    try:
        with open(p) as fh:
            t = json.load(fh)
        if t.get("source_sha") == source_hash():
            return float(t["bytes_per_launch_full_grid"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seconds=15.0, n=64):
    """The CPU oracle, as it stands, on a bounded sample of the workload: the
    same bubble physics in an n^3 closed box (bubble radius n/4), FP64."""
    import oracle
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    prm, f = inputs.bubble3d(n, n, n, R=n / 8.0, gap=n / 8.0)
    st = oracle.init_state(prm, f["phi"], w=f["w"])
    t0 = time.perf_counter()
    st = oracle.step(prm, st, 1)
    t1 = time.perf_counter()
    steps = 1
    more = int(max(0, (seconds - (t1 - t0)) / max(t1 - t0, 1e-3)))
    if more:
        st = oracle.step(prm, st, more)
        steps += more
    el = time.perf_counter() - t0
    return {"value": n ** 3 * steps / el, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{n}^3 closed box, same bubble physics, FP64 oracle, {steps} step(s) in {el:.1f} s"}


def measure_batch2d(stream, steps=20, warmup=3, n=96):
    """The batched 2D workload (96 uneven drops and bubbles, FP32): aggregate
    cell-updates/s of the batch (autotuned persistent or per-sweep form, one
    graph per step) against a loop that steps each instance through its own
    single-problem handle on the same stream."""
    import torch
    from paper_2011_00814_gb300 import gpe2p
    prms, fields = inputs.batch_instances(n=n, seed=0, precision=32)
    cells = sum(p["nx"] * p["ny"] for p in prms)
    out = {"workload": f"{n} uneven 2D drops/bubbles (sides 64-512), FP32, TVD-RK2 CH", "cells": cells}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with gpe2p.Batch(prms, stream=stream.cuda_stream) as b:
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        for _ in range(warmup):
            b.step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            b.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["batched"] = {"cell_updates_per_s": cells / (ms / 1e3), "ms_per_step": ms, **b.config()}
        out["batched"]["tile"] = list(out["batched"]["tile"])
    solvers = []
    try:
        for p, f in zip(prms, fields):
            s = gpe2p.Solver(p, stream=stream.cuda_stream)
            s.init_fields(f)
            solvers.append(s)
        for _ in range(warmup):
            for s in solvers:
                s.step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            for s in solvers:
                s.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["loop"] = {"cell_updates_per_s": cells / (ms / 1e3), "ms_per_step": ms}
    finally:
        for s in solvers:
            s.close()
    out["speedup"] = out["batched"]["cell_updates_per_s"] / out["loop"]["cell_updates_per_s"]
    peak, _ = load_peaks()
    gbs = 49 * 4 * out["batched"]["cell_updates_per_s"] / 1e9
    out["step_algorithmic_gbs"] = gbs
    out["step_frac"] = gbs / peak
    return out


def measure_axisym(stream, steps=400, warmup=5):
    """The axisymmetric falling drop at the paper's resolution (50 cells per
    radius, 400 x 1200 cells, Eo = 144, Oh = 0.0466): cell-updates/s of full
    steps in FP32 and FP64, device-timed on the solver's stream.  The state (~25 MB) stays in
    L2, so no HBM roofline applies; the step is bound by launch and load
    latency."""
    import torch
    from paper_2011_00814_gb300 import gpe2p
    out = {"workload": "axisymmetric falling drop 400x1200 (r x z), TVD-RK2 CH, D2Q9"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for prec in (32, 64):
        prm, f = inputs.falling_drop(precision=prec)
        cells = prm["nx"] * prm["ny"]
        with gpe2p.Solver(prm, stream=stream.cuda_stream) as s:
            s.init_fields(f)
            for _ in range(warmup):
                s.step()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                s.step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            d = s.diagnostics()
        out[f"fp{prec}"] = {"cell_updates_per_s": cells / (ms / 1e3), "ms_per_step": ms, "steps": steps,
                            "nan": d["nan_flag"]}
    out["cells"] = cells
    return out


def measure_static_drop(stream, steps=2000, settled=8000):
    """The 64 x 64 static drop (R = 16, density and viscosity ratio 10, FP64 on
    the GPU): after `steps` steps, the pressure jump of the stored p and of
    P = p + sigma phi mu (the pressure of the equivalent mu grad phi form,
    which carries the Laplace jump) between the inner disc r < R/2 and the
    outer band r > R + 8, against sigma / R_eff with R_eff the radius of the
    phi > 0 area; the relative drift of the phi integral, in the paper's
    advective CH form and in the conservative variant; and the largest
    spurious velocity, also as a fraction of the capillary velocity
    sigma / eta_L.  The same jump after `settled` steps, once the slow
    transient has decayed."""
    import torch
    from paper_2011_00814_gb300 import gpe2p
    prm, f = inputs.static_drop()
    n = prm["nx"]
    x, y = inputs.cell_centres(prm)
    r = np.hypot(x - n / 2.0, y - n / 2.0)
    inner, outer = r < 8.0, r > 24.0
    abs0 = float(np.sum(np.abs(f["phi"]))) * prm["dx"] ** 2
    Uc = prm["sigma"] / prm["etaL"]

    def jump(out):
        R_eff = math.sqrt(float(np.sum(out["phi"] > 0)) / math.pi)
        P = out["p"] + prm["sigma"] * out["phi"] * out["mu"]
        dp = float(np.mean(out["p"][inner]) - np.mean(out["p"][outer]))
        dP = float(np.mean(P[inner]) - np.mean(P[outer]))
        lap = prm["sigma"] / R_eff
        return {"R_eff": R_eff, "sigma_over_R_eff": lap, "dp": dp, "dP": dP, "dP_over_laplace": dP / lap,
                "dp_over_laplace": dp / lap, "within_2pct": abs(dP / lap - 1.0) <= 0.02}

    res = {"workload": "static drop 64x64 periodic, R=16, FP64, density/viscosity ratio 10, 2000 steps",
           "U_c": Uc}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for form in (0, 1):
        with gpe2p.Solver(dict(prm, precision=64, ch_advection=form), stream=stream.cuda_stream) as s:
            s.init_fields(f)
            d0 = s.diagnostics()
            e0.record(stream)
            s.advance(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            out = s.read_fields()
            d = s.diagnostics()
            row = {"int_phi_drift": abs(d["int_phi"] - d0["int_phi"]) / abs0,
                   "max_spurious_u": float(max(np.max(np.abs(out["u"])), np.max(np.abs(out["v"])))),
                   "ms_per_step": e0.elapsed_time(e1) / steps}
            row["max_spurious_u_over_Uc"] = row["max_spurious_u"] / Uc
            if form == 0:
                row.update(jump(out))
                s.advance(settled - steps)
                row["settled"] = dict(jump(s.read_fields()), steps=settled)
            res["advective" if form == 0 else "conservative"] = row
    return res


def measure_fp_rates():
    """The measured multiply-add rates of the device in FP64 and FP32
    (gpe2p_fma_rate), the bound of the FP64 path."""
    from paper_2011_00814_gb300 import gpe2p
    out = {}
    for prec in (64, 32):
        r = gpe2p.fma_rate(prec)
        out[f"fp{prec}_tflops"] = r["flops_per_s"] / 1e12
    # the surrogate convolutions' bound: tcgen05.mma cycles per MMA of one SM
    # (M = 128, K = 16) at their N, with the two issuing CTAs per SM they run
    # with, and at N = 256 (the tensor pipe's own rate)
    mma = {}
    for n, k in ((32, 2), (64, 2), (128, 2), (256, 1)):
        c = gpe2p.mma_rate(n, k)
        mma[f"n{n}_issuers{k}"] = {"cycles_per_mma": c, "mac_per_cycle_per_sm": 128 * n * 16 / c}
    out["tcgen05_mma"] = mma
    return out


def cpu_baseline_axisym(steps=2):
    """The CPU oracle on a two-step sample of the axisymmetric falling drop."""
    import oracle
    prm, f = inputs.falling_drop()
    st = oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"])
    t0 = time.perf_counter()
    oracle.step(prm, st, steps)
    sec = time.perf_counter() - t0
    return {"value": prm["nx"] * prm["ny"] * steps / sec, "unit": UNIT, "kind": "oracle",
            "sample": f"falling drop 400x1200, {steps} steps", "cores": int(os.environ.get("OMP_NUM_THREADS", 1))}


SURROGATE_WEIGHTS = os.path.join(ROOT, "paper_2011_00814_gb300", "data", "unet_two_drops_256.npz")


def measure_surrogate(cases=(0, 1, 2, 3), calls=64):
    """The learned surrogate on held-out two-drop problems (256 x 256, K = 64
    steps per call, 64 calls = 4096 steps): time to solution of the
    controller (network calls with a solver check every 4th call: phi L2 of
    the call <= 2e-2 and its interface displacement within the tolerance
    calibrated on other held-out problems) against the plain
    FP32 solver on the same stream, the final phase errors against the
    solver, the same with the network replaced by persistence (the method
    without the network), and the network's forward throughput against the
    BF16 tensor peak."""
    import torch
    from paper_2011_00814_gb300 import surrogate as S
    if not os.path.exists(SURROGATE_WEIGHTS):
        return {"unavailable": "no trained weights file"}
    sur = S.Surrogate.load(SURROGATE_WEIGHTS, max_batch=8)
    cal = sur.calibration or {}
    out = {"workload": "two drops, periodic 256x256, FP32, K=64 steps per call, 64 calls (4096 steps), "
                       "check every 4th call",
           "check_tol": sur.check_tol,
           "check_tol_disp_cells": sur.check_tol_disp,
           "check_tol_source": (f"phi L2 tolerance {sur.check_tol} as configured; interface-displacement "
                                f"tolerance calibrated on {cal.get('cases')} held-out problems (seeds "
                                f"{cal.get('seeds')}), margin {cal.get('margin')}") if cal else "defaults",
           "bars": {"phi_l2": S.BAR_PHI_L2, "interface_cells": S.BAR_INTERFACE},
           "cases": []}
    for c in cases:
        prm, f = inputs.two_drops(50000 + c)
        row = {"case": c, "r_rho": prm["r_rho"]}
        for key, pers in (("network", False), ("persistence", True)):
            r = S.compare_to_solver(sur, prm, f, calls=calls, repeats=2, persistence=pers)
            r["stats"].pop("check_l2", None)
            row[key] = r
        out["cases"].append(row)

    def summary(key):
        rs = [row[key] for row in out["cases"]]
        return {"speedup": statistics.mean(r["speedup"] for r in rs),
                "phi_l2_max": max(r["phi_l2"] for r in rs),
                "interface_max_cells": max(r["interface_max"] for r in rs),
                "interface_mean_cells": max(r["interface_mean"] for r in rs),
                "phi_l2_of_change": statistics.mean(r["phi_l2_of_change"] for r in rs),
                "check_failures": sum(r["stats"]["failures"] for r in rs),
                "meets_bars_every_case": all(r["meets_bars"] for r in rs)}
    out["network"] = summary("network")
    out["persistence"] = summary("persistence")
    # the speedup of the default (calibrated) configuration, if it meets both bars on every case
    out["speedup_at_tolerance"] = out["network"]["speedup"] if out["network"]["meets_bars_every_case"] else None
    # network forward, batch 8 and 1, inference (BF16 tensor cores)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    for B in (8, 1):
        x = torch.randn(B, sur.n, sur.n, S.NCH, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            sur.forward(x, y, B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 20
        e0.record(sur.torch_stream)
        for _ in range(n):
            sur.forward(x, y, B)
        e1.record(sur.torch_stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        tf = sur.flops(B) / (ms / 1e3) / 1e12
        out["forward" if B == 8 else "forward_batch1"] = {
            "batch": B, "ms": ms, "gflop": sur.flops(B) / 1e9,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_kind": kind}}
    sur.close()
    return out


def max_over_ranks(ms, dist, device):
    """The timed region of the job: the slowest rank's milliseconds (every
    rank gets the same number), then a barrier."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(world, ncell, steps, ms):
    """Whole-job cell-updates/s: every rank steps its own replica of ncell
    cells, so the job processes world * ncell * steps cell-updates in ms."""
    return world * ncell * steps / (ms / 1e3)


def dist_setup(n_gpus):
    if n_gpus <= 1 and "WORLD_SIZE" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, dist


def run_reference(args):
    rank, world, dist = 0, 1, None
    if "WORLD_SIZE" in os.environ and int(os.environ["WORLD_SIZE"]) > 1:
        if int(os.environ.get("RANK", 0)) != 0:
            return 0
    import oracle
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    # size one step's sample so that warmup + steps end within about 2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = 8
    for cand in (64, 48, 32, 24, 16, 12, 8):
        if cand ** 3 / 6.0e5 <= budget:
            n = cand
            break
    prm, f = inputs.bubble3d(n, n, n, R=n / 8.0, gap=n / 8.0)
    st = oracle.init_state(prm, f["phi"], w=f["w"])
    for _ in range(args.warmup):
        st = oracle.step(prm, st, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = oracle.step(prm, st, 1)
    el = time.perf_counter() - t0
    val = n ** 3 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{n}^3 closed box per step"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": f"{n}^3 closed box, same bubble physics, FP64"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 2D measurement")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate measurement")
    ap.add_argument("--no-axisym", action="store_true", help="skip the axisymmetric falling-drop measurement")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2011_00814_gb300 import build, gpe2p

    rank, world, dist = dist_setup(args.gpus)
    dev = torch.cuda.current_device()
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    gpe2p.lib()

    prm, f = inputs.bubble3d()
    prm = dict(prm, precision=32)
    ncell = prm["nx"] * prm["ny"] * prm["nz"]
    stream = torch.cuda.Stream()
    solver = gpe2p.Solver(prm, stream=stream.cuda_stream)
    solver.init_fields(f)

    # live per-launch timing of eager steps (CUDA events on the handle's stream)
    prof = solver.profile_steps(args.profile_steps)
    names = [n for n, _ in prof]
    launches_per_step = len(prof)

    for _ in range(args.warmup):
        solver.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = None
    with ClockSampler(gpu_id) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            solver.step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    d = solver.diagnostics()
    value = job_value(world, ncell, args.steps, ms)

    # end to end through the public API: pinned host inputs in, state out, every step
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in f.items()}
    outb = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory().numpy() for k, v in f.items()}
    lib = gpe2p.lib()
    dptr = gpe2p._dptr
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        solver._check(lib.gpe2p_init_fields(solver.h, dptr(pin["phi"]), dptr(pin["u"]), dptr(pin["v"]),
                                            dptr(pin["w"]), dptr(pin["p"])))
        solver.step()
        solver._check(lib.gpe2p_read_fields(solver.h, dptr(outb["phi"]), dptr(outb["u"]), dptr(outb["v"]),
                                            dptr(outb["w"]), dptr(outb["p"]), None))
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, dist, "cuda")
    e2e_val = job_value(world, ncell, args.e2e_steps, e2e_ms)
    solver.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (the flow stage with the q^n combine)
    peak, peak_kind = load_peaks()
    by_name = {}
    for n, t in prof:
        by_name.setdefault(n, []).append(t)
    step_ms = sum(t for _, t in prof)
    share = {n: sum(v) / step_ms for n, v in by_name.items()}
    dom = "flow_stage2"
    dom_ms = statistics.mean(by_name["flow_stage2"] + by_name["flow_stage3"])
    # the mean launch of stages 2 and 3: mean algorithmic bytes over mean time
    dom_bytes = (WORDS["flow_stage2"] + WORDS["flow_stage3"]) / 2 * 4 * ncell
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    words_step = (WORDS["flow_stage1"] + WORDS["flow_stage2"] + WORDS["flow_stage3"] + sum(CH_WORDS_RK4)
                  + 4 * WORDS["mu"])
    step_gbs = words_step * 4 * ncell / (ms / args.steps / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": ncell, "precision": "fp32", "ch_scheme": "RK4",
                   "iso": "D3Q15", "l2": "state ~2.7 GB > L2 (no flush needed)",
                   "parallelism": f"{world} independent replica(s)"},
        "roofline": {"bound": "hbm", "kernel": "flow3d_kernel<float,2,4,1> (RK3 stages 2 and 3)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": stored_traffic(),
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "step_algorithmic_gbs": step_gbs, "step_frac": step_gbs / peak,
                     "target_frac": TARGET_FRAC, "gap_to_target": TARGET_FRAC - achieved / peak,
                     "shares": {k: round(v, 4) for k, v in share.items()}},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 5 * 8 * ncell,
                "d2h_bytes_per_step": 5 * 8 * ncell, "steps": args.e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "diag": {"int_phi": d["int_phi"], "umax": d["umax"], "nan": d["nan_flag"]},
    }
    if world == 1:
        line["fp_rates"] = measure_fp_rates()
        line["static_drop"] = measure_static_drop(stream)
    if not args.no_batch:
        line["batch2d"] = measure_batch2d(stream)
    if not args.no_axisym and world == 1:
        line["axisym"] = measure_axisym(stream)
    if not args.no_surrogate and world == 1:
        line["surrogate"] = measure_surrogate()
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline()
        if not args.no_axisym:
            line["cpu_baseline"]["axisym"] = cpu_baseline_axisym()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
