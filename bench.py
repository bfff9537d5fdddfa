#!/usr/bin/env python3
"""Benchmark of one coarse step of the nested-mesh solver on GB300.

Workload (default): the precision configuration, the largest single-GPU one: 5
nested levels of 128^3 cells (10.5 M cells), ratio 2, coarse box [-16,16]^3, Mach
1.2 wind, GM=0.01, chi=1, Gaussian luminosity L_c.  The headline run holds the
state in FP64; the same workload in FP32 state (FP64 force, time step and frontier
flux sums) runs beside it in the same line, with its error against the FP64 run.
A step is one coarse step: the Eq. 55 time-step reduction, the Sec. 3.3 recursion
over all levels (31 level steps), CommFlux/CommUp/CommMean, and the Eq. 18 force.

Metric: cell-updates/s summed over levels (sub-cycles counted).  `value` is timed
with inputs resident in HBM; `e2e` through the C ABI with the state uploaded from
pinned host memory and the force read back every step.  Multi-GPU runs are
independent replicas (weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle (the reference arm) on whole coarse steps
of the same workload.
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

import numpy as np  # noqa: E402

from paper_1812_03191_gb300 import inputs as I  # noqa: E402

METRIC = "cell-updates/s"
UNIT = "cell-updates/s"
# FP64 state: stored as double-float pairs whose values are doubles of at most 47
# significant bits; the stencils compute in double-float on the FP32 pipe, the
# reductions, CommMean and the boundary fill in FP64
DTYPE_FP64 = "df64-state(47-bit doubles)/df64-stencils/f64-reductions"


def workload(name):
    if name == "nested":
        return I.nested()
    if name == "single":
        return I.single_mesh()
    if name == "precision":
        return I.precision()
    raise SystemExit(f"unknown workload {name}")


def cell_updates_per_step(cfg):
    n = cfg["n"]
    n3 = n**3 if isinstance(n, int) else n[0] * n[1] * n[2]
    return sum(n3 * 2**l for l in range(cfg["n_levels"]))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- algorithmic bytes
# Arrays each stencil kernel reads + writes once per element of its box (the
# compulsory traffic of the kernel as designed, neighbour reuse assumed cached).
ARRAYS_PER_ELEM = {
    "source": 12,        # rho, e, phi, v3 -> v3, pi3
    "compress_lum": 8,   # e, v3, rho, lumw -> e, e/rho
    "diffuse": 4,        # rho, e/rho, e -> e (+1 before separate transport kernels: the
                         # x sweep's e/rho, whose preparation kernel then is not launched)
    "tprep": 9,          # rho, e, pi3 -> e/rho, w3: the y and z sweeps' (the workloads
                         # all diffuse, so the x sweep's comes from the diffusion)
    "tflux": 5,          # rho, e/rho, v_d -> F, E
    "tmom": 8,           # w3, F, v_d -> P3
    "tupdate": 15,       # F, E, P3, rho, e, pi3 -> rho, e, pi3
    "vrec_source": 9,    # rho, e, phi, pi3 -> v3 (after fused sweeps also -> rho, e)
    "sweep": 11,         # fused sweep: rho, e, pi3, v_d -> rho, e, pi3
}



# DRAM bytes (read + write) per box element of a launch, from the ncu captures in
# profiles/ (k_sweep_fused_precision_5x128_fp32.md: fused sweeps, 144^3 box,
# 80.2 / 99.5 / 85.0 MB; k_tmom_df64_nested_3x64.md: double-float momentum fluxes, 80^3
# box, 20.09 / 20.09 / 13.47 MB, a smaller case of the same kernel, whose traffic
# grows with the box); `traffic` scales them to the mean box of the timed launches.
# A kernel without a capture of its current code reports null.
_TMOM_DF64 = (20.0865e6 + 20.0840e6 + 13.4705e6) / 3 / 80**3
TRAFFIC_PER_ELEM = {("precision_5x128^3", 4, "sweep"): (80.2e6 + 99.5e6 + 85.0e6) / 3 / 144**3,
                    ("precision_5x128^3", 8, "tmom"): _TMOM_DF64,
                    ("nested_3x64^3_fp64", 8, "tmom"): _TMOM_DF64}


def level_step_boxes(cfg):
    """box elements of every level step of one coarse step (level 0: margin 4, one
    more element on the upper side; finer levels: first sub-cycle margin 8, second
    margin 4; capped at the array)."""
    n, G = cfg["n"], cfg["G"]
    out = [min(n + 9, n + 2 * G) ** 3]
    for l in range(1, cfg["n_levels"]):
        out += [min(n + 2 * m, n + 2 * G) ** 3 for m in (8, 4)] * 2 ** (l - 1)
    return out


def bytes_per_launch(cfg, kind, esz, fused=False):
    boxes = level_step_boxes(cfg)
    n, G = cfg["n"], cfg["G"]
    if kind in ARRAYS_PER_ELEM:
        arrays = ARRAYS_PER_ELEM[kind] + (2 if fused and kind == "vrec_source" else 0)
        arrays += 1 if kind == "diffuse" and not fused else 0
        return arrays * esz * sum(boxes) / len(boxes)
    if kind == "commup":  # write every fine ghost element, read each coarse host once
        return 5 * esz * (((n + 2 * G) ** 3 - n**3) + (n // 2 + G + 2) ** 3)
    if kind == "commmean":  # read 8 fine cells / 4 faces, write the covered coarse cell
        return 5 * esz * (n**3 + (n // 2) ** 3)
    return None


def kernel_hbm_table(cfg, kinds, esz, fused, peak):
    """Algorithmic HBM bandwidth of every timed kernel kind with a byte count: bytes
    per launch (ARRAYS_PER_ELEM over the mean box) / mean event-timed launch, and its
    fraction of the peak."""
    out = {}
    for kind, (ms, n) in kinds.items():
        bpl = bytes_per_launch(cfg, kind, esz, fused)
        if bpl is None or not n or ms <= 0:
            continue
        gbs = bpl / (ms / n / 1e3) / 1e9
        out[kind] = {"gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
    return out


def job_time_ms(ms, dist, device):
    """The job's timed-region duration: the slowest rank's (replicas run independent
    runs; the only collective is this reduction, outside the timed region)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step, steps, world, ms):
    """whole-job throughput: the units every rank processed / the job's time"""
    return units_per_rank_step * steps * world / (ms / 1e3)


def tile_summary(shapes):
    """{op: [shape of x, y, z sweep]} for the ops whose tuned shape is not flat"""
    if shapes is None:
        return "flat"
    from paper_1812_03191_gb300 import binding
    return {binding.OP_NAMES[o]: row for o, row in enumerate(shapes) if any(row)}


def cpu_oracle_rate(cfg, budget_s, steps_cap=None, omp=False):
    """Oracle cell-updates/s on a bounded sample: whole coarse steps until budget
    (omp: the OpenMP build of the oracle on every host core)."""
    from oracle import Oracle
    lo, hi = cfg["lo"], cfg["hi"]
    orc = Oracle(cfg["n_levels"], cfg["n"], lo, hi, cfg["G"], cfg["params"], omp=omp)
    cu = cell_updates_per_step(cfg)
    done = 0
    t0 = time.perf_counter()
    while True:
        orc.step(1)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (steps_cap and done >= steps_cap):
            break
    orc.close()
    return cu * done / el, done, el


def oracle_openmp_rate(cfg, budget_s):
    """The same oracle loops on every host core (its OpenMP build, bitwise the plain
    build's results; sums stay serial), or why that build is unavailable."""
    try:
        import oracle
        oracle.build_oracle(omp=True)
        cores = oracle.threads(os.cpu_count() or 1)
    except Exception as exc:  # a host compiler without OpenMP
        return {"unavailable": f"{type(exc).__name__}: {exc}".splitlines()[0][:200]}
    rate, nsteps, el = cpu_oracle_rate(cfg, budget_s, omp=True)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle (OpenMP build)",
            "sample": f"{nsteps} whole coarse steps of {cfg['name']} ({el:.1f} s, "
                      f"{cores} threads, plane loops in parallel, sums serial)"}


def run_reference(args, cfg):
    """The reference arm: the FP64 oracle timed on whole coarse steps of the workload,
    on the host cores.  The precision workload (6.5e7 cell-updates per coarse step,
    about 25 s single-threaded) runs on the oracle's OpenMP build, bitwise the plain
    build's results, so that W + K steps end within a few minutes; the smaller
    workloads run single-threaded."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cu = cell_updates_per_step(cfg)
    from oracle import Oracle
    omp = cfg["name"].startswith("precision")
    cores = 1
    if omp:
        import oracle
        cores = oracle.threads(os.cpu_count() or 1)
    orc = Oracle(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"], cfg["params"],
                 omp=omp)
    for _ in range(args.warmup):
        orc.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.step(1)
        times.append(time.perf_counter() - t0)
    orc.close()
    tot = sum(times)
    value = cu * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the FP64 workload of the GPU arm's line, named as that line names it
        "config": {"workload": cfg["name"].replace("_fp64", "") + "_fp64",
                   "n_levels": cfg["n_levels"], "n": cfg["n"],
                   "box": [cfg["lo"][0], cfg["hi"][0]], "ghost": cfg["G"],
                   "mach": cfg["params"]["mach"], "chi": cfg["params"]["chi"],
                   "luminosity": cfg["params"]["L"], "cell_updates_per_step": cu},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle (OpenMP build)" if omp else "oracle",
                         "sample": f"{args.steps} whole coarse steps of {cfg['name']} "
                                   f"after {args.warmup} warm-up steps, "
                                   + (f"{cores} threads (plane loops in parallel, sums "
                                      f"serial)" if omp else "single-threaded C")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """64 uneven runs in one pool (FP32 state, FP64 reductions), one coarse step of
    every run per step; tiles picked by the pool's autotuner."""
    import torch

    from paper_1812_03191_gb300 import binding
    runs = I.batched()
    cu = sum(r["n"] ** 3 * (2 ** r["n_levels"] - 1) for r in runs)
    if args.impl == "reference":
        return 0
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t_e2e0 = time.perf_counter()
    pool = binding.Pool(64 << 30, precision=binding.DF_FP32_STATE, stream=stream.cuda_stream)
    for r in runs:
        pool.admit(r["n_levels"], r["n"], r["lo"], r["hi"], r["G"], r["params"])
    t_admit = time.perf_counter() - t_e2e0
    tiles = pool.autotune()
    for _ in range(args.warmup):
        pool.step(1)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = pool.info()["launches"]
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            pool.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = pool.info()["launches"] - l0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value = cu * args.steps / (ms / 1e3)
    # per-kernel times (events around every launch) over the same number of steps
    pool.set_timing(True)
    for _ in range(args.steps):
        pool.step(1)
    kinds = {}
    for kind in range(binding.KERNEL_KINDS):
        kms, kn = pool.kernel_time(kind)
        if kn:
            kinds[binding.kernel_name(kind)] = (kms, kn)
    pool.set_timing(False)
    total_k = sum(v[0] for v in kinds.values())
    dom = max((k for k in kinds if k in ARRAYS_PER_ELEM), key=lambda k: kinds[k][0])
    # algorithmic bytes of all launches of that kind in one step, from the runs' boxes
    esz = 4
    per_step_bytes = 0.0
    for r in runs:
        swept = True  # the library's choice for the FP32 state in a pool of several runs
        if (dom == "sweep" and not swept) or (dom in ("tprep", "tflux", "tmom", "tupdate")
                                              and swept):
            continue
        boxes = level_step_boxes(dict(n=r["n"], G=r["G"], n_levels=r["n_levels"]))
        mult = 3 if dom in ("tprep", "tflux", "tmom", "tupdate", "sweep") else 1
        arrays = ARRAYS_PER_ELEM[dom] + (2 if dom == "vrec_source" and swept else 0)
        per_step_bytes += arrays * esz * sum(boxes) * mult
    dom_ms, dom_n = kinds[dom]
    achieved = per_step_bytes * args.steps / (dom_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    # e2e: admission from host parameters, K steps, forces read back every step
    t0 = time.perf_counter()
    pool2 = binding.Pool(64 << 30, precision=binding.DF_FP32_STATE, stream=stream.cuda_stream)
    for r in runs:
        pool2.admit(r["n_levels"], r["n"], r["lo"], r["hi"], r["G"], r["params"])
    pool2.set_tiles(tiles)
    for _ in range(args.steps):
        pool2.step(1)
        pool2.query()
    e2e_s = time.perf_counter() - t0
    q = pool.query()
    # FP32-state error against FP64: the same runs in an FP64 pool, stepped as many
    # coarse steps as the timed pool took (warm-up, timed steps, timing pass)
    n_done = args.warmup + 2 * args.steps
    p64 = binding.Pool(64 << 30, precision=binding.DF_FP64, stream=stream.cuda_stream)
    for r in runs:
        p64.admit(r["n_levels"], r["n"], r["lo"], r["hi"], r["G"], r["params"])
    p64.step(n_done)
    q64 = p64.query()
    p64.close()
    rel = []
    for k, r in enumerate(runs):
        d = np.asarray(r["params"]["flow_dir"], dtype=float)
        f32 = -float(np.dot(q[k, :3], d)) / np.linalg.norm(d)
        f64 = -float(np.dot(q64[k, :3], d)) / np.linalg.norm(d)
        rel.append(abs(f32 - f64) / max(abs(f64), 1e-300))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-state/f64-reductions",
        "data": "synthetic",
        "config": {"workload": "batched_64_runs", "runs": len(runs), "levels": "2..4",
                   "mesh": "{32,48,64,96}^3", "cell_updates_per_step": cu,
                   "l2": "flushed between timed steps; working set 5.6 GB",
                   "tiles_blocks_per_sm": tiles, "admission_s": t_admit},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": peak_kind, "launches_timed": dom_n,
                     "share_of_kernel_time": dom_ms / total_k},
        "cpu_baseline": None,
        "e2e": {"value": cu * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 6 * 8 * len(runs),
                "note": "admission of the 64 runs from host parameters included"},
        "gpu_launches": launches, "clocks": clk.summary(),
        "kernels_ms": {k: round(v[0], 4) for k, v in sorted(kinds.items(), key=lambda x: -x[1][0])},
        "unhealthy_runs": int(np.nansum(q[:, 5])),
        "fp32_state_force_error_vs_fp64": {
            "coarse_steps": n_done, "max_rel": max(rel), "median_rel": float(np.median(rel)),
            "runs": len(rel), "time_equal": bool(np.all(q[:, 3] == q64[:, 3]))},
    }
    print(json.dumps(line), flush=True)
    pool.close()
    pool2.close()
    return 0


def run_precision_compare(args):
    """The precision workload (5 x 128^3, Mach 1.2, L_c) in FP32 state and in FP64,
    K coarse steps each (each computes its own time steps): per-field relative L2
    error of the FP32 state and relative force error against FP64."""
    import torch

    from paper_1812_03191_gb300 import binding
    cfg = I.precision()
    out = {}
    sims = {}
    for prec in (binding.DF_FP64, binding.DF_FP32_STATE):
        sim = binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"],
                          cfg["params"], precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(args.steps)
        F, Fm = sim.force()
        out[prec] = dict(F=F, Fm=Fm, t=sim.status()[0], wall=time.perf_counter() - t0)
        sims[prec] = sim
    errs = {}
    names = ["rho", "e", "vx", "vy", "vz"]
    for f in range(5):
        num = den = 0.0
        for l in range(cfg["n_levels"]):
            a = sims[binding.DF_FP32_STATE].get_field(l, f)
            b = sims[binding.DF_FP64].get_field(l, f)
            pr = cfg["params"]
            e0 = pr["cs"] ** 2 * pr["rho0"] / (pr["gamma"] * (pr["gamma"] - 1))
            V = [pr["mach"] * pr["cs"] * c for c in pr["flow_dir"]]
            base = pr["rho0"] if f == 0 else (e0 if f == 1 else V[f - 2])
            num += float(((a - b) ** 2).sum())
            den += float(((b - base) ** 2).sum())  # relative to the perturbation
        errs[names[f]] = (num / max(den, 1e-300)) ** 0.5
    F64, F32 = out[binding.DF_FP64]["Fm"], out[binding.DF_FP32_STATE]["Fm"]
    cu = cell_updates_per_step(cfg)
    line = {
        "metric": "FP32-state error vs FP64", "value": abs(F32 - F64) / abs(F64),
        "unit": "relative force error", "n_gpus": 1, "steps": args.steps, "warmup": 0,
        "higher_is_better": False, "dtype": "f32-state vs f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "coarse_steps": args.steps},
        "force_along_motion": {"fp64": F64, "fp32_state": F32},
        "time": {"fp64": out[binding.DF_FP64]["t"], "fp32_state": out[binding.DF_FP32_STATE]["t"]},
        "field_rel_l2_error_of_perturbation": errs,
        "cell_updates_per_s": {k: cu * args.steps / v["wall"] for k, v in
                               (("fp64", out[binding.DF_FP64]),
                                ("fp32_state", out[binding.DF_FP32_STATE]))},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_heating_ladder(args):
    """Heating force by differencing (Eq. 5) over a ladder of 4..7 nested levels at
    Mach 3 (Sec. 4.1 set-up): the hot and cold run of every level count in one pool
    (FP32 state, FP64 reductions), stepped to 100 tau; each added level should raise
    the heating force by the Eq. 24 increment (its asymptotic value; the finite
    resolution of Eq. 10-12 lowers it)."""
    import torch

    from paper_1812_03191_gb300 import ladder
    if args.impl == "reference":
        return 0
    torch.cuda.set_device(0)
    with ClockSampler(0) as clk:
        out = ladder.run(levels=(4, 5, 6, 7), sample_every=8)
        low = ladder.low_mach(mach=0.1)
        cold = ladder.cold_thermal(mach=0.1)
        paper = ladder.paper_cold_thermal(n_levels=10)
    pred = out["predicted_increment"]
    ratios = {k: v / pred for k, v in out["increments"].items()}
    line = {
        "metric": "heating-force increment per added level / Eq. 24", "value":
            float(np.mean(list(ratios.values()))), "unit": "ratio", "n_gpus": 1,
        "steps": sum(r["steps"] for r in out["runs"].values()), "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-state/f64-reductions", "data": "synthetic",
        "config": {"workload": "heating_ladder_mach3", "levels": out["levels"], "n": 32,
                   "gamma": 1.4, "GM": 1e-3, "chi": 0.1, "L": 2e-4, "half_width": out["half"],
                   "t_end": out["t_end"]},
        "heating_force_final": {k: r["final"] for k, r in out["runs"].items()},
        "increments": out["increments"], "eq24_increment": pred, "ratios": ratios,
        "low_mach": {"mach": 0.1, "levels": 6, "heating_force": low["runs"][6]["final"],
                     "eq8_times_eq23_share": low["expected"], "ratio": low["ratio"]},
        "cold_thermal_low_mach": {"mach": 0.1, "levels": 6, "force": cold["runs"][6]["final"],
                                  "eq51_times_eq23_share": cold["expected"],
                                  "ratio": cold["ratio"]},
        "cold_thermal_paper_geometry": {
            "mach": 0.1, "levels": 10, "box_half_width": paper["half"],
            "geometry": "quadrant, ground 64x64x128, levels 32x32x64, first over a quarter",
            "force": paper["final"], "eq51_times_eq23_share": paper["expected"],
            "ratio": paper["ratio"], "wall_s": paper["wall_s"]},
        "pool_cell_updates_per_s": out["cell_updates"] / out["wall_s"],
        "wall_s": out["wall_s"], "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Poisson stream of simulation requests through the continuous-batching server
    (FP32 state, FP64 reductions), against the same stream solved one request at a
    time on the same machinery, in FP64 (the plain method) and in FP32 state (so the
    gain of batching shows apart from that of precision).  Same stopping rule and
    step cap for all three.  Requests: levels 2..3 and meshes {24,32}^3 (the
    the benchmark spec's distribution of Mach, chi and luminosity), so that most of them
    converge by the rule within the cap and the latencies are times to a converged
    force; the capped fraction is reported."""
    import torch

    from paper_1812_03191_gb300 import binding
    from paper_1812_03191_gb300 import serve as S
    if args.impl == "reference":
        return 0
    torch.cuda.set_device(0)
    budget = 16 << 30
    sizes, levels = (24, 32), (2, 3)
    # capacity: all requests resident in one pool, cell-updates/s of a few steps
    probe = I.requests(args.requests, 1.0, sizes=sizes, levels=levels)
    cu = [sp["n"] ** 3 * (2 ** sp["n_levels"] - 1) for _, sp in probe]
    pool = binding.Pool(64 << 30, precision=binding.DF_FP32_STATE)
    for _, sp in probe:
        pool.admit(sp["n_levels"], sp["n"], sp["lo"], sp["hi"], sp["G"], sp["params"])
    tiles = pool.autotune()
    pool.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pool.step(200)
    pool.query()
    step_s = (time.perf_counter() - t0) / 200
    pool.close()
    # a request takes about half the cap on average (measured on this distribution)
    capacity = 1.0 / (step_s * 0.5 * args.step_cap / len(probe) * 1.0)
    rate = 0.8 * capacity
    reqs = I.requests(args.requests, rate, sizes=sizes, levels=levels)
    srv = S.Server(budget, precision=binding.DF_FP32_STATE, tol=1e-3, step_cap=args.step_cap,
                   tiles=tiles, keep_history=True)
    with ClockSampler(0) as clk:
        res, summ = srv.run(reqs)
    max_active, batches = srv.max_active, srv.batches
    srv.close()
    seq64, summ64 = S.serve_sequential(reqs, budget, precision=binding.DF_FP64, tol=1e-3,
                                       step_cap=args.step_cap, keep_history=True)
    # one run alone is faster with the separate transport kernels than with the fused
    # sweeps (too few blocks per sweep on these small levels); the FP32 baseline uses
    # them, so that the batching gain is not overstated
    seq32, summ32 = S.serve_sequential(reqs, budget, precision=binding.DF_FP32_STATE, tol=1e-3,
                                       step_cap=args.step_cap,
                                       transport=binding.TRANSPORT_SEPARATE)
    # FP32-state error of each served result against the FP64 run of the same request
    # at the same coarse step
    h64 = {r.rid: r.history for r in seq64}
    errs = []
    for r in res:
        h = h64.get(r.rid)
        if r.error is None and h and r.history:
            k = min(len(h), len(r.history)) - 1
            errs.append(abs(r.history[k] - h[k]) / max(abs(h[k]), 1e-300))
    same_stop = sum(1 for r in res for q in seq64 if q.rid == r.rid and q.steps == r.steps)
    line = {
        "metric": "serving requests/s", "value": summ["throughput_req_per_s"],
        "unit": "requests/s", "n_gpus": 1, "steps": args.requests, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-state/f64-reductions", "data": "synthetic",
        "config": {"workload": f"serving_{args.requests}_requests", "arrival_rate_per_s": rate,
                   "capacity_req_per_s": capacity, "step_cap": args.step_cap, "tol": 1e-3,
                   "levels": list(levels), "mesh": [f"{n}^3" for n in sizes],
                   "budget_bytes": budget, "max_active": max_active, "host_checks": batches,
                   "seed": 1812031911},
        "serving": summ, "sequential_fp64": summ64, "sequential_fp32_state": summ32,
        "throughput_ratio_vs_sequential_fp64":
            summ["throughput_req_per_s"] / summ64["throughput_req_per_s"],
        "throughput_ratio_vs_sequential_fp32_state (batching alone)":
            summ["throughput_req_per_s"] / summ32["throughput_req_per_s"],
        "fp32_state_force_error_vs_fp64": {
            "max_rel": max(errs) if errs else None,
            "median_rel": float(np.median(errs)) if errs else None,
            "requests_compared": len(errs), "same_stopping_step": same_stop},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_paper_hierarchy(args):
    """The paper's cold-thermal-force hierarchy (Sec. 4.2, set up as in Sec. 4.1.1):
    the quadrant domain with mirror planes x = 0 and y = 0, a ground of 64 x 64 x 128
    cells and 11 levels of 32 x 32 x 64, the first over a quarter of the ground,
    l = 3200 lambda, Mach 0.1, chi = 0.1, GM = 1e-3, a cold perturber; xi = 2 on every
    level, so one coarse step is 2^11 finest-level steps.  Graph-replayed coarse
    steps, timed with CUDA events."""
    import torch

    from paper_1812_03191_gb300 import binding
    if args.impl == "reference":
        return 0
    torch.cuda.set_device(0)
    chi, gamma, mach = 0.1, 1.4, 0.1
    half = 3200.0 * chi / (gamma * mach)  # l = 3200 lambda (Eq. 7)
    cfg = I.quadrant(n=64, n_levels=12, half=half, mach=mach, quarter=True, GM=1e-3, chi=chi,
                     L=0.0)
    prec = binding.DF_FP64 if args.precision == "fp64" else binding.DF_FP32_STATE
    stream = torch.cuda.current_stream()
    sim = binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"], cfg["params"],
                      precision=prec, stream=stream.cuda_stream, n0=cfg["n0"])
    n0, n = cfg["n0"], cfg["n"]
    cu = n0[0] * n0[1] * n0[2] + sum(n[0] * n[1] * n[2] * 2**l for l in range(1, 12))
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = sim.kernel_launches()
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = sim.kernel_launches() - l0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    sim.set_timing(True)
    sim.step(1)
    kinds = {}
    for kind in range(binding.KERNEL_KINDS):
        kms, kn = sim.kernel_time(kind)
        if kn:
            kinds[binding.kernel_name(kind)] = (kms, kn)
    sim.set_timing(False)
    F, Fmot = sim.force()
    bad = sim.status()[2]
    line = {
        "metric": METRIC, "value": cu * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_FP64 if prec == binding.DF_FP64 else "f32-state/f64-reductions",
        "data": "synthetic",
        "config": {"workload": "paper_hierarchy_quadrant_64x64x128+11x32x32x64",
                   "n0": n0, "n": n, "n_levels": 12, "half_width": half, "mach": mach,
                   "chi": chi, "GM": 1e-3, "cell_updates_per_step": cu,
                   "l2": "not flushed (the working set, 0.3 GB, is the run itself)"},
        "gpu_launches": launches, "launches_per_step": launches / args.steps,
        # one step with an event pair around every launch (no graph): the shares, not
        # the sum, are comparable with ms_per_step
        "kernels_ms_one_step": {k: round(v[0], 3) for k, v in sorted(kinds.items(),
                                                                   key=lambda x: -x[1][0])},
        "force": {"F": list(F), "F_along_motion": Fmot}, "unhealthy": bad,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def time_sim(sim, cfg, args, stream, flush, local, fused):
    """Autotune (state restored), W warm-up coarse steps, then K graph-replayed coarse
    steps bracketed by CUDA events on the launching stream with the L2 flushed between
    steps; then K more steps with an event pair around every launch (no graph) for
    the per-kernel times.  Returns the measurements."""
    from paper_1812_03191_gb300 import binding
    import torch
    shapes = sim.autotune() if args.tiles == "auto" else None
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = sim.kernel_launches()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = sim.kernel_launches() - l0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    sim.set_timing(True)
    for _ in range(args.steps):
        flush.zero_()
        sim.step(1)
    kinds = {}
    for kind in range(binding.KERNEL_KINDS):
        kms, kn = sim.kernel_time(kind)
        if kn:
            kinds[binding.kernel_name(kind)] = (kms, kn)
    sim.set_timing(False)
    F, Fmot = sim.force()
    return dict(ms=ms, launches=launches, clocks=clk.summary(), kinds=kinds, F=F, Fmot=Fmot,
                shapes=shapes, fused=fused)


# algorithmic bytes per cell-update of a whole level step: the five fields read and
# written once (rho, e, v_x, v_y, v_z)
B_ALG = {8: 80, 4: 40}
# kernels launched once per level step (or per sweep of one), each over one level's
# active cells: the units one launch processes are that level's cells
LEVEL_STEP_KERNELS = ("source", "compress_lum", "diffuse", "tprep", "tflux", "tmom",
                      "tupdate", "vrec_source", "sweep", "frontier_diff")


def roofline_block(cfg, m, cu, esz, peak, peak_kind, fp64_peak=None):
    """Roofline of the dominant level-step kernel and of the whole step on the
    algorithmic bytes per cell-update (B_ALG), plus, for FP64, its FP64-pipe
    roofline against the measured FP64 peak."""
    kinds, ms = m["kinds"], m["ms"] / (m["steps"])
    n = cfg["n"]
    units = n**3 if isinstance(n, int) else int(np.prod(n))  # every level: n^3 cells
    total_k = sum(v[0] for v in kinds.values())
    dom = max((k for k in kinds if k in LEVEL_STEP_KERNELS), key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    avg_s = dom_ms / dom_n / 1e3
    b_alg = B_ALG[esz]
    achieved = b_alg * units / avg_s / 1e9
    boxes_all = level_step_boxes(cfg)
    tpe = TRAFFIC_PER_ELEM.get((cfg["name"], esz, dom))
    traffic = tpe * sum(boxes_all) / len(boxes_all) if tpe is not None else None
    step_gbs = cu * b_alg / (ms / 1e3) / 1e9
    out = {
        "kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
        "algorithmic_bytes_per_launch": b_alg * units,
        "units_per_launch": f"{units} cell-updates (one level step of one {n}^3 level) "
                            f"x {b_alg} B",
        "launches_timed": dom_n, "avg_launch_ms": dom_ms / dom_n,
        "share_of_kernel_time": dom_ms / total_k if total_k else None,
        "step": {"achieved": step_gbs, "frac": step_gbs / peak,
                 "algorithmic_bytes_per_step": cu * b_alg},
    }
    if esz == 8 and fp64_peak:
        # the FP64 state's stencils compute in double-float on the FP32 pipe: the
        # FP64 pipe's measured peak is why, and no longer their bound
        out["fp64_pipe"] = {
            "measured_peak_tflops": fp64_peak["tflops"],
            "stencil_arithmetic": "double-float (float pairs) on the FP32 pipe; the "
                                  "FP64 pipe runs the reductions and inter-level operators"}
    return out


def state_errors(cfg, s32, s64):
    """per-field relative L2 error of the FP32-state perturbation against FP64 over
    every level's active cells, and the relative error of the force along the motion"""
    names = ["rho", "e", "vx", "vy", "vz"]
    pr = cfg["params"]
    e0 = pr["cs"] ** 2 * pr["rho0"] / (pr["gamma"] * (pr["gamma"] - 1))
    V = [pr["mach"] * pr["cs"] * c for c in pr["flow_dir"]]
    errs = {}
    for f in range(5):
        num = den = 0.0
        base = pr["rho0"] if f == 0 else (e0 if f == 1 else V[f - 2])
        for l in range(cfg["n_levels"]):
            a, b = s32.get_field(l, f), s64.get_field(l, f)
            num += float(((a - b) ** 2).sum())
            den += float(((b - base) ** 2).sum())
        errs[names[f]] = (num / max(den, 1e-300)) ** 0.5
    return errs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision",
                    choices=["nested", "single", "precision", "batched", "serving",
                             "precision_compare", "heating_ladder", "paper_hierarchy"])
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--step-cap", type=int, default=6000)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="state precision of the headline run (the precision workload also "
                         "runs the FP32 state beside its FP64 run)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--transport", default="auto", choices=["auto", "separate", "fused"],
                    help="transport kernels: fused sweeps or separate kernels (default: "
                         "the library's choice: fused sweeps for the FP32 state in pools and "
                         "on levels of at least 512 Ki cells)")
    ap.add_argument("--tiles", default="auto", choices=["auto", "flat"],
                    help="tile shapes of the stencil launches: autotuned (before the "
                         "warm-up, untimed) or flat enumeration")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "precision_compare":
        return run_precision_compare(args)
    if args.workload == "heating_ladder":
        return run_heating_ladder(args)
    if args.workload == "paper_hierarchy":
        return run_paper_hierarchy(args)
    cfg = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch

    from paper_1812_03191_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # CPU baseline first (oracle on the host cores, rank 0 only, bounded sample)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, nsteps, el = cpu_oracle_rate(cfg, args.cpu_budget, steps_cap=1)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nsteps} whole coarse step(s) of {cfg['name']} ({el:.1f} s, "
                         f"single-threaded C, -O2)"}
        cpu["openmp"] = oracle_openmp_rate(cfg, args.cpu_budget / 2)

    prec = binding.DF_FP64 if args.precision == "fp64" else binding.DF_FP32_STATE
    both = args.workload == "precision" and prec == binding.DF_FP64
    stream = torch.cuda.current_stream()
    cu = cell_updates_per_step(cfg)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    transport = {"auto": binding.TRANSPORT_AUTO, "separate": binding.TRANSPORT_SEPARATE,
                 "fused": binding.TRANSPORT_FUSED}[args.transport]
    n3 = cfg["n"] ** 3 if isinstance(cfg["n"], int) else int(np.prod(cfg["n"]))
    peak, peak_kind = peaks()

    # measured FP64 peak (the FP64 kernels are bound by the FP64 pipe), clocks sampled
    with ClockSampler(local) as pclk:
        tf, tf_ms = binding.measure_fp64_peak(local, repeats=5)
    fp64_peak = {"tflops": tf, "best_launch_ms": tf_ms, "clocks": pclk.summary()}

    def make(pr):
        sim = binding.Sim(cfg["n_levels"], cfg["n"], cfg["lo"], cfg["hi"], cfg["G"],
                          cfg["params"], precision=pr, device=local, stream=stream.cuda_stream)
        sim.set_transport(transport)
        fused = transport == binding.TRANSPORT_FUSED or (
            transport == binding.TRANSPORT_AUTO and pr == binding.DF_FP32_STATE
            and n3 >= 512 * 1024)  # the library's per-level choice
        return sim, fused

    sim, fused = make(prec)
    if dist:
        dist.barrier()
    m = time_sim(sim, cfg, args, stream, flush, local, fused)
    m["steps"] = args.steps
    if dist:
        dist.barrier()
    ms = job_time_ms(m["ms"], dist, "cuda")
    value = job_value(cu, args.steps, world, ms)
    esz = 8 if prec == binding.DF_FP64 else 4
    roofline = roofline_block(cfg, m, cu, esz, peak, peak_kind, fp64_peak)
    kinds = m["kinds"]

    # the FP32-state run of the same workload beside the FP64 one, the same number of
    # coarse steps (each takes its own time steps), and its error against FP64
    fp32 = None
    if both:
        s32, fused32 = make(binding.DF_FP32_STATE)
        m32 = time_sim(s32, cfg, args, stream, flush, local, fused32)
        m32["steps"] = args.steps
        errs = state_errors(cfg, s32, sim)
        F64, F32 = m["Fmot"], m32["Fmot"]
        fp32 = {
            "value": cu * args.steps / (m32["ms"] / 1e3), "unit": UNIT,
            "ms_per_step": m32["ms"] / args.steps, "dtype": "f32-state/f64-reductions",
            "transport": "fused sweeps" if fused32 else "separate kernels",
            "roofline": roofline_block(cfg, m32, cu, 4, peak, peak_kind),
            "gpu_launches": m32["launches"], "clocks": m32["clocks"],
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(m32["kinds"].items(),
                                                                 key=lambda x: -x[1][0])},
            "kernels_hbm": kernel_hbm_table(cfg, m32["kinds"], 4, fused32, peak),
            "error_vs_fp64": {
                "coarse_steps": args.warmup + 2 * args.steps,
                "force_along_motion_rel": abs(F32 - F64) / abs(F64),
                "force_along_motion": {"fp64": F64, "fp32_state": F32},
                "time": {"fp64": sim.status()[0], "fp32_state": s32.status()[0]},
                "field_rel_l2_error_of_perturbation": errs},
        }
        s32.close()

    # ---- e2e: state from pinned host memory, one step, force back, every step
    nstate = sim.state_size()
    host = torch.empty(nstate, dtype=torch.float64, pin_memory=True)
    st_np, t_now = sim.get_state(host.numpy())
    e2e_times = []
    for k in range(max(3, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_state(st_np, t_now)
        sim.step(1)
        sim.force()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_times) / len(e2e_times)
    e2e = {"value": cu * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nstate * 8,
           "d2h_bytes_per_step": 3 * 8 + 4}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_FP64 if prec == binding.DF_FP64 else "f32-state/f64-reductions",
            "data": "synthetic",
            "config": {"workload": cfg["name"].replace("_fp64", "")
                       + ("_fp64" if prec == binding.DF_FP64 else "_fp32_state"),
                       "n_levels": cfg["n_levels"], "n": cfg["n"],
                       "box": [cfg["lo"][0], cfg["hi"][0]], "ghost": cfg["G"],
                       "mach": cfg["params"]["mach"], "chi": cfg["params"]["chi"],
                       "luminosity": cfg["params"]["L"],
                       "cell_updates_per_step": cu, "l2": "flushed between timed steps "
                       "(256 MB write outside the step events); working set above L2",
                       "parallelism": f"replicas{world}" if world > 1 else "single-gpu",
                       "tile_shapes": tile_summary(m["shapes"]),
                       "transport": "fused sweeps" if fused else "separate kernels"},
            "roofline": roofline,
            "fp64_peak_measured": fp64_peak,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": m["launches"],
            "clocks": m["clocks"],
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(kinds.items(),
                                                                 key=lambda x: -x[1][0])},
            "kernels_hbm": kernel_hbm_table(cfg, kinds, esz, fused, peak),
            "force": {"F": list(m["F"]), "F_along_motion": m["Fmot"]},
        }
        if fp32 is not None:
            line["fp32_state"] = fp32
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
