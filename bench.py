"""Benchmark: phase-space point updates per second of the fused BGK step.

One benchmark "step" is one whole run of the workload: reset the state to
the seeded initial condition, then the workload's number of time steps
(each: streaming, moments, Maxwellian, relaxation, boundaries).  Default
workload: the 2D lid-driven cavity, Kn 0.05, lid Mach 0.05, 256x256 cells,
48x48 velocities, its first 200 time steps in FP64; the same line carries
the FP32 and BF16-deviation forms of that run (`forms`, with their errors
against the oracle's stored fields after 2000 steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads: cavity256 (default), cavity256_full (all 20000 steps), cavity64
(64x64 cells, 32x32 velocities, 5000 steps), shock (200 cells, 64
velocities, 4000 steps), batch (64 cavities and 16 shocks; --persistent for
the single-launch form), adjoint (gradient of the lid shear, 128x128 x
32x32, 2000 steps), shock3v / shock3v_m15 (full 3D velocity grid), dsweep
(drag and flow rate against rarefaction); --precision f32 / bf16 for the
reduced forms, --accuracy for the per-field errors of a whole run.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on
the host cores instead (bounded samples of the same workload).  With N > 1
(under torch.distributed.run) every rank runs its own replica of the
workload (the single-GPU path does not shard here); value sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space updates/s (Nx*Nv per step) & % HBM roofline; mixed vs FP64 at stated err"
UNIT = "updates/s"
FP64_NOMINAL_FLOPS = 1.25e12   # GB300 FP64 peak from the unit counts and clocks (nominal)
# Algorithmic FP64 flops per point update (g and h at one (cell, velocity)),
# FMA = 2: stream 2 x (mul + 2 fma) = 10, moments 1 + 2 + 2 + 3 = 8,
# relaxation 2 x (mul + fma) = 6 (2D); 1D: stream 6, moments 6, relaxation 6.
FLOPS_PER_UPDATE = {1: 18.0, 2: 24.0}
# read f^n once, write f^{n+1} once (g and h): 2 x 2 values of the storage type
BYTES_PER_UPDATE = {"f64": 32.0, "f32": 16.0, "bf16": 8.0}
PRECISION = {"f64": 0, "f32": 1, "bf16": 2}
DTYPE = {"f64": "f64", "f32": "f32", "bf16": "bf16"}
DETAIL = {"f64": "FP64 state and arithmetic",
          "f32": ("FP32 state and arithmetic; moment sums carried in float-float (about 48 bits) and rounded "
                  "once to FP32 per cell; FP32 effective parameters; normalisation in float-float rounded to FP32"),
          "bf16": ("BF16 deviation from the absolute Maxwellian (FP32 arithmetic, stochastic rounding on store); "
                   "moment sums in float-float rounded once to FP32 per cell; FP32 effective parameters; "
                   "normalisation in float-float rounded to FP32")}


CAVITY256_200 = "cavity_kn0.05_ma0.05_256x256_v48x48_200steps"

# DRAM bytes per launch of the step kernel from an ncu capture (dram__bytes_
# read.sum + write.sum), valid only for the kernel sources that were
# captured and for the kernel that is launched: the SHA-1 of those files
# and the kernel name must match, else traffic is reported as null.  The
# capture commands sit with the ncu summaries under profiles/.
MEASURED_TRAFFIC = {
    ("cavity_kn0.1_ma0.1_64x64_v32x32_f64", "f64"): {
        "bytes": 170.2e6, "sources": ("csrc/bgk_step.cu", "csrc/bgk_device.cuh"),
        "sha1": "c04036d50a56b465b9502fa52f0cd08b44b65df3", "kernel": "bgk::step_f64_kernel"},
    # captured on 128^2 x 48^2 at 8 cells per CTA (2.458 GB per launch,
    # 65.1 B per update: the parked f~ of the resident cells exceeds L2 at
    # 48^2 velocities) and scaled by the 4x updates of a 256^2 x 48^2 launch
    (CAVITY256_200, "f64"): {
        "bytes": 4 * 2.458e9, "sources": ("csrc/bgk_step.cu", "csrc/bgk_device.cuh"),
        "sha1": "c04036d50a56b465b9502fa52f0cd08b44b65df3", "kernel": "bgk::step_f64_kernel",
        "note": "captured on 128^2 x 48^2 cells x velocities at 8 cells per CTA, scaled by updates"},
    (CAVITY256_200, "f32"): {
        "bytes": 2.544e9, "sources": ("csrc/bgk_mixed.cu", "csrc/bgk_device.cuh"),
        "sha1": "b79fe2943df7966e824c40d48003f385d010c245", "kernel": "bgk::step_mixed_pipe_kernel"},
    (CAVITY256_200, "bf16"): {
        "bytes": 1.171e9, "sources": ("csrc/bgk_mixed.cu", "csrc/bgk_device.cuh"),
        "sha1": "b79fe2943df7966e824c40d48003f385d010c245", "kernel": "bgk::step_mixed_kernel"},
}


def measured_traffic(workload: str, precision: str, kernel: str):
    """Captured DRAM bytes per launch for this workload, if the captured kernel is the one built
    and the one launched."""
    import hashlib

    rec = MEASURED_TRAFFIC.get((workload, precision))
    if rec is None or rec["kernel"] != kernel:
        return None
    h = hashlib.sha1()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_0903_4044_gb300", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest() == rec["sha1"] else None


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if self.proc is None or not getattr(self, "out", ""):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def workload(name: str) -> dict:
    from paper_0903_4044_gb300 import workloads as W

    if name in ("cavity64", W.CAVITY_64["name"]):
        return W.CAVITY_64
    if name in ("shock", W.SHOCK_M2["name"]):
        return W.SHOCK_M2
    if name in ("cavity256_f64", "cavity256"):
        return W.scaled(W.CAVITY_256, steps=200, name=CAVITY256_200)
    if name == "cavity256_full":
        return W.CAVITY_256
    raise SystemExit(f"unknown workload {name}")


def bench_config(w: dict, precision: str, world: int) -> dict:
    """The `config` object of a single-workload line (both arms print the same one)."""
    ncell, nv, _ = sizes(w)
    state_gb = BYTES_PER_UPDATE[precision] / 2 * ncell * nv / 1e9
    return {"workload": w["name"], "cells": ncell, "velocities": nv, "time_steps": w["steps"],
            "precision": precision, "arithmetic": DETAIL[precision], "parallelism": f"replica x{world}",
            "l2": (f"state {state_gb:.2f} GB per buffer; L2 flushed (256 MB write) between timed GPU steps")}


BATCH_NAME = "batch_64_cavities_16_shocks_seed0"


def batch_points(ws) -> int:
    return sum(w["n"] ** 2 * w["nv"] ** 2 if w["kind"] == "cavity" else w["nx"] * w["nvx"] for w in ws)


def config_for(args, w, world: int) -> dict:
    """The `config` object of a line; the GPU arm and the reference arm print the same one."""
    from paper_0903_4044_gb300 import workloads as W

    if args.workload == "batch":
        ws = W.batch_instances(0)
        return {"workload": BATCH_NAME, "instances": len(ws), "points": batch_points(ws),
                "time_steps": args.time_steps or 20, "precision": "f32",
                "launch": ("one persistent cooperative kernel per benchmark step (grid barrier between time "
                           "steps), captured in a CUDA graph") if args.persistent else
                          "one CUDA graph per benchmark step, one branch of step kernels per instance",
                "parallelism": f"replica x{world}",
                "l2": "inputs larger than L2 (9.4 GB of FP32 state)"}
    if args.workload == "adjoint":
        ncell, nv, _ = sizes(w)
        return {"workload": f"adjoint_{w['name']}", "cells": ncell, "velocities": nv, "time_steps": w["steps"],
                "checkpoint_every": args.checkpoint_every, "objective": "lid-integrated shear",
                "gradients": "Kn, lid speed, every entry of f0",
                "update": "one (cell, velocity) point of one differentiated time step",
                "precision": "f64", "parallelism": f"replica x{world}",
                "l2": "inputs larger than L2 (268 MB state, 27 GB of segment states)"}
    if args.workload in ("shock3v", "shock3v_m15"):
        ncell, nv = w["nx"], w["nv"][0] * w["nv"][1] * w["nv"][2]
        return {"workload": w["name"], "cells": ncell, "velocities": nv, "time_steps": w["steps"],
                "precision": "f64", "parallelism": f"replica x{world}",
                "l2": "flushed (256 MB write) between timed GPU steps; state larger than L2"}
    return bench_config(w, args.precision, world)


def sizes(w: dict) -> tuple[int, int, int]:
    if w["kind"] == "shock":
        return w["nx"], w["nvx"], 1
    return w["n"] * w["n"], w["nv"] * w["nv"], 2


# --------------------------------------------------------------------------
# CPU oracle legs (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the architecture."""
    import platform
    import subprocess

    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
    return f"{name or 'unknown'} ({platform.machine()})"


def oracle_sample(w: dict, sample_steps: int):
    """Time `sample_steps` oracle time steps of workload w; returns (updates/s, seconds, threads)."""
    import oracle
    from paper_0903_4044_gb300 import workloads as W

    oracle.build()
    if w["kind"] == "shock":
        prob, g, h = oracle.shock_problem(**w)
    else:
        prob0, _, _ = oracle.cavity_problem(**w)
        xi = W.perturbation(w.get("seed", 0), prob0.ncell, prob0.nv)
        prob, g, h = oracle.cavity_problem(**w, xi=xi)
    t0 = time.perf_counter()
    oracle.step(prob, g, h, sample_steps)
    dt = time.perf_counter() - t0
    return prob.ncell * prob.nv * sample_steps / dt, dt, oracle.threads()


def reference_sampler(name: str, w: dict | None):
    """(label, updates per sample, sample function) for the oracle on a bounded
    sample of workload `name`; the function returns (seconds, threads)."""
    import oracle
    from paper_0903_4044_gb300 import workloads as W

    oracle.build()
    if name in ("shock3v", "shock3v_m15"):
        w3 = W.SHOCK3V_M3 if name == "shock3v" else W.SHOCK3V_M15
        prob, f = oracle.shock3v_problem(**w3)
        k = max(1, int(2.0e8 // (prob.ncell * prob.nv)))

        def run():
            t0 = time.perf_counter()
            oracle.step3v(prob, f, k)
            return time.perf_counter() - t0, oracle.threads()
        return f"{k} time steps of {w3['name']}", prob.ncell * prob.nv * k, run, w3["name"]
    if name == "adjoint":
        wa = W.CAVITY_128
        prob0, _, _ = oracle.cavity_problem(**wa)
        xi = W.perturbation(wa.get("seed", 0), prob0.ncell, prob0.nv)
        prob, g, h = oracle.cavity_problem(**wa, xi=xi)
        k = 2

        def run():
            t0 = time.perf_counter()
            oracle.adjoint_lid_shear(prob, g, h, k)
            return time.perf_counter() - t0, oracle.threads()
        return (f"oracle forward + reverse pass over {k} time steps of {wa['name']}", prob.ncell * prob.nv * k,
                run, f"adjoint_{wa['name']}")
    if name == "batch":
        probs = []
        for w_ in W.batch_instances(0)[::4]:  # every fourth instance, one time step each
            w_ = dict(w_, steps=1)
            if w_["kind"] == "shock":
                prob, g, h = oracle.shock_problem(**w_)
            else:
                prob0, _, _ = oracle.cavity_problem(**w_)
                xi = W.perturbation(w_.get("seed", 0), prob0.ncell, prob0.nv)
                prob, g, h = oracle.cavity_problem(**w_, xi=xi)
            probs.append((prob, g, h))
        pts = sum(p.ncell * p.nv for p, _, _ in probs)

        def run():
            t0 = time.perf_counter()
            for prob, g, h in probs:
                oracle.step(prob, g, h, 1)
            return time.perf_counter() - t0, oracle.threads()
        return (f"one time step of every fourth batch instance ({len(probs)} instances)", pts, run,
                "batch_64_cavities_16_shocks_seed0")
    ncell, nv, _ = sizes(w)
    k = max(1, int(2.0e8 // (ncell * nv)))  # a few seconds per sample

    def run():
        _, dt, threads = oracle_sample(w, k)
        return dt, threads
    return f"{k} time steps of {w['name']}", ncell * nv * k, run, w["name"]


def reference_arm(args, w, rank, pg):
    """The oracle as it stands, on the host cores, on bounded samples of the
    workload (rank 0 only; other ranks exit without work)."""
    if rank != 0:
        return
    label, updates, run, wname = reference_sampler(args.workload, w)
    for _ in range(args.warmup):
        run()
    times, threads = [], None
    for _ in range(args.steps):
        dt, threads = run()
        times.append(dt)
    total = sum(times)
    value = updates * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_for(args, w, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{label} per benchmark step", "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def kernel_name(precision: str, dim: int, tile: int) -> str:
    if precision == "f64":
        return "bgk::step_f64_kernel"
    if dim == 1:
        return "bgk::step_mixed1d_kernel"
    # tile 1 of the 2D reduced-precision step is the pipelined kernel
    return "bgk::step_mixed_pipe_kernel" if tile == 1 else "bgk::step_mixed_kernel"


def roofline(w: dict, precision: str, per_launch: float, kname: str, traffic_override=None) -> dict:
    """Roofline of the step kernel from its CUDA-event launch time: FP64 forms
    against the nominal FP64 rate when that binds, else against measured HBM."""
    ncell, nv, dim = sizes(w)
    peaks = load_peaks()
    bytes_launch = BYTES_PER_UPDATE[precision] * ncell * nv
    flops_launch = FLOPS_PER_UPDATE[dim] * ncell * nv if precision == "f64" else 0.0
    hbm_achieved = bytes_launch / per_launch / 1e9
    alu_achieved = flops_launch / per_launch / 1e12
    t_hbm = bytes_launch / (peaks["hbm_gbs"] * 1e9)
    t_alu = flops_launch / FP64_NOMINAL_FLOPS
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": alu_achieved, "peak": FP64_NOMINAL_FLOPS / 1e12,
                "unit": "TFLOP/s", "frac": alu_achieved / (FP64_NOMINAL_FLOPS / 1e12),
                "peak_source": "nominal FP64 (unit counts x clock)"}
    else:
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hbm_achieved / peaks["hbm_gbs"], "peak_source": peaks["source"]}
    traffic = traffic_override if traffic_override is not None else measured_traffic(w["name"], precision, kname)
    note = MEASURED_TRAFFIC.get((w["name"], precision), {}).get("note")
    if traffic is not None and traffic_override is None and note:
        roof["traffic_note"] = note
    roof.update({"traffic": traffic, "kernel": kname, "launch_ms": per_launch * 1e3,
                 "bytes_per_update": BYTES_PER_UPDATE[precision], "hbm_gbs": hbm_achieved,
                 "hbm_frac": hbm_achieved / peaks["hbm_gbs"]})
    if precision == "f64":
        roof.update({"flops_per_update": FLOPS_PER_UPDATE[dim], "fp64_tflops": alu_achieved,
                     "fp64_frac": alu_achieved / (FP64_NOMINAL_FLOPS / 1e12)})
    return roof


def time_single(args, w, precision, world, local, pg, stream, e2e=True):
    """Device-timed and end-to-end rates of one solver on workload w.
    Returns (value, elapsed_s, per_launch_s, e2e_dict, tile, launches)."""
    import torch

    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import solver
    from paper_0903_4044_gb300 import workloads as W

    ncell, nv, dim = sizes(w)
    nsteps = w["steps"]
    prec = PRECISION[precision]
    if w["kind"] == "shock":
        s = solver.make_shock(w, stream=stream.cuda_stream, tile_cells=args.tile, precision=prec)
    else:
        xi = W.perturbation(w.get("seed", 0), ncell, nv)
        s = solver.make_cavity(w, xi=xi, stream=stream.cuda_stream, tile_cells=args.tile, precision=prec)
    f0_host = torch.empty((ncell, nv, 2), dtype=torch.float64, pin_memory=True)
    B.bgk_get_state(s.h, f0_host.numpy())
    f0_dev = f0_host.to(f"cuda:{local}")
    mom_host = torch.empty((ncell, 4), dtype=torch.float64, pin_memory=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def one_step(ev=None):
        B.bgk_set_state(s.h, f0_dev)
        if ev is not None:
            ev[0].record(stream)
        B.bgk_step(s.h, nsteps)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize()
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(pg)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        flush.zero_()           # L2 flush between timed steps (256 MB write)
        one_step(pairs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    B.bgk_sync(s.h)
    elapsed = max_over_ranks(pg, t_start.elapsed_time(t_end) / 1e3)
    kernel_s = sum(a.elapsed_time(b) for a, b in pairs) / 1e3
    launches = args.steps * nsteps
    per_launch = kernel_s / launches
    updates = ncell * nv * nsteps * args.steps
    value = world * updates / elapsed

    # end to end through the C ABI with host buffers (pinned)
    def e2e_step():
        B.bgk_set_state(s.h, f0_host.numpy())       # H2D, synchronous on the source
        B.bgk_step(s.h, nsteps)
        B.bgk_moments(s.h, mom_host.numpy(), 0)     # D2H, synchronises
    e2e_out = None
    if e2e and not args.no_e2e:
        for _ in range(args.warmup):
            e2e_step()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
        barrier(pg)
        e2e_out = {"value": world * updates / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(f0_host.numel() * 8),
                   "d2h_bytes_per_step": int(mom_host.numel() * 8)}
    tile = int(s.info.tile_cells)
    s.close()
    del flush, f0_dev
    torch.cuda.empty_cache()
    return value, elapsed, per_launch, e2e_out, tile, launches


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def load_cavity256_golden():
    """The oracle's stored fields after a prefix of the 256^2 x 48^2 cavity run
    (written by tests/golden/gen_cavity256.py): (steps, sampled moments rows,
    lid rows, J, mass), or None when no file is present."""
    import glob
    import re

    files = sorted(glob.glob(os.path.join(GOLDEN_DIR, "cavity256_*steps_moments.txt")))
    if not files:
        return None
    f = files[-1]
    steps = int(re.search(r"cavity256_(\d+)steps_moments", f).group(1))
    mom = np.loadtxt(f)
    lidf = f.replace("_moments.txt", "_lid.txt")
    J = mass = None
    with open(lidf) as fh:
        for line in fh:
            if line.startswith("# J "):
                J = float(line.split()[2])
            if line.startswith("# mass "):
                mass = float(line.split()[2])
    return steps, mom, np.loadtxt(lidf), J, mass


def oracle_errors(forms, local):
    """Per-field errors of each form after the stored prefix of the 256^2 x 48^2
    cavity run, against the oracle's stored fields (sampled cells and the lid)."""
    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import solver
    from paper_0903_4044_gb300 import workloads as W

    g = load_cavity256_golden()
    if g is None:
        return None
    steps, rows, lid, J, mass = g
    w = W.CAVITY_256
    n = w["n"]
    ix, iy = rows[:, 0].astype(int), rows[:, 1].astype(int)
    want = rows[:, 2:6]
    uw = w["lid_mach"] * (5.0 / 6.0) ** 0.5
    xi = W.perturbation(w["seed"], n * n, w["nv"] * w["nv"])
    out = {"time_steps": steps, "reference": f"oracle fields after {steps} steps "
           f"(tests/golden/cavity256_{steps}steps_*.txt; {len(rows)} sampled cells, every lid cell)"}
    for name in forms:
        s = solver.make_cavity(w, xi=xi, precision=PRECISION[name])
        t0 = time.perf_counter()
        s.step(steps)
        mom = s.moments().reshape(n, n, 4)
        fl = s.wall_fluxes(B.BGK_FACE_YHI)
        secs = time.perf_counter() - t0
        dx = s.info.dx
        s.close()
        got = mom[iy, ix]
        Jg = float(dx * fl[:, 1].sum())
        massg = float(mom[:, :, 0].sum() * dx * dx)
        out[name] = {
            "err_n_rel_max": float(np.abs(got[:, 0] - want[:, 0]).max() / np.abs(want[:, 0]).max()),
            "err_u_over_lid_speed_max": float(np.abs(got[:, 1:3] - want[:, 1:3]).max() / uw),
            "err_u_over_lid_speed_rms": float(np.sqrt(((got[:, 1:3] - want[:, 1:3]) ** 2).mean()) / uw),
            "err_theta_rel_max": float(np.abs(got[:, 3] - want[:, 3]).max() / np.abs(want[:, 3]).max()),
            "err_lid_shear_cell_rel_max": float(np.abs(fl[:, 1] - lid[:, 2]).max() / np.abs(lid[:, 2]).max()),
            "err_lid_shear_J_rel": abs(Jg - J) / abs(J),
            "err_mass_rel": abs(massg - mass) / mass,
            "seconds": secs,
        }
    return out


def ours_arm(args, w, world, rank, local, pg):
    import torch

    from paper_0903_4044_gb300 import build

    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ncell, nv, dim = sizes(w)
    nsteps = w["steps"]

    with ClockSampler(local) as clk:
        value, elapsed, per_launch, e2e, tile, launches = time_single(args, w, args.precision, world, local,
                                                                      pg, stream)
        kname = kernel_name(args.precision, dim, tile)
        roof = roofline(w, args.precision, per_launch, kname, args.traffic)
        # the reduced-precision forms of the same workload, timed the same way
        forms = None
        if w["name"] == CAVITY256_200 and args.precision == "f64" and not args.no_forms:
            forms = {}
            for name in ("f32", "bf16"):
                v, el, pl, e2, t, ln = time_single(args, w, name, world, local, pg, stream)
                forms[name] = {"value": v, "unit": UNIT, "ms_per_step": 1e3 * el / args.steps,
                               "tile_cells": t, "arithmetic": DETAIL[name],
                               "roofline": roofline(w, name, pl, kernel_name(name, dim, t)), "e2e": e2, "gpu_launches": ln,
                               "speedup_vs_f64": v / value}
                launches += ln
    clocks = clk.summary()
    if forms is not None and rank == 0:
        errs = oracle_errors(["f64", "f32", "bf16"], local)
        if errs is not None:
            forms["f64"] = {"err_vs_oracle": errs["f64"]}
            for name in ("f32", "bf16"):
                forms[name]["err_vs_oracle"] = errs[name]
            forms["err_reference"] = {k: errs[k] for k in ("time_steps", "reference")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = max(1, int(3.0e9 // (ncell * nv)))  # about 10 s on 16 host cores
        rate, dt, threads = oracle_sample(w, sample)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{sample} time steps of {w['name']} ({dt:.1f} s)", "cpu_model": cpu_model()}
        # the same oracle on one core, on a shorter sample (about 5 s)
        import oracle

        sample1 = max(1, int(1.0e8 // (ncell * nv)))
        oracle.set_threads(1)
        try:
            rate1, dt1, _ = oracle_sample(w, sample1)
        finally:
            oracle.set_threads(threads)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT,
                                "sample": f"{sample1} time steps of {w['name']} ({dt1:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": config_for(args, w, world),
            "tile_cells": tile,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches,
        }
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line), flush=True)


def accuracy_arm(args, w):
    """Per-field error of a reduced-precision run against the FP64 GPU path
    over the whole run (20000 steps of the 256^2 cavity are beyond the
    oracle's reach on the host; the FP64 path itself is compared with the
    oracle's stored fields after a prefix of that run by the GPU tests and by
    the `forms` of the default benchmark): n, U, theta of every cell and the
    lid's mean shear flux."""
    import torch

    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import build, solver
    from paper_0903_4044_gb300 import workloads as W

    build.build()
    torch.cuda.set_device(0)
    ncell, nv, _ = sizes(w)
    xi = W.perturbation(w.get("seed", 0), ncell, nv)
    # --precision f64 (the default) compares both reduced forms with one FP64 run
    forms = ["f32", "bf16"] if args.precision == "f64" else [args.precision]
    out = {}
    for name in ["f64"] + forms:
        s = solver.make_cavity(w, xi=xi, precision=PRECISION[name])
        t0 = time.perf_counter()
        s.step(w["steps"])
        mom = s.moments()
        lid = s.wall_fluxes(B.BGK_FACE_YHI)
        out[name] = (mom, lid, time.perf_counter() - t0)
        s.close()
    m64, l64, t64 = out["f64"]
    uw = w["lid_mach"] * (5.0 / 6.0) ** 0.5
    for name in forms:
        mr, lr, tr = out[name]
        shear64, shear = float(l64[:, 1].mean()), float(lr[:, 1].mean())
        line = {
            "mode": "accuracy", "workload": w["name"], "precision": name, "time_steps": w["steps"],
            "reference": "FP64 GPU path over the same run",
            "err_n_rel_max": float(np.abs(mr[:, 0] - m64[:, 0]).max() / np.abs(m64[:, 0]).max()),
            "err_u_over_lid_speed_max": float(np.abs(mr[:, 1:3] - m64[:, 1:3]).max() / uw),
            "err_theta_rel_max": float(np.abs(mr[:, 3] - m64[:, 3]).max() / np.abs(m64[:, 3]).max()),
            "err_u_over_lid_speed_rms": float(np.sqrt(((mr[:, 1:3] - m64[:, 1:3]) ** 2).mean()) / uw),
            "lid_shear_f64": shear64, "lid_shear": shear,
            "err_lid_shear_rel": abs(shear - shear64) / abs(shear64),
            "mass_drift_rel": float(abs(mr[:, 0].sum() - m64[:, 0].sum()) / m64[:, 0].sum()),
            "seconds": {"f64": t64, name: tr},
        }
        print(json.dumps(line), flush=True)


# The paper's table of the drag coefficient D and reduced flow rate G of the
# main vortex versus the rarefaction parameter delta (Sec. 5, "Results and
# discussion"): delta -> (D, G) of its parallel code.
PAPER_DG = {0.1: (0.675, 0.0975), 1.0: (0.624, 0.103), 10.0: (0.393, 0.143)}


def dsweep_arm(args):
    """The cavity of Sec. 5 at delta = 0.1, 1, 10 (side delta mean free
    paths, 160^2 cells, 20^2 reduced velocities on [-3, 3]^2, lid speed 0.01,
    FP64) stepped to a steady lid shear, with D and G under the reading stated
    in the line (the paper does not give their normalisation) and the
    normalisation-free ratios to delta = 0.1 beside the paper's."""
    import torch

    from paper_0903_4044_gb300 import build, solver

    build.build()
    torch.cuda.set_device(0)
    uw, n, nv = 0.01, 160, 20
    out = {}
    for delta, (d_paper, g_paper) in PAPER_DG.items():
        w = dict(kind="cavity", kn=1.0 / delta, n=n, nv=nv, vbox=(-3.0, 3.0), omega=0.5, cfl=0.5)
        s = solver.Solver(solver.cavity_config(**w, lid_speed=uw))
        s.init_uniform((1.0, 0.0, 0.0, 1.0))
        t0, steps, J, chunk = time.perf_counter(), 0, None, 2000
        while steps < 400000:
            s.step(chunk)
            steps += chunk
            Jn = s.lid_shear()
            done = J is not None and abs(Jn - J) < 1e-7 * abs(Jn)
            J = Jn
            if done:
                break
        mom = s.moments().reshape(n, n, 4)
        s.close()
        # D: mean lid shear over the lid length, in units of P0 U_W / v0
        # (P0 = n0 m v0^2 / 2, v0 = sqrt(2 R T0)); its free-molecular value
        # is 1 / sqrt(pi) = 0.564
        D = 2.0 * (J / delta) / uw
        # G: integral of u_x / U_W along the vertical centre line from the
        # vortex centre (where u_x changes sign) to the lid, per unit side
        ux = 0.5 * (mom[:, n // 2 - 1, 1] + mom[:, n // 2, 1]) / uw
        k0 = int(np.nonzero(ux <= 0.0)[0].max()) + 1 if np.any(ux <= 0.0) else 0
        G = float(ux[k0:].sum()) / n
        out[delta] = dict(D=D, G=G, steps=steps, seconds=time.perf_counter() - t0, D_paper=d_paper, G_paper=g_paper)
    for delta, r in out.items():
        r["D_over_paper"] = r["D"] / r["D_paper"]
        r["G_over_paper"] = r["G"] / r["G_paper"]
        r["D_over_D01"] = r["D"] / out[0.1]["D"]
        r["D_over_D01_paper"] = r["D_paper"] / PAPER_DG[0.1][0]
        r["G_over_G01"] = r["G"] / out[0.1]["G"]
        r["G_over_G01_paper"] = r["G_paper"] / PAPER_DG[0.1][1]
        print(json.dumps({"mode": "dsweep", "delta": delta, "unpinned": True,
                          "reading": "D = 2 <tau_xy>_lid / U_W (units P0 U_W / v0); G = int u_x / U_W dy / L "
                                     "from the vortex centre to the lid on x = L/2",
                          **r}), flush=True)


def batch_arm(args, world, rank, local, pg):
    """The batched workload: 64 uneven cavities and 16 shocks, FP32 state
    in one bgk_batch, tiles chosen by the autotuner; a benchmark step is
    --time-steps (default 20) steps of every instance, continuing the
    evolution from the initial states set once before the warm-up.  The
    end-to-end leg sets every instance's state from pinned host memory,
    steps it and reads its moments back, per benchmark step."""
    import torch

    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import build, solver
    from paper_0903_4044_gb300 import workloads as W

    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ws = W.batch_instances(0)
    b = solver.Batch(ws, stream=stream.cuda_stream, perturb=False)
    b.autotune(3)
    if args.persistent:
        b.set_persistent(True)
    nsteps = args.time_steps or 20
    pts = b.points()

    for _ in range(args.warmup):
        b.step(nsteps)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(pg)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            b.step(nsteps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    b.sync()
    elapsed = max_over_ranks(pg, ev0.elapsed_time(ev1) / 1e3)
    value = world * pts * nsteps * args.steps / elapsed

    e2e = None
    if not args.no_e2e:
        # one pinned host buffer holding every instance's state (ABI layout,
        # FP64) and one for every instance's moments
        offs, moffs, o, mo = [], [], 0, 0
        for s_ in b.solvers:
            offs.append(o)
            moffs.append(mo)
            o += s_.ncell * s_.nv * 2
            mo += s_.ncell * 4
        host = torch.empty(o, dtype=torch.float64, pin_memory=True)
        mom = torch.empty(mo, dtype=torch.float64, pin_memory=True)
        hv, mv = host.numpy(), mom.numpy()
        for s_, off in zip(b.solvers, offs):
            B.bgk_get_state(s_.h, hv[off:off + s_.ncell * s_.nv * 2])

        def e2e_step():
            for s_, off in zip(b.solvers, offs):
                B.bgk_set_state(s_.h, hv[off:off + s_.ncell * s_.nv * 2])   # H2D
            b.step(nsteps)
            for s_, mo_ in zip(b.solvers, moffs):
                B.bgk_moments(s_.h, mv[mo_:mo_ + s_.ncell * 4], 0)          # D2H
        e2e_step()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": world * pts * nsteps * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(o * 8), "d2h_bytes_per_step": int(mo * 8)}
        del host, mom

    peaks = load_peaks()
    hbm = BYTES_PER_UPDATE["f32"] * pts * nsteps * args.steps / elapsed / 1e9
    roof = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": hbm / peaks["hbm_gbs"], "peak_source": peaks["source"], "traffic": None,
            "kernel": ("bgk::batch_persistent_kernel" if args.persistent else
                       "all step kernels of the batch (bgk::step_mixed_kernel, step_mixed_pipe_kernel, "
                       "step_mixed1d_kernel)"),
            "bytes_per_update": BYTES_PER_UPDATE["f32"],
            "note": "algorithmic bytes of every instance (16 B per point and time step) over the whole batch step"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        label, updates, run, _ = reference_sampler("batch", None)
        dt, threads = run()
        cpu = {"value": updates / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{label} ({dt:.1f} s; FP64 oracle)", "cpu_model": cpu_model()}
    if rank == 0:
        tiles = sorted({int(s_.info.tile_cells) for s_ in b.solvers})
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_for(args, None, world), "tiles_chosen": tiles,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": args.steps if args.persistent else len(ws) * nsteps * args.steps,
        }), flush=True)
    b.close()


# Algorithmic cost per point and time step of the gradient evaluation (FP64
# state, FMA = 2 flops).  Forward step and its recomputation: 32 B and 24
# flops each.  Reverse step (adj_step_kernel): reads lambda~^{n+1} and
# f^{n+1}, writes lambda~^n (48 B); gather 10 flops, collision sums 17,
# output polynomial 10 (37 flops).
ADJ_BYTES_PER_UPDATE = {"forward": 32.0, "recompute": 32.0, "adj_step": 48.0}
ADJ_FLOPS_PER_UPDATE = {"forward": 24.0, "recompute": 24.0, "adj_step": 37.0}


def adjoint_arm(args, w, world, rank, local, pg):
    """Gradient of the lid-integrated shear (128^2 cells, 32^2 velocities,
    Kn 0.1, lid Mach 0.1, 2000 FP64 steps, a checkpoint every 100 steps) with
    respect to Kn, the lid speed and every entry of f0.  A benchmark step is
    one whole gradient evaluation: forward with checkpoints, segment
    recomputation, reverse pass."""
    import torch

    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import build, solver
    from paper_0903_4044_gb300 import workloads as W

    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ncell, nv, _ = sizes(w)
    nsteps, K = w["steps"], args.checkpoint_every
    xi = W.perturbation(w.get("seed", 0), ncell, nv)
    s = solver.make_cavity(w, xi=xi, stream=stream.cuda_stream)
    f0_host = torch.empty((ncell, nv, 2), dtype=torch.float64, pin_memory=True)
    B.bgk_get_state(s.h, f0_host.numpy())
    f0_dev = f0_host.to(f"cuda:{local}")
    grad_dev = torch.empty_like(f0_dev)
    grad_host = torch.empty_like(f0_host).pin_memory()

    def one(dev=True):
        if dev:
            B.bgk_set_state(s.h, f0_dev)
            return B.bgk_adjoint_lid_shear(s.h, nsteps, K, grad_dev)
        B.bgk_set_state(s.h, f0_host.numpy())
        return B.bgk_adjoint_lid_shear(s.h, nsteps, K, grad_host.numpy())

    for _ in range(args.warmup):
        out = one()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(pg)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            out = one()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    elapsed = max_over_ranks(pg, ev0.elapsed_time(ev1) / 1e3)
    updates = ncell * nv * nsteps
    value = world * updates * args.steps / elapsed
    e2e = None
    if not args.no_e2e:
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one(dev=False)
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": world * updates * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(f0_host.numel() * 8), "d2h_bytes_per_step": int(grad_host.numel() * 8)}
    peaks = load_peaks()
    bytes_eval = sum(ADJ_BYTES_PER_UPDATE.values()) * updates
    flops_eval = sum(ADJ_FLOPS_PER_UPDATE.values()) * updates
    hbm = bytes_eval * args.steps / elapsed / 1e9
    alu = flops_eval * args.steps / elapsed / 1e12
    roof = {"bound": "alu", "achieved": alu, "peak": FP64_NOMINAL_FLOPS / 1e12, "unit": "TFLOP/s",
            "frac": alu / (FP64_NOMINAL_FLOPS / 1e12), "traffic": args.traffic,
            "peak_source": "nominal FP64 (unit counts x clock)",
            "kernel": "whole gradient evaluation (step_f64_kernel x2, adj_step_kernel)",
            "flops_per_update": ADJ_FLOPS_PER_UPDATE, "bytes_per_update": ADJ_BYTES_PER_UPDATE,
            "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"], "hbm_peak_source": peaks["source"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        sample = 3
        prob, g, h = oracle.cavity_problem(**w, xi=xi)
        t0 = time.perf_counter()
        oracle.adjoint_lid_shear(prob, g, h, sample)
        dt = time.perf_counter() - t0
        cpu = {"value": ncell * nv * sample / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"oracle forward + reverse pass over {sample} time steps of {w['name']} ({dt:.1f} s; "
                         "the reverse sweep runs on one core)"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_for(args, w, world),
            "result": {"J": out[0], "dJ_dlnL": out[1], "dJ_dUW": out[2]},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            # forward, recomputation, one reverse kernel per step plus the
            # final streaming adjoint, lid table and seed
            "gpu_launches": args.steps * (3 * nsteps + 3),
        }), flush=True)
    s.close()


# Full velocity grid (1D space): per update (one f value at one (cell,
# velocity) point) read f^n once and write f^{n+1} once (16 B); FP64 flops:
# streaming 3, the five moment sums 9, relaxation b f~ + px py pz 4.
FLOPS_PER_UPDATE_3V = 16.0
BYTES_PER_UPDATE_3V = 16.0


def shock3v_arm(args, w, world, rank, local, pg):
    """The shock of Sec. 4.1 as the paper computed it (full 3D velocity grid);
    a benchmark step is the workload's time steps from the step profile."""
    import torch

    import oracle
    from paper_0903_4044_gb300 import bgk as B
    from paper_0903_4044_gb300 import build, solver

    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    s = solver.make_shock3v(w, stream=stream.cuda_stream)
    ncell, nv, nsteps = s.ncell, s.nv, w["steps"]
    f0_host = torch.empty((ncell, nv), dtype=torch.float64, pin_memory=True)
    B.bgk3v_get_state(s.h, f0_host.numpy())
    f0_dev = f0_host.to(f"cuda:{local}")
    mom_host = torch.empty((ncell, 5), dtype=torch.float64, pin_memory=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def one_step(ev=None):
        B.bgk3v_set_state(s.h, f0_dev)
        if ev is not None:
            ev[0].record(stream)
        B.bgk3v_step(s.h, nsteps)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize()
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(pg)
        torch.cuda.synchronize()
        t_start.record(stream)
        for k in range(args.steps):
            flush.zero_()
            one_step(pairs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    B.bgk3v_sync(s.h)
    elapsed = max_over_ranks(pg, t_start.elapsed_time(t_end) / 1e3)
    per_launch = sum(a.elapsed_time(b) for a, b in pairs) / 1e3 / (args.steps * nsteps)
    updates = ncell * nv * nsteps
    value = world * updates * args.steps / elapsed
    e2e = None
    if not args.no_e2e:
        def e2e_step():
            B.bgk3v_set_state(s.h, f0_host.numpy())
            B.bgk3v_step(s.h, nsteps)
            B.bgk3v_moments(s.h, mom_host.numpy(), 0)
        e2e_step()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": world * updates * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(f0_host.numel() * 8), "d2h_bytes_per_step": int(mom_host.numel() * 8)}
    peaks = load_peaks()
    alu = FLOPS_PER_UPDATE_3V * ncell * nv / per_launch / 1e12
    hbm = BYTES_PER_UPDATE_3V * ncell * nv / per_launch / 1e9
    roof = {"bound": "alu", "achieved": alu, "peak": FP64_NOMINAL_FLOPS / 1e12, "unit": "TFLOP/s",
            "frac": alu / (FP64_NOMINAL_FLOPS / 1e12), "traffic": args.traffic,
            "peak_source": "nominal FP64 (unit counts x clock)", "kernel": "bgk::step3v_kernel",
            "launch_ms": per_launch * 1e3, "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle.build()
        sample = max(1, int(2e9 // (ncell * nv)))  # about 10 s on the host cores
        prob, f = oracle.shock3v_problem(**w)
        t0 = time.perf_counter()
        oracle.step3v(prob, f, sample)
        dt = time.perf_counter() - t0
        cpu = {"value": ncell * nv * sample / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{sample} time steps of {w['name']} ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_for(args, w, world), "max_courant": s.info.max_courant,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": args.steps * nsteps,
        }), flush=True)
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="cavity256")
    ap.add_argument("--no-forms", action="store_true",
                    help="cavity256: skip the FP32 and BF16-deviation forms and their oracle errors")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the step kernel from an ncu capture")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="override the workload's time steps per benchmark step (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--tile", type=int, default=0, help="cells per CTA of the step kernel (0 = library choice)")
    ap.add_argument("--accuracy", action="store_true",
                    help="report per-field errors of --precision (both reduced forms when f64) against the FP64 path instead of timing")
    ap.add_argument("--precision", default="f64", choices=sorted(PRECISION),
                    help="state storage: f64, f32, or bf16 deviation from the absolute Maxwellian")
    ap.add_argument("--checkpoint-every", type=int, default=100, help="adjoint workload: steps per checkpoint")
    ap.add_argument("--persistent", action="store_true",
                    help="batch workload: one persistent cooperative launch per benchmark step")
    args = ap.parse_args()
    world, rank, local, pg = dist_setup()
    w = resolve_workload(args)
    if args.impl == "reference":
        reference_arm(args, w, rank, pg)
    elif args.workload in ("shock3v", "shock3v_m15"):
        shock3v_arm(args, w, world, rank, local, pg)
    elif args.workload == "batch":
        batch_arm(args, world, rank, local, pg)
    elif args.workload == "adjoint":
        adjoint_arm(args, w, world, rank, local, pg)
    elif args.workload == "dsweep":
        if rank == 0:
            dsweep_arm(args)
    elif args.accuracy:
        if rank == 0:
            accuracy_arm(args, w)
    else:
        ours_arm(args, w, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


def resolve_workload(args):
    """Raw parameters of --workload with --time-steps applied (None for the batch)."""
    from paper_0903_4044_gb300 import workloads as W

    if args.workload in ("batch", "dsweep"):
        return None
    if args.workload == "adjoint":
        w = W.CAVITY_128
    elif args.workload in ("shock3v", "shock3v_m15"):
        w = W.SHOCK3V_M3 if args.workload == "shock3v" else W.SHOCK3V_M15
    else:
        w = workload(args.workload)
    if args.time_steps is not None and args.time_steps != w["steps"]:
        w = dict(w, steps=args.time_steps, name=f"{w['name']}_{args.time_steps}steps")
    return w


if __name__ == "__main__":
    main()
