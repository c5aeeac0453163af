#!/usr/bin/env python3
"""Phase-space updates/s of the discrete-velocity BGK scheme (HOFKS) on GB300.

    python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--impl reference]

One step = one full time step of the hot path: alpha reduction, the MUSCL Euler
sub-steps, the kinetic pass over all N_c x N_v phase-space points and the
end-of-step cell update, replayed from the captured CUDA graph.  Inputs are
seeded synthetic fields (``paper_1212_0204_gb300.workloads``) shaped like the
paper's workloads.  The default workload is the 3D-3V periodic density wave,
96^3 cells x 24^3 velocities (1.22e10 phase-space points, f = 48.9 GB in FP32);
f is far larger than L2 in every workload, so no flush is needed between steps.

Prints one JSON line on rank 0.  Under torchrun every rank runs an independent
replica of the workload (weak scaling; the method has no exchange step on one
problem per GPU) and ``value`` is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1212_0204_gb300 import workloads as W  # noqa: E402

METRIC = "phase-space updates/s"
UNIT = "updates/s"

# name -> (case builder, precision, bytes of f per update: one read + one write)
WORKLOADS = {
    "quadrant_2d": (lambda: W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=500), "f32"),
    "quadrant_2d_tau1e-5": (lambda: W.quadrant_2d(n=256, nv=32, tau=1e-5, steps=500), "f32"),
    "quadrant_2d_tau1e-1": (lambda: W.quadrant_2d(n=256, nv=32, tau=1e-1, steps=500), "f32"),
    "density_wave_3d": (lambda: W.density_wave_3d(n=96, nv=24, tau=1e-4, steps=100), "f32"),
    "density_wave_3d_64": (lambda: W.density_wave_3d(n=64, nv=24, tau=1e-4, steps=100), "f32"),
    "quadrant_2d_f64": (lambda: W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=500), "f64"),
    "quadrant_2d_bf16": (lambda: W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=500), "bf16"),
    "density_wave_3d_bf16": (lambda: W.density_wave_3d(n=96, nv=24, tau=1e-4, steps=100), "bf16"),
    "sod_1d": (lambda: W.sod_1d(nx=200, nv=32, tau=1e-4), "f64"),
    "batched_tubes": (lambda: W.batched_tubes(ncases=512, steps=100), "f32"),
    "shear_learned": (lambda: W.shear_layer_2d(n=512, nv=32, steps=50, dv=0.4), "f32"),
    "implosion_2d": (lambda: W.implosion_2d(n=200, nv=30, tau=1e-3), "f32"),
    "vortex_weno_2d": (lambda: W.isentropic_vortex_2d(200, scheme=W.HOFKS_WENO), "f64"),
}
DESCR = {
    "quadrant_2d": "2D-2V four-quadrant Riemann problem, 256x256 periodic cells x 32x32 velocities, "
                   "tau=1e-3, HOFKS, FP32 f / FP64 moments",
    "quadrant_2d_tau1e-5": "2D-2V four-quadrant Riemann problem, 256x256 periodic cells x 32x32 velocities, "
                           "tau=1e-5, HOFKS, FP32 f / FP64 moments",
    "quadrant_2d_tau1e-1": "2D-2V four-quadrant Riemann problem, 256x256 periodic cells x 32x32 velocities, "
                           "tau=1e-1, HOFKS, FP32 f / FP64 moments",
    "density_wave_3d": "3D-3V periodic density wave, 96^3 cells x 24^3 velocities, tau=1e-4, HOFKS, "
                       "FP32 f / FP64 moments",
    "density_wave_3d_64": "3D-3V periodic density wave, 64^3 cells x 24^3 velocities, tau=1e-4, HOFKS, "
                          "FP32 f / FP64 moments",
    "quadrant_2d_f64": "2D-2V four-quadrant Riemann problem, 256^2 x 32^2, HOFKS, FP64 f",
    "quadrant_2d_bf16": "2D-2V four-quadrant Riemann problem, 256^2 x 32^2, HOFKS, BF16 f storage",
    "density_wave_3d_bf16": "3D-3V periodic density wave, 96^3 cells x 24^3 velocities, tau=1e-4, HOFKS, "
                            "BF16 f storage / FP32 arithmetic / FP64 moments",
    "sod_1d": "1D-1V Sod tube, 200 cells x 32 velocities, tau=1e-4, outflow, HOFKS, FP64",
    "shear_learned": "2D-2V shear layer, 512x512 periodic cells x 32x32 velocities, "
                     "tau = 1e-5*10^(5r) (seeded smooth r), HOFKS FP32 + learned regime path vs plain "
                     "FP32 and plain FP64, 50 steps",
    "implosion_2d": "2D-2V implosion (Section 5.4): [0,2]^2, 200x200 cells x 30x30 velocities on [-20,20)^2, "
                    "tau=1e-3, outflow, p=3 (t=0.07 in 28 steps), HOFKS, FP32 f / FP64 moments",
    "vortex_weno_2d": "2D-2V isentropic vortex (Section 5.2), 200x200 cells x 40x40 velocities, tau=1e-4, "
                      "HOFKS with the WENO5 Euler solver (Section 4.3.3), FP64",
    "batched_tubes": "512 independent 1D-1V Riemann tubes in one batched launch per phase, "
                     "N_x ~ U{100..2000}, N_v in {32,64,128}, tau = 10^U(-5,0), outflow, HOFKS, "
                     "FP32 f / FP64 moments",
}
BYTES_PER_UPDATE = {"f64": 16, "f32": 8, "bf16": 4}
DTYPE = {"f64": "f64", "f32": "f32", "bf16": "bf16"}


def conserved(case):
    """Conserved moments (Eqs. Mo/E) from the recipe's primitive fields, host side."""
    d = case.d
    U = np.zeros((d + 2, case.ncells))
    U[0] = case.rho
    for i in range(d):
        U[1 + i] = case.rho * case.u[i]
    U[d + 1] = 0.5 * case.rho * (case.u ** 2).sum(0) + 0.5 * d * case.rho * case.T
    return U


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kinetic_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("dvm_kinetic.cu", "dvm_kinetic_shapes.cu", "dvm_window_kernel.cuh", "dvm_window.cuh",
              "dvm_internal.cuh", "dvm_linmom.cu", "dvm_tile_kernel.cuh"):
        with open(os.path.join(ROOT, "paper_1212_0204_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per kinetic-pass launch from the committed ncu summary, if it was
    taken on the current kernel source and this workload; else None."""
    path = os.path.join(ROOT, "profiles", "kinetic_pass_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kinetic_source_hash()
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split())
        if kv.get("workload") == workload and kv.get("source") == src:
            return float(kv["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[2:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


def oracle_sample(case, budget_points: float):
    """A bounded sample of the workload for the CPU oracle: same velocity grid and
    initial-data recipe, fewer cells (a square/cubic sub-problem), or for a batch
    the first tubes up to the budget.  Returns (list of cases, description)."""
    if isinstance(case, list):
        picked, pts = [], 0
        for c in case:
            picked.append(c)
            pts += c.points
            if pts >= budget_points:
                break
        return picked, f"the first {len(picked)} of {len(case)} tubes ({pts} points)"
    if case.name in ("quadrant_2d", "implosion_2d"):
        n = int(max(8, min(case.nx[0], round((budget_points / case.nvel) ** 0.5))))
        if case.name == "implosion_2d":
            return ([W.implosion_2d(n=n, nv=case.nv[0], tau=case.tau)], f"{n}x{n} cells x {case.nvel} velocities")
        return ([W.quadrant_2d(n=n, nv=case.nv[0], tau=case.tau, steps=1, dv=case.dv)],
                f"{n}x{n} cells x {case.nvel} velocities")
    if case.name == "density_wave_3d":
        n = int(max(4, min(case.nx[0], round((budget_points / case.nvel) ** (1 / 3)))))
        return ([W.density_wave_3d(n=n, nv=case.nv[0], tau=case.tau, steps=1, dv=case.dv)],
                f"{n}^3 cells x {case.nvel} velocities")
    return [case], f"{case.nx[0]} cells x {case.nvel} velocities"


def time_oracle(cases, steps: int, warmup: int = 0):
    """Single-thread FP64 oracle over the sample: (updates/s, seconds timed)."""
    import oracle
    from tests.helpers import grid
    total_pts, secs = 0, 0.0
    for case in cases:
        s = oracle.Scheme(grid(case), tau=case.tau)
        s.set_moments(conserved(case))
        if warmup:
            s.step(warmup)
        t0 = time.perf_counter()
        s.step(steps)
        secs += time.perf_counter() - t0
        total_pts += case.points * steps
    return total_pts / secs, secs


def cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, e.g. on Arm)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_replica(args):
    """One independent oracle run (a worker of the all-core timing): the sample
    cases advanced `steps` steps; returns the phase-space points updated."""
    descr, steps = args
    cases = [W.Case(**c) for c in descr]
    import oracle
    from tests.helpers import grid
    pts = 0
    for case in cases:
        s = oracle.Scheme(grid(case), tau=case.tau)
        s.set_moments(conserved(case))
        s.step(steps)
        pts += case.points * steps
    return pts


def time_oracle_all_cores(cases, steps: int, cores: int):
    """The oracle as it stands (single-threaded) run as `cores` independent
    replicas of the sample at once, one process each (spawned, so no CUDA
    state is inherited): whole-host updates/s over the wall time of all of
    them, and the seconds that took."""
    import dataclasses
    import multiprocessing as mp
    descr = [dataclasses.asdict(c) for c in cases]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_replica, [(descr, 1)] * cores)   # start-up and page-in, untimed
        t0 = time.perf_counter()
        pts = sum(pool.map(_oracle_replica, [(descr, steps)] * cores))
        secs = time.perf_counter() - t0
    return pts / secs, secs


def moment_err(Ug, Uo) -> float:
    """Largest relative moment error; each row scaled by max(|U_i|_inf, |rho|_inf)."""
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    return float((np.abs(Ug - Uo).max(axis=1) / scale).max())


def precision_error(dvm, sample, precision, batch: bool, steps: int = 2):
    """The error of the bench's precision tier against the FP64 oracle, stated with
    the result: the library at that precision and the oracle advance the same cases
    from the same initial moments for `steps` steps.  Reported: the largest relative
    moment error over the cases and, for single problems, the largest error of f at
    the cell centres relative to max |f| (f carries the storage rounding; in the
    fluid regime the moments hardly see it, since lambda f is what enters them)."""
    import oracle
    from tests.helpers import grid
    cases = sample[:8]
    ref, fref = [], []
    for c in cases:
        o = oracle.Scheme(grid(c), tau=c.tau)
        o.set_moments(conserved(c))
        o.step(steps)
        ref.append(o.moments())
        if not batch:
            fref.append(o.f())
        del o
    out = {"steps": steps, "cases": len(cases)}
    if batch:
        b = dvm.Batch(cases, precision=precision)
        b.set_moments(b.pack([conserved(c) for c in cases]))
        b.step(steps)
        U = b.moments()
        got = [b.case_moments(U, i) for i in range(len(cases))]
        out["kinetic_kernel"] = "batch"
        b.close()
    else:
        got, ferr = [], 0.0
        for c, fo in zip(cases, fref):
            s = dvm.Solver.from_case(c, precision=precision)
            s.set_moments(conserved(c))
            s.step(steps)
            got.append(s.moments())
            ferr = max(ferr, float(np.abs(s.f() - fo).max() / np.abs(fo).max()))
            out["kinetic_kernel"] = s.kinetic_kernel()
            s.close()
        out["max_rel_f_err"] = ferr
    out["max_rel_moment_err"] = max(moment_err(g, r) for g, r in zip(got, ref))
    return out


def run_reference(args, case, descr, rank):
    """Reference arm: the FP64 CPU oracle, untuned, on bounded samples of the workload."""
    if rank != 0:
        return 0
    per_step_budget = 90.0 / max(1, args.steps + args.warmup)  # seconds, ~90 s total
    sample, what = oracle_sample(case, per_step_budget * 8e6)
    value, secs = time_oracle(sample, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": descr, "sample": what},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{what}, {args.steps} steps after {args.warmup} warm-up "
                                   f"steps, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class Job:
    """The GPU side of one workload: a single problem (dvm.Solver) or a batch of
    tubes (dvm.Batch), with the calls the benchmark times."""

    def __init__(self, dvm, case, precision):
        self.batch = isinstance(case, list)
        if self.batch:
            self.obj = dvm.Batch(case, precision=precision)
            self.U0 = self.obj.pack([conserved(c) for c in case])
            self.points = sum(c.points for c in case)
            self.rows, self.cells = self.obj.rows, self.obj.ncells
        else:
            self.obj = dvm.Solver.from_case(case, precision=precision)
            self.U0 = conserved(case)
            self.points = case.points
            self.rows, self.cells = case.d + 2, case.ncells
        self.stream = self.obj.stream
        self.tiling = None

    def set_moments(self, U):
        self.obj.set_moments(U)

    def prepare(self, dvm, case, precision, warmup):
        self.obj.set_moments(self.U0)
        if self.batch:
            self.tiling = dvm.autotune_cached(self.obj, case, precision, dvm.HOFKS)
        self.obj.step(warmup)

    def launches_per_step(self):
        return 3 if self.batch else self.obj.launches_per_step()

    def kinetic_ms(self, steps):
        """Average kinetic-pass time, CUDA events on the launching stream."""
        if self.batch:
            return self.obj.kinetic_ms(steps)
        self.obj.profile_begin()
        self.obj.step_async(steps)
        ms, n = self.obj.profile_end()
        self.obj.sync_status()
        return ms / n


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (a replica's time: the job ends with
    the slowest replica); x itself without a process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job phase-space updates per second: every replica advances its own
    problem of `points` updates per step (weak scaling)."""
    return points * steps * world / seconds


def run_learned(args, case, descr, rank, local):
    """The learned regime path against the plain scheme on the 2D shear layer:
    updates/s of FP32 + learned, plain FP32 and plain FP64 over the same steps, and
    the L1 density error of each FP32 run against the FP64 run (the FP64 GPU form
    agrees with the oracle to 1e-12).  value = learned / plain-FP64 speedup."""
    import torch
    from paper_1212_0204_gb300 import dvm, learned

    torch.cuda.set_device(local)
    net = learned.train_for_shear_layer(n=128, nv=case.nv[0], nsnap=200, warmup=10, dv=case.dv)
    mlp_prec = dvm.BF16S if args.mlp == "bf16" else dvm.F32

    # an ideal regime detector: the fluid zones themselves (lambda = exp(-dt/tau) <
    # 5e-5, where the kinetic part lambda f of the update is below FP32 resolution
    # of the new value), given as fixed flags instead of the network's
    dt = case.dx / (case.p * case.dv)
    fluid = np.exp(-dt / np.asarray(case.tau, dtype=np.float64)) < 5e-5

    def run(precision, with_net, given=None):
        s = dvm.Solver.from_case(case, precision=precision)
        s.set_primitive(case.rho, case.u, case.T)
        if with_net:
            learned.enable(s, net, args.thr, mlp_precision=mlp_prec)
        elif given is not None:
            s.learn_enable(dvm.LEARN_GIVEN)
            s.learn_set_flags(given)
        s.step(args.warmup)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(s.stream)
        s.step_async(args.steps - args.warmup)
        stop.record(s.stream)
        stop.synchronize()
        s.sync_status()
        ms = start.elapsed_time(stop) / (args.steps - args.warmup)
        U = s.moments()
        st = s.learn_stats() if (with_net or given is not None) else None
        kin = None
        if precision == dvm.F32:
            s.profile_begin()
            s.step(3)
            kms, nk = s.profile_end()
            kin = kms / nk
        s.close()
        return U, ms, st, kin

    with ClockSampler(physical_gpu_index(local)) as clk:
        U64, ms64, _, _ = run(dvm.F64, False)
        U32, ms32, _, kin32 = run(dvm.F32, False)
        UL, msl, st, kinl = run(dvm.F32, True)
        UI, msi, sti, kini = run(dvm.F32, False, given=fluid)
    l1 = lambda U: float(np.abs(U[0] - U64[0]).sum() / np.abs(U64[0]).sum())
    pts = case.points
    ups = lambda ms: pts / (ms * 1e-3)
    peak, peak_kind = load_peaks()
    achieved = BYTES_PER_UPDATE["f32"] * pts / (kinl * 1e-3) / 1e9
    if rank != 0:
        return 0
    line = {
        "metric": "learned/plain speedup at same L1 err", "value": ups(msl) / ups(ms64), "unit": "x",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": msl,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": descr, "cells": case.ncells, "points": pts,
                   "l2": "f larger than L2 (no flush)", "threshold": args.thr,
                   "network": f"10-64-64-1 {args.mlp}, trained on 200 snapshots of the plain FP64 run at 128^2",
                   "l1_horizon_steps": args.steps},
        "learned": {"updates_per_s": ups(msl), "ms_per_step": msl, "l1_vs_fp64": l1(UL),
                    "flagged_fraction_avg": st["flagged_total"] / max(st["steps"], 1) / case.ncells,
                    "checks": st["checks"], "checked": st["checked"], "failed": st["failed"],
                    "vetoed": st["vetoed"], "written_back": st["materialised"],
                    "net_train_mse": net.train_mse, "net_val_mse": net.val_mse},
        "plain_fp32": {"updates_per_s": ups(ms32), "ms_per_step": ms32, "l1_vs_fp64": l1(U32),
                       "kinetic_ms": kin32},
        "plain_fp64": {"updates_per_s": ups(ms64), "ms_per_step": ms64},
        "ideal_flags": {"what": "fixed flags on the fluid zones (lambda < 5e-5), no network: "
                                "an upper bound on what a regime detector can skip here",
                        "flagged_fraction": float(fluid.mean()), "updates_per_s": ups(msi),
                        "ms_per_step": msi, "kinetic_ms": kini, "l1_vs_fp64": l1(UI)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "kinetic_pass (learned run)",
                     "peak_source": peak_kind, "kernel_ms": kinl},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": None,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="density_wave_3d", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--thr", type=float, default=-3.5,
                    help="shear_learned: flag threshold on the predicted log10 non-equilibrium")
    ap.add_argument("--mlp", default="bf16", choices=["bf16", "f32"],
                    help="shear_learned: network precision (bf16 = tensor cores)")
    ap.add_argument("--cells", type=int, default=None,
                    help="override the cells per dimension (small profiling captures)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    make, prec = WORKLOADS[args.workload]
    case = make()
    if args.cells and not isinstance(case, list):
        import dataclasses
        kw = {"n": args.cells} if case.d > 1 else {"nx": args.cells}
        fn = {"quadrant_2d": W.quadrant_2d, "density_wave_3d": W.density_wave_3d,
              "sod_1d": W.sod_1d}[case.name]
        small = fn(**kw, nv=case.nv[0], tau=case.tau, steps=case.steps, dv=case.dv)
        case = dataclasses.replace(small, name=case.name)
    if args.steps is None:
        args.steps = case[0].steps if isinstance(case, list) else case.steps
    args.warmup = max(3, args.warmup)
    descr = DESCR[args.workload]
    if args.impl == "reference":
        return run_reference(args, case, descr, rank)
    if args.workload == "shear_learned":
        return run_learned(args, case, descr, rank, local)

    import torch
    from paper_1212_0204_gb300 import dvm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    precision = {"f64": dvm.F64, "f32": dvm.F32, "bf16": dvm.BF16S}[prec]
    job = Job(dvm, case, precision)
    stream = job.stream
    U0 = torch.from_numpy(job.U0).contiguous().pin_memory()
    job.prepare(dvm, case, precision, args.warmup)
    launches = job.launches_per_step()

    # ---- device-timed region: K graph replays on the job's stream
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(physical_gpu_index(local)) as clk:
        barrier()
        start.record(stream)
        job.obj.step_async(args.steps)
        stop.record(stream)
        stop.synchronize()
        barrier()
    job.obj.sync_status()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    value = job_rate(job.points, args.steps, world, ms * 1e-3)

    # ---- kinetic-pass roofline: the same steps, kinetic pass bracketed by events
    kin_ms = job.kinetic_ms(args.steps)
    bytes_alg = BYTES_PER_UPDATE[prec] * job.points
    achieved = bytes_alg / (kin_ms * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    traffic = recorded_traffic(args.workload)

    # ---- end to end through the public API with host buffers: the initial
    # moments uploaded from pinned memory, then every step advanced and its
    # moments read back into pinned host memory: step i's moments are read
    # with the pipelined read-back while step i + 1 runs, and waited for
    # (status included) before step i + 2 is enqueued.
    outs = [torch.empty((job.rows, job.cells), dtype=torch.float64).pin_memory() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    job.set_moments(U0)             # H2D of the initial moments, builds f^0
    prev = None
    for i in range(args.steps):
        job.obj.step_async(1)
        t = job.obj.moments_async(outs[i & 1])   # D2H of this step's moments
        if prev is not None:
            job.obj.moments_wait(prev)           # step i - 1's moments are on the host
        prev = t
    job.obj.moments_wait(prev)
    how = ("dvm_batch_moments_async" if job.batch else "dvm_moments_async") + \
        " after each step, waited one step later"
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    mom_bytes = 8 * job.rows * job.cells
    e2e = {"value": job_rate(job.points, args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": mom_bytes / args.steps, "d2h_bytes_per_step": mom_bytes,
           "note": "initial moments uploaded once (bytes spread over the steps); every step's "
                   "moments read back to pinned host memory through " + how}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        sample, what = oracle_sample(case, 4e6)
        pts = sum(c.points for c in sample)
        nst = max(1, int(round(12.0 * 2e7 / pts)))
        v1, secs1 = time_oracle(sample, steps=nst)
        ncores = host_cores()
        try:
            vn, secsn = time_oracle_all_cores(sample, nst, ncores)
        except Exception as e:  # a report beside the number, not part of the timing
            vn, secsn, ncores = None, 0.0, 1
            print(f"all-core oracle timing unavailable: {type(e).__name__}: {e}", file=sys.stderr)
        model = cpu_model()
        if vn is not None:
            cpu = {"value": vn, "unit": UNIT, "cores": ncores, "kind": "oracle",
                   "sample": f"{what}, {nst} steps, {ncores} independent single-thread FP64 "
                             f"oracle processes at once ({secsn:.1f} s wall)",
                   "cpu_model": model, "value_1core": v1,
                   "sample_1core": f"{what}, {nst} steps, one thread ({secs1:.1f} s)"}
        else:
            cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{what}, {secs1:.1f} s of single-thread FP64 oracle",
                   "cpu_model": model}
        try:
            # the full-size problem where the oracle advances it in seconds (the same
            # lambda regime as the timed run), else the bounded sample
            if not job.batch and case.points <= 1e8:
                err = precision_error(dvm, [case], precision, False)
                err["sample"] = "the full-size problem"
            else:
                err = precision_error(dvm, sample, precision, job.batch)
                err["sample"] = what
        except Exception as e:  # the stated error is a report, not part of the timing
            err = {"unavailable": f"{type(e).__name__}: {e}"}
    else:
        err = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": descr, "cells": job.cells, "points": job.points,
                   "l2": "f larger than L2 (no flush)",
                   "parallelism": f"{world} independent replica(s)",
                   **({"tiling": job.tiling} if job.tiling else {})},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "kinetic_pass",
                     "peak_source": peak_kind,
                     "kernel_ms": kin_ms, "bytes_per_launch": bytes_alg},
        "cpu_baseline": cpu,
        "error_vs_oracle": err,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
