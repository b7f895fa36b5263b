#!/usr/bin/env python3
"""Throughput of the WENO-ZN SSP-RK3 solver for the 2D Euler equations (FP64) on GB300.

One step = one SSP-RK3 step (three stages: LF-speed reduction, x and y interface fluxes
with characteristic WENO-ZN reconstruction, flux difference and stage update) over the
whole grid of the seeded four-quadrant Riemann problem, outflow boundaries, CFL 0.5.
Metric: cell-updates per second (one cell advanced by one RK3 step).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--n 4096]

Multi-GPU: each rank advances its own independent problem (replicas, weak scaling); the
only collectives are the timing barrier and a max-reduction of the elapsed time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WENO-ZN cell-updates/s (2D Euler FP64)"
UNIT = "cell-updates/s"

# FP64 peak of one GB300 derived from the nominal FP64 rate (1.25 TFLOP/s), 152 SMs and
# the 2070 MHz maximum SM clock: 2 FP64 FMA lanes per SM per clock.
FP64_LANES_PER_SM = 2
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_GFLOPS = 2 * FP64_LANES_PER_SM * SMS * SM_MAX_MHZ / 1e3   # 1258.6

# DRAM bytes (read + write) of one 4096x4096 launch of the step's flux kernel (both sweeps of
# a stage) from the ncu capture summarised in profiles/flux_xy_kernel_euler2d_2560.md (scaled
# by the interface count), valid only for the kernel sources with this hash prefix; any other
# source reports null.
TRAFFIC_CAPTURE = {"sha256_16": "8caed8a5cce072a2", "n": 4096, "bytes": 2040.8e6, "capture_n": 2560,
                   "profile": "profiles/flux_xy_kernel_euler2d_2560.md",
                   "fp64_pipe": {"xy": 0.892, "x": 0.891, "y": 0.892}}   # ncu FP64-pipe busy, same captures


def hbm_peak() -> tuple:
    """Measured HBM copy bandwidth of the GB300s (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("flux_kernels.cu", "wenozn_device.cuh", "euler_device.cuh"):
        with open(os.path.join(ROOT, "paper_2004_07954_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Units all ranks processed per second: every rank advances its own replica."""
    return world * steps * units_per_rank_step / (ms_max / 1e3)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=4096, help="grid is n x n")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--kernel-reps", type=int, default=5, help="launches per flux kernel timing")
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-fd-dirs", type=int, default=20)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-euler1d", action="store_true")
    ap.add_argument("--no-euler2d-1024", action="store_true")
    ap.add_argument("--no-reconstruct", action="store_true")
    ap.add_argument("--only", choices=["batched", "adjoint", "variants", "euler1d", "euler2d_1024", "reconstruct"],
                    default=None,
                    help="run only this part and print its object (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU work of the baseline sample")
    return ap.parse_args()


# Algorithmic FP64 operations (one per add, mul, div, sqrt of the scheme as the paper writes
# it, comparisons apart) per unit, as the oracle's op-counting instantiation counts them
# (oracle.opcount_parts; tests/test_opcount.py checks these tables against it):
# (interface flux, split fluxes and Roe ingredients per cell and sweep, LF-speed evaluation
# per cell (both directions in 2D, with the per-field speeds where the splitting needs them),
# flux difference per cell (all directions), RK3 combination per cell and step).
OPS_2D = {  # (weights, split): per-unit counts, 2D Euler
    (0, 0): (1090.0, 42.0, 28.0, 20.0, 48.0),     # WENO-ZN, global LF (the default scheme)
    (0, 1): (1274.0, 22.0, 58.0, 20.0, 48.0),     # per-field LF
    (0, 2): (1274.0, 22.0, 28.0, 20.0, 48.0),     # local LF
    (0, 3): (1090.0, 152.0, 28.0, 20.0, 48.0),    # Steger-Warming
}
OPS_1D_CELL_UPDATE = 2448.0     # 1D Euler, default scheme, per cell-update (large grid)
OPS_1D = (755.0, 32.0, 11.0, 6.0)   # 1D Euler: interface, cell per sweep, LF speed, difference
RECON_FLOPS = 85.0                   # one WENO-ZN reconstruction f^_{i+1/2} (wenozn_reconstruct, per point)


def algorithmic_flops(nx: int, ny: int, weights: int = 0, split: int = 0) -> dict:
    """Algorithmic FP64 operations of one 2D RK3 step and of its flux launches."""
    iface, cell, speed, diff, rk = OPS_2D[(weights, split)]
    x_flux = iface * (nx + 1) * ny + cell * nx * ny
    y_flux = iface * nx * (ny + 1) + cell * nx * ny
    per_stage = x_flux + y_flux + (speed + diff) * nx * ny
    step = 3 * per_stage + rk * nx * ny
    return {"x_flux": x_flux, "y_flux": y_flux, "step": step,
            "per_cell_update": step / (nx * ny), "per_interface": iface}


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        smi = shutil.which("nvidia-smi")
        if not smi:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([smi, f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def bench_batched(wenozn, inputs, seed: int, K: int, B: int = 2048) -> dict:
    """Batched ragged 1D Euler: B instances, sizes log-uniform in [128, 16384], one persistent
    launch per RK stage, K RK3 steps captured in one CUDA graph; against one launch sequence
    per instance (wenozn_rk3_step on each instance), eager and graph-captured."""
    import numpy as np
    import torch
    sizes, offsets, U0 = inputs.euler1d_batch(B, seed)
    dx = 10.0 / sizes
    cells = int(offsets[-1])
    U = torch.from_numpy(U0).cuda()
    bt = wenozn.Batch(offsets, dx, U)
    tune_ms = bt.tune(U.clone(), steps=2)
    bt.init(U)
    graph = bt.capture(U, K)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / K
    status = bt.status()
    del graph
    # baseline: every instance on its own (one wenozn_rk3_step launch sequence each)
    solvers, states = [], []
    for b in range(B):
        n = int(sizes[b])
        p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_1D, n, 1, float(dx[b]), 1.0)
        solvers.append(wenozn.Solver(p))
        states.append(torch.from_numpy(U0[:, offsets[b]:offsets[b + 1]].reshape(3, 1, n).copy()).cuda())

    def per_instance_step():
        for S, u in zip(solvers, states):
            S.step(u)
    per_instance_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for _ in range(2):
        per_instance_step()
    e1.record()
    torch.cuda.synchronize()
    eager_ms = (time.perf_counter() - t0) * 1e3 / 2
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        per_instance_step()
    g2.replay()
    torch.cuda.synchronize()
    e0.record()
    g2.replay()
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    del g2, solvers, states
    shape = wenozn.wenozn_batch_shape(bt.bp.shape)
    flops = OPS_1D_CELL_UPDATE * cells          # algorithmic flops per cell-update
    return {"workload": f"{B} independent 1D Euler problems (seeded Shu-Osher family), sizes log-uniform "
                        f"in [128, 16384], {cells} cells, outflow, per-instance CFL 0.5 step",
            "metric": "cell-updates/s", "value": cells / (ms_step / 1e3), "ms_per_step": ms_step,
            "steps_per_graph": K, "launches_per_step": 3, "tuned_shape": {"tile": shape[0], "threads": shape[1]},
            "tune_ms_per_step": [round(x, 3) for x in tune_ms],
            "fp64_frac": round(flops / (ms_step / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
            "per_instance_baseline": {"launches_per_step": 7 * B, "eager_ms_per_step": round(eager_ms, 2),
                                      "graph_ms_per_step": round(graph_ms, 2),
                                      "speedup_vs_eager": round(eager_ms / ms_step, 1),
                                      "speedup_vs_graph": round(graph_ms / ms_step, 2)},
            "device_status": status}


def bench_euler1d(wenozn, inputs, seed: int, n: int = 1 << 20, K: int = 100) -> dict:
    """Single 1D Euler problem of n cells (the seeded Shu-Osher family, outflow, CFL 0.5):
    K chained RK3 steps in one call after 3 warm-up steps, CUDA events; the x-flux kernel
    timed alone for its FP64 fraction (algorithmic flops of the oracle's count)."""
    import torch
    U0 = inputs.euler1d_ic(n, seed)
    p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_1D, n, 1, 10.0 / n, 1.0)
    U = torch.from_numpy(U0).cuda()
    S = wenozn.Solver(p)
    S.steps(U, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S.steps(U, K)
    e1.record()
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / K
    status = S.status()
    alpha = torch.zeros(2, dtype=torch.float64, device="cuda")
    wenozn.wenozn_max_wavespeed(p, U, alpha)
    buf = torch.empty(wenozn.flux_shape(p, 0), dtype=torch.float64, device="cuda")
    wenozn.wenozn_flux(p, U, alpha, 0, buf)
    reps = 20
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        wenozn.wenozn_flux(p, U, alpha, 0, buf)
    e1.record()
    torch.cuda.synchronize()
    flux_ms = e0.elapsed_time(e1) / reps
    iface, cell, _, _ = OPS_1D
    flux_flops = iface * (n + 1) + cell * n
    return {"workload": f"1D Euler, {n} cells, seeded Shu-Osher family (seed {seed}), outflow, CFL 0.5, "
                        f"{K} chained SSP-RK3 steps",
            "metric": "cell-updates/s", "value": n / (ms_step / 1e3), "ms_per_step": round(ms_step, 4),
            "fp64_frac": round(OPS_1D_CELL_UPDATE * n / (ms_step / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
            "flux_kernel": {"kernel": "flux_kernel<3,0> (507-interface tiles)", "ms": round(flux_ms, 4),
                            "frac": round(flux_flops / (flux_ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4)},
            "device_status": status}


def bench_reconstruct(wenozn, seed: int, n: int = 1 << 27, reps: int = 10) -> dict:
    """The reconstruction entry point alone (wenozn_reconstruct) on n points of seeded data
    with jumps (larger than L2: 1 GiB in, 1 GiB out at 2^27): both sides, CUDA events."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    f = torch.rand(n + 6, dtype=torch.float64, device="cuda", generator=g)
    f += torch.floor(torch.linspace(0.0, 64.0, n + 6, dtype=torch.float64, device="cuda"))   # 64 steps
    out = {}
    for side in (1, -1):
        fhat = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        wenozn.wenozn_reconstruct(f, fhat, side)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            wenozn.wenozn_reconstruct(f, fhat, side)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        pts = (n + 1) / (ms / 1e3)
        hbm, _ = hbm_peak()
        out["plus" if side > 0 else "minus"] = {
            "ms": round(ms, 4), "points_per_s": pts,
            "fp64_frac": round(RECON_FLOPS * pts / 1e9 / FP64_PEAK_GFLOPS, 4),
            "hbm_frac": round(16.0 * pts / 1e9 / hbm, 4) if hbm else None}
        del fhat
    return {"workload": f"wenozn_reconstruct on {n} points of seeded uniform data with 64 unit jumps, eps 1e-40, A 10",
            "bound": "FP64 pipe (85 algorithmic flops against 16 bytes per point)", **out}


def bench_euler2d(wenozn, inputs, seed: int, n: int, K: int, reps: int = 5) -> dict:
    """The headline workload on an n x n grid: K chained RK3 steps after 3 warm-up steps
    (CUDA events on the launching stream), and the flux kernel of a stage alone (both sweeps
    in one launch, as the step runs it; and each sweep alone) for its FP64 fraction."""
    import torch
    p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_2D, n, n, 1.0 / n, 1.0 / n)
    U = torch.from_numpy(inputs.euler2d_ic(n, n, seed)).cuda()
    S = wenozn.Solver(p)
    S.steps(U, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S.steps(U, K)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    status = S.status()
    alpha = torch.zeros(2, dtype=torch.float64, device="cuda")
    wenozn.wenozn_max_wavespeed(p, U, alpha)
    kern = {}
    for d in (2, 0, 1):
        buf = torch.empty(wenozn.flux_shape(p, d), dtype=torch.float64, device="cuda")
        wenozn.wenozn_flux(p, U, alpha, d, buf)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            wenozn.wenozn_flux(p, U, alpha, d, buf)
        e1.record()
        torch.cuda.synchronize()
        kern[d] = e0.elapsed_time(e1) / reps
    fl = algorithmic_flops(n, n)
    xy = fl["x_flux"] + fl["y_flux"]
    return {"workload": f"2D Euler {n}x{n} seeded four-quadrant Riemann problem (seed {seed}), outflow, "
                        f"CFL 0.5, {K} chained SSP-RK3 steps",
            "metric": "cell-updates/s", "value": n * n / (ms / 1e3), "ms_per_step": round(ms, 4),
            "step_frac": round(fl["step"] / (ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
            "xy_flux": {"ms": round(kern[2], 4), "frac": round(xy / (kern[2] / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4)},
            "x_flux": {"ms": round(kern[0], 4), "frac": round(fl["x_flux"] / (kern[0] / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4)},
            "y_flux": {"ms": round(kern[1], 4), "frac": round(fl["y_flux"] / (kern[1] / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4)},
            "device_status": status}


VARIANTS = [("weno_z", 1, 0), ("jiang_shu", 3, 0), ("per_field_lf", 0, 1), ("local_lf", 0, 2),
            ("steger_warming", 0, 3)]


def bench_variants(wenozn, inputs, seed: int, n: int = 4096, K: int = 3) -> dict:
    """The variant weight functions and flux splittings (generic kernels) on the benchmark's
    2D Euler workload: K RK3 steps after one warm-up step each, CUDA events; the default
    scheme timed the same way for the ratio.  The FP64 fraction uses the oracle's operation
    count of each splitting (weight variants: none, since the oracle also evaluates the
    WENO-ZN quantities for them)."""
    import torch
    U0 = torch.from_numpy(inputs.euler2d_ic(n, n, seed)).cuda()
    out = {"workload": f"2D Euler {n}x{n}, the benchmark's seeded four-quadrant problem, outflow, CFL 0.5",
           "steps": K}
    base_ms = None
    for name, weights, split in [("default", 0, 0)] + VARIANTS:
        eps = 1e-6 if weights == 3 else 1e-40
        p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_2D, n, n, 1.0 / n, 1.0 / n, weights=weights,
                                       split=split, eps=eps)
        S = wenozn.Solver(p)
        U = U0.clone()
        S.steps(U, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        S.steps(U, K)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        rec = {"weights": weights, "split": split, "ms_per_step": round(ms, 3),
               "cell_updates_per_s": n * n / (ms / 1e3), "device_status": S.status()}
        if (weights, split) in OPS_2D:
            fl = algorithmic_flops(n, n, weights, split)["step"]
            rec["fp64_frac"] = round(fl / (ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4)
        if base_ms is None:
            base_ms = ms
        else:
            rec["time_vs_default"] = round(ms / base_ms, 3)
        out[name] = rec
        del S, U
        torch.cuda.empty_cache()
    return out


def bench_adjoint(wenozn, inputs, seed: int, n: int = 8192, steps: int = 2000, fd_dirs: int = 20) -> dict:
    """Discrete adjoint of a fixed-step rollout of the 1D Euler equations: loss
    1/2 ||rho(T) - rho_target||^2, gradient with respect to the initial conserved state.
    Times the forward rollout, the adjoint with every state kept and with a checkpoint
    every 50 steps, and checks the gradient against central differences (h = 1e-7) of the
    GPU forward along `fd_dirs` seeded smooth directions.  (Cell-to-cell noise directions
    are not checked by differences: on this smooth state the squared fourth difference tau8
    is of order dx^8, so a perturbation of size h ~ 1e-7 already dominates it and the loss
    is far from linear on any usable h; the test suite checks such directions against the
    oracle's exact forward-mode derivative instead.)"""
    import numpy as np
    import torch
    from paper_2004_07954_gb300.rollout import cfl_step, rollout
    p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_1D, n, 1, 10.0 / n, 1.0, bc_x=wenozn.WENOZN_BC_PERIODIC)
    ws = wenozn.vjp_workspace(p)
    U0 = torch.from_numpy(inputs.adjoint_ic(n, seed)).cuda()
    dt = cfl_step(p, U0, ws)
    with torch.no_grad():
        target = rollout(torch.from_numpy(inputs.adjoint_ic(n, seed + 1)).cuda(), p, dt, steps, ws=ws)[0].clone()

    def fwd_only(U):
        U = U.clone()
        wenozn.wenozn_rk3_run(p, U, steps, ws, dt)      # the fastest forward: chained steps
        return U

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    fwd_only(U0)
    _, t_fwd = timed(lambda: fwd_only(U0))
    res = {}
    for every in (1, 50):
        def fwd_bwd():
            U = U0.clone().requires_grad_(True)
            UT = rollout(U, p, dt, steps, checkpoint_every=every, ws=ws)
            loss = 0.5 * ((UT[0] - target) ** 2).sum()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            (g,) = torch.autograd.grad(loss, U)
            torch.cuda.synchronize()
            return g, loss, time.perf_counter() - t1
        fwd_bwd()
        (g, loss, t_bwd), t_all = timed(fwd_bwd)
        res[every] = {"forward_with_checkpoints_s": round(t_all - t_bwd, 4), "adjoint_s": round(t_bwd, 4),
                      "adjoint_over_forward": round(t_bwd / t_fwd, 3)}
    grad = g.cpu().numpy()
    u0 = U0.cpu().numpy()
    gen = np.random.default_rng(seed + 7)
    h = 1e-7
    x = (np.arange(n) + 0.5) * (10.0 / n) - 5.0
    checks = {}

    def fd_at(v, hh):
        vt = torch.from_numpy(v).cuda()
        lp = 0.5 * float(((fwd_only(U0 + hh * vt)[0] - target) ** 2).sum())
        lm = 0.5 * float(((fwd_only(U0 - hh * vt)[0] - target) ** 2).sum())
        return (lp - lm) / (2 * hh)

    with torch.no_grad():
        worst = 0.0
        for _ in range(fd_dirs):
            # a few random Fourier modes per variable, scaled like U0
            v = np.zeros_like(u0)
            for k in range(3):
                for m in range(1, 5):
                    v[k, 0] += gen.normal() * np.sin(2 * np.pi * m * x / 10 + gen.uniform(0, 2 * np.pi))
                v[k, 0] *= np.abs(u0[k, 0]).mean()
            gv = float(np.sum(grad * v))
            fd = fd_at(v, h)
            worst = max(worst, abs(gv - fd) / abs(fd))
        if fd_dirs > 0:
            checks["smooth_directions"] = {"directions": fd_dirs, "max_rel_err": worst}
    return {"workload": f"1D Euler N={n}, seeded smooth periodic multi-wave state, {steps} SSP-RK3 steps of "
                        f"fixed dt (CFL 0.5 of U0), loss 1/2||rho(T) - rho_target||^2, rho_target from seed+1",
            "forward_s": round(t_fwd, 4), "store_all": res[1], "checkpoint_every_50": res[50],
            "loss": float(loss.detach()), "fd_check": {"h": h, **checks},
            "reverse_scaling": adjoint_scaling(wenozn, inputs, seed)}


def adjoint_scaling(wenozn, inputs, seed: int, sizes=(8192, 1 << 17, 1 << 20), steps: int = 10) -> list:
    """Forward and reverse step times on lines of several lengths (the same seeded smooth
    state, fixed dt): one chained forward call (wenozn_rk3_run), and the reverse of a kept
    segment (wenozn_rk3_vjp_run); lines of 10240 cells and more take the
    one-thread-per-interface stage kernel."""
    import torch
    out = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_us(fn):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(3):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e3 / steps)
        return best

    for n in sizes:
        p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_1D, n, 1, 10.0 / n, 1.0, bc_x=wenozn.WENOZN_BC_PERIODIC)
        ws = wenozn.vjp_workspace(p)
        U0 = torch.from_numpy(inputs.adjoint_ic(n, seed)).cuda()
        dt = 0.5 * wenozn.wenozn_cfl_dt(p, U0, ws)
        X = torch.empty((steps + 1,) + tuple(U0.shape), dtype=torch.float64, device="cuda")
        S1, S2 = torch.empty_like(X[:steps]), torch.empty_like(X[:steps])
        A = torch.empty(3 * steps + 1, dtype=torch.float64, device="cuda")
        X[0].copy_(U0)
        wenozn.wenozn_rk3_run_keep(p, X, S1, S2, A, steps, dt, ws)
        U = U0.clone()
        fwd = timed_us(lambda: wenozn.wenozn_rk3_run(p, U, steps, ws, dt))
        lam = torch.ones_like(U0)
        rev = timed_us(lambda: wenozn.wenozn_rk3_vjp_run(p, X, S1, S2, A, steps, dt, lam.clone(), ws))
        out.append({"n": n, "forward_step_us": round(fwd, 1), "reverse_step_us": round(rev, 1),
                    "reverse_over_forward": round(rev / fwd, 2)})
        del X, S1, S2
    return out


def cpu_baseline(n_full: int, seed: int, target_s: float, steps: int = 1) -> dict:
    """The CPU oracle as it stands, on the host's cores, on a bounded sample of the same
    workload: the same problem family on an m x m grid, m chosen so the sample takes
    about `target_s` seconds."""
    import numpy as np  # noqa: F401
    from oracle import oracle as O
    from paper_2004_07954_gb300 import inputs
    O.build()
    cores = O.num_threads()
    m = 128
    U = inputs.euler2d_ic(m, m, seed)
    P = O.problem(O.EULER2D, m, m, dx=1.0 / m, dy=1.0 / m)
    t0 = time.perf_counter()
    O.rk3_step(P, U)
    per_cell = (time.perf_counter() - t0) / (m * m)
    m = int(math.sqrt(max(1.0, target_s / max(per_cell, 1e-9) / steps)))
    m = max(128, min(n_full, m))
    U = inputs.euler2d_ic(m, m, seed)
    P = O.problem(O.EULER2D, m, m, dx=1.0 / m, dy=1.0 / m)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = O.rk3_step(P, U)
    el = time.perf_counter() - t0
    # the same oracle on one core, one step on a 512 x 512 sample
    m1 = min(512, n_full)
    U1 = inputs.euler2d_ic(m1, m1, seed)
    P1 = O.problem(O.EULER2D, m1, m1, dx=1.0 / m1, dy=1.0 / m1)
    O.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        O.rk3_step(P1, U1)
        el1 = time.perf_counter() - t0
    finally:
        O.set_num_threads(cores)
    return {"value": steps * m * m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} SSP-RK3 step(s) of the same seeded four-quadrant 2D Euler problem on a "
                      f"{m}x{m} grid (plain FP64 C++ oracle, OpenMP over grid lines), {el:.1f} s",
            "single_core": {"value": m1 * m1 / el1, "cores": 1,
                            "sample": f"1 SSP-RK3 step on a {m1}x{m1} grid, {el1:.2f} s"}}


def run_reference(args, rank: int):
    """Reference arm: the CPU oracle timed on this host's cores, bounded sample per step."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2004_07954_gb300 import inputs
    O.build()
    cores = O.num_threads()
    # the benchmark's own grid when warmup + steps fit in about three minutes (a 4096^2 step
    # takes about 3 s on 16 cores), else the largest square sample that does; the rate is
    # calibrated on one 512^2 step
    m = min(512, args.n)
    U = inputs.euler2d_ic(m, m, args.seed)
    P = O.problem(O.EULER2D, m, m, dx=1.0 / m, dy=1.0 / m)
    t0 = time.perf_counter()
    O.rk3_step(P, U)
    per_cell = (time.perf_counter() - t0) / (m * m)
    budget = 200.0 / max(1, args.steps + args.warmup)
    m = max(64, min(args.n, int(math.sqrt(budget / max(per_cell, 1e-9)))))
    U = inputs.euler2d_ic(m, m, args.seed)
    P = O.problem(O.EULER2D, m, m, dx=1.0 / m, dy=1.0 / m)
    for _ in range(args.warmup):
        U, _ = O.rk3_step(P, U)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _ = O.rk3_step(P, U)
    el = time.perf_counter() - t0
    value = args.steps * m * m / el
    sample = (f"each step: one SSP-RK3 step of the seeded four-quadrant 2D Euler problem on a {m}x{m} "
              + ("grid (the whole workload)" if m == args.n else
                 f"grid (bounded sample of the {args.n}x{args.n} workload)")
              + f", plain FP64 C++ oracle on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"2D Euler {args.n}x{args.n} four-quadrant Riemann, seed {args.seed}, "
                                   "outflow, CFL 0.5, one SSP-RK3 step per step", "sample_grid": [m, m]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2004_07954_gb300 import build as _b
    from paper_2004_07954_gb300 import inputs, wenozn

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _b.build()
    if args.only is not None:
        if args.only == "batched":
            part = bench_batched(wenozn, inputs, args.seed + rank, args.batched_steps)
        elif args.only == "variants":
            part = bench_variants(wenozn, inputs, args.seed + rank, args.n)
        elif args.only == "euler1d":
            part = bench_euler1d(wenozn, inputs, args.seed + rank)
        elif args.only == "euler2d_1024":
            part = bench_euler2d(wenozn, inputs, args.seed + rank, 1024, 100)
        elif args.only == "reconstruct":
            part = bench_reconstruct(wenozn, args.seed + rank)
        else:
            part = bench_adjoint(wenozn, inputs, args.seed + rank, steps=args.adjoint_steps,
                                 fd_dirs=args.adjoint_fd_dirs)
        if rank == 0:
            print(json.dumps({"part": args.only, **part}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.n
    p = wenozn.wenozn_problem_init(wenozn.WENOZN_EULER_2D, n, n, 1.0 / n, 1.0 / n)
    U0 = inputs.euler2d_ic(n, n, args.seed + rank)          # one independent problem per rank
    U = torch.from_numpy(U0).cuda()
    S = wenozn.Solver(p)
    stream = torch.cuda.current_stream()

    S.steps(U, args.warmup)
    torch.cuda.synchronize()
    if S.status() != 0:
        raise RuntimeError("non-finite state during warm-up")

    clocks = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    S.steps(U, args.steps)          # chained RK3 steps (wenozn_rk3_run), CFL step on the device
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    status = S.status()
    value = job_throughput(n * n, args.steps, world, ms)

    # ---- dominant kernels, timed live on the launching stream ------------------------
    alpha = torch.zeros(2, dtype=torch.float64, device="cuda")
    wenozn.wenozn_max_wavespeed(p, U, alpha)
    # the step's flux kernel (both sweeps of a stage in one launch, direction 2), and each
    # sweep alone for the split
    kern = {}
    for d in (2, 0, 1):
        buf = torch.empty(wenozn.flux_shape(p, d), dtype=torch.float64, device="cuda")
        wenozn.wenozn_flux(p, U, alpha, d, buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.kernel_reps):
            wenozn.wenozn_flux(p, U, alpha, d, buf)
        b.record(stream)
        torch.cuda.synchronize()
        kern[d] = a.elapsed_time(b) / args.kernel_reps
        del buf
    fl = algorithmic_flops(n, n)
    achieved = (fl["x_flux"] + fl["y_flux"]) / (kern[2] / 1e3) / 1e9
    # the FP64 rate pure FMA register arithmetic reaches on this GPU, beside the nominal peak
    probe = max(wenozn.wenozn_fp64_fma_rate(1 << 17, stream) for _ in range(3))
    captured = kernel_source_hash() == TRAFFIC_CAPTURE["sha256_16"] and n == TRAFFIC_CAPTURE["n"]
    traffic = TRAFFIC_CAPTURE["bytes"] if captured else None
    hbm_gbs, hbm_src = hbm_peak()
    roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4), "traffic": traffic,
                "kernel": "flux_xy_kernel (a stage's x and y interface fluxes in one launch, as the step runs them)",
                "peak_source": "derived: 2 FP64 FMA/SM/clk x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s FP64)",
                "kernel_ms": {"xy_flux": round(kern[2], 3), "x_flux": round(kern[0], 3), "y_flux": round(kern[1], 3)},
                "x_flux_frac": round(fl["x_flux"] / (kern[0] / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
                "y_flux_frac": round(fl["y_flux"] / (kern[1] / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
                "step_frac": round(fl["step"] * world * args.steps / (ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS / world, 4),
                "algorithmic_flops_per_cell_update": round(fl["per_cell_update"], 1),
                "fp64_fma_probe": {"gflops": round(probe, 1), "of_peak": round(probe / FP64_PEAK_GFLOPS, 4),
                                   "frac_of_probe": round(achieved / probe, 4),
                                   "what": "pure FP64 FMA register arithmetic, 2 blocks x 256 threads per SM "
                                           "(wenozn_fp64_fma_rate), measured in this run"},
                # ncu counters of the same kernels (null once the kernel sources changed)
                "fp64_pipe_ncu": TRAFFIC_CAPTURE["fp64_pipe"] if captured else None,
                "traffic_source": {"measured_in_this_run": False,
                                   "capture": f"ncu, {TRAFFIC_CAPTURE['capture_n']}^2 case of the same kernel "
                                              f"({TRAFFIC_CAPTURE['profile']})",
                                   "scaled": f"by the interface count to {n}^2",
                                   "kernel_sources_sha256_16": TRAFFIC_CAPTURE["sha256_16"],
                                   "sources_match": captured},
                "dram": None if traffic is None else {
                    "gbs": round(traffic / (kern[2] / 1e3) / 1e9, 1), "peak_gbs": hbm_gbs,
                    "frac": round(traffic / (kern[2] / 1e3) / 1e9 / hbm_gbs, 5), "peak_source": hbm_src}}

    # ---- end to end: host buffers, copies inside the timed region --------------------
    # One library call (wenozn_rk3_stream_host) takes the K steps' states from pinned host
    # memory and returns their results to pinned host memory: each state is uploaded on an
    # upload stream into one of two device staging buffers, stepped on the compute stream and
    # downloaded on a download stream, so the copies of one state overlap the step of the
    # next; the call is ordered after the work on the compute stream and before what follows.
    host_in = torch.from_numpy(U0).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    bufs = [torch.empty_like(U) for _ in range(2)]
    up_s, down_s = torch.cuda.Stream(), torch.cuda.Stream()
    ke = max(1, args.e2e_steps)

    def e2e_run(k_steps):
        wenozn.wenozn_rk3_stream_host(p, [host_in] * k_steps, [host_out[k % 2] for k in range(k_steps)],
                                      bufs[0], bufs[1], S.ws, stream=stream, upload_stream=up_s,
                                      download_stream=down_s)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(ke)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = max_over_ranks(e0.elapsed_time(e1), world)
    nbytes = U.numel() * U.element_size()
    e2e = {"value": job_throughput(n * n, ke, world, ems), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": ke, "device_status": S.status(),
           "api": "wenozn_rk3_stream_host (one C-ABI call: host states in, host results out)",
           "copies": "pinned host <-> device on an upload and a download stream inside the call, "
                     "overlapping the neighbouring states' steps"}
    del bufs

    def part(skip, fn, *a, **kw):
        """A secondary measurement; its failure is reported in its own object, the headline
        line is printed regardless."""
        if skip:
            return None
        try:
            return fn(*a, **kw)
        except Exception as exc:          # noqa: BLE001 - recorded, not hidden
            return {"error": f"{type(exc).__name__}: {exc}"[:300]}

    batched = part(args.no_batched, bench_batched, wenozn, inputs, args.seed + rank, args.batched_steps)
    euler1d = part(args.no_euler1d, bench_euler1d, wenozn, inputs, args.seed + rank)
    euler2d_1024 = part(args.no_euler2d_1024, bench_euler2d, wenozn, inputs, args.seed + rank, 1024, 100)
    reconstruct = part(args.no_reconstruct, bench_reconstruct, wenozn, args.seed + rank)
    variants = part(args.no_variants, bench_variants, wenozn, inputs, args.seed + rank, n)
    adjoint = part(args.no_adjoint, bench_adjoint, wenozn, inputs, args.seed + rank,
                   steps=args.adjoint_steps, fd_dirs=args.adjoint_fd_dirs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, args.seed, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"2D Euler {n}x{n} seeded four-quadrant Riemann problem "
                                       f"(seed {args.seed} + rank), outflow BC, CFL 0.5, gamma 1.4",
                           "grid": [n, n], "step": "one SSP-RK3 step (3 stages)",
                           "parallelism": f"{world} independent replica(s), one per GPU",
                           "l2": "inputs larger than L2 (512 MiB per state buffer at 4096^2), no flush",
                           "device_status": status},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "batched": batched, "euler1d": euler1d, "euler2d_1024": euler2d_1024, "reconstruct": reconstruct, "variants": variants, "adjoint": adjoint,
                "gpu_launches": 6 * args.steps + 1, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
