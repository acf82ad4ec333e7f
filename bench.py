"""Benchmark of the fused BGK collide-and-stream path on GB300.

Default workload: the D3Q19 lid-driven cavity 128^3 (halfway bounce-back on five
walls, moving lid u = 0.05 on the whole top plane, Re = 400 through tau with
L = 126, rho = 1, u = 0 plus seeded 1e-6 uniform population noise), FP32
populations, 2000 collide-and-stream steps.  One bench step = the whole workload:
equilibrium initialisation from the resident input fields, 2000 steps, and the
lattice statistics of the last collision (fused into its kernel).

Metric: MLUPS (million fluid-cell updates per second), with the HBM roofline of
the step kernel (152 algorithmic bytes per fluid-cell update in FP32: 19
populations read once and written once).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-variants]

--impl reference times the FP64 CPU oracle (the plain reference implementation of
the same map) on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) each rank runs an independent replica on its own GPU
(the path has no exchange step on one lattice per GPU); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_11752_gb300 import inputs as I  # noqa: E402

N_SIDE = 128
LBM_STEPS = 2000
LID = 0.05
TAU = I.cavity_tau(N_SIDE, 400.0, LID)
SEED = 1
METRIC = "MLUPS"
# GB300 HBM3e bandwidth as specified (the roofline's `peak` is the measured copy bandwidth instead; kernels here
# reach slightly above that copy figure on large all-fluid lattices, so both fractions are reported)
NOMINAL_HBM_GBS = 7900.0
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")


def workload_config():
    return {"workload": f"D3Q19 BGK lid-driven cavity {N_SIDE}^3, halfway bounce-back on 5 walls, "
                        f"moving lid u={LID}, Re=400 (tau={TAU:.6f}, L={N_SIDE - 2}), rho=1 u=0 + "
                        f"1e-6 seeded population noise, {LBM_STEPS} steps per bench step",
            "lattice": "D3Q19", "cells": N_SIDE ** 3, "fluid_cells": (N_SIDE - 2) ** 3,
            "lbm_steps_per_step": LBM_STEPS, "storage": "f32", "scheme": None,
            "l2_policy": "inputs larger than L2: two 159 MB population buffers + 2 MB material per "
                         "LBM step (318 MB streamed per step vs 129 MB L2)"}


# --------------------------------------------------------------------------------------
# distributed plumbing
# --------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples next to the run's other outputs when OLB_CLOCKS_DIR is set, else in
        # the temp directory; the JSON line carries their summary
        self.path = os.path.join(os.environ.get("OLB_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"olb_clocks_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in ("paper_2307_11752_gb300/csrc/olb_kernels.cuh", "paper_2307_11752_gb300/csrc/olb_pair.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key: str, units: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, scaled
    to `units` fluid cells; None when the kernel source changed since the capture."""
    try:
        with open(PROFILE_TRAFFIC) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    entry = rec.get(kernel_key)
    if not entry or entry.get("source_sha") != kernel_source_sha():
        return None
    return float(entry["dram_bytes_per_fluid_cell"]) * units


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def make_cavity(olb, torch, dtype="f32", scheme="pull", n=N_SIDE):
    m = I.cavity(n)
    lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype=dtype, scheme=scheme)
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 0)
    lat.set_wall_velocity(I.LID, (LID, 0.0, 0.0))
    lat.set_bgk(I.cavity_tau(n, 400.0, LID))
    noise = torch.from_numpy(I.population_noise(SEED, 19, m, 1e-6).reshape(-1)).cuda()
    return lat, m, noise


def run_workload(lat, noise, steps=LBM_STEPS):
    lat.init_equilibrium()
    lat.perturb(noise)
    return lat.step_stats(steps)


def time_device(torch, lat, noise, K, W, steps=LBM_STEPS, flush=None):
    for _ in range(W):
        run_workload(lat, noise, steps)
    torch.cuda.synchronize()
    t0, k0 = lat.counters()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(lat.stream)
    for _ in range(K):
        stats = run_workload(lat, noise, steps)
    end.record(lat.stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    t1, k1 = lat.counters()
    return ms, k1 - k0, stats


def time_step_kernel(torch, lat, steps):
    """Average duration of the step kernel alone: CUDA events around `steps`
    back-to-back olb_step launches on the lattice's stream."""
    lat.step(4)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(lat.stream)
    lat.step(steps)
    end.record(lat.stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / steps


def e2e_run(olb, torch, m, K):
    """Same workload through the C ABI with host (pinned) buffers: the initial
    fields go host -> device inside every step, the moments come back to the host."""
    n = N_SIDE
    lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype="f32", scheme="pull")
    lat.set_material(np.ascontiguousarray(m.reshape(-1)), 0)
    lat.set_wall_velocity(I.LID, (LID, 0.0, 0.0))
    lat.set_bgk(TAU)
    cells = n ** 3
    rho_h = torch.ones(cells, dtype=torch.float64).pin_memory()
    u_h = torch.zeros(3 * cells, dtype=torch.float64).pin_memory()
    noise_h = torch.from_numpy(I.population_noise(SEED, 19, m, 1e-6).reshape(-1)).pin_memory()
    rho_o = torch.empty(cells, dtype=torch.float64).pin_memory()
    u_o = torch.empty(3 * cells, dtype=torch.float64).pin_memory()

    def one():
        lat.init_equilibrium(rho_h, u_h)
        lat.perturb(noise_h)
        lat.step(LBM_STEPS)
        lat.moments(rho_o, u_o)

    one()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(K):
        one()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t
    h2d = (rho_h.numel() + u_h.numel() + noise_h.numel()) * 8
    d2h = (rho_o.numel() + u_o.numel()) * 8
    lat.close()
    return sec, h2d, d2h


def variants(olb, torch):
    """Short measurements of the other storage types, the AA pattern, the 3D
    Taylor-Green vortex at 512^3 and the adjoint (channel 256x128x128)."""
    out = {}
    peak, _ = measured_peak_gbs()
    fluid = (N_SIDE - 2) ** 3
    for dtype, scheme in (("f32", "aa"), ("f16", "pull"), ("f16", "aa"), ("bf16", "pull"),
                          ("f64", "pull")):
        lat, m, noise = make_cavity(olb, torch, dtype, scheme)
        run_workload(lat, noise, 200)
        ms = time_step_kernel(torch, lat, 400)
        b = 19 * 2 * olb.STATE_ELEM[olb.DTYPES[dtype]]
        key = f"cavity128_{dtype}_{scheme}"
        out[key] = {
            "MLUPS": round(fluid / ms / 1e3, 1), "bytes_per_update": b,
            "roofline_frac": round(fluid * b / (ms * 1e-3) / 1e9 / peak, 4)}
        traffic = profiled_traffic(key, fluid)
        if traffic is not None:
            out[key]["traffic"] = round(traffic)  # DRAM bytes per launch (ncu), mean over the pattern's launches
        lat.close()
    # the same cavity with the TRT collision (magic parameter 3/16)
    for dtype in ("f32", "f16"):
        lat, m, noise = make_cavity(olb, torch, dtype, "pull")
        lat.set_trt(I.cavity_tau(N_SIDE, 400.0, LID), 3.0 / 16.0)
        run_workload(lat, noise, 200)
        ms = time_step_kernel(torch, lat, 400)
        b = 19 * 2 * olb.STATE_ELEM[olb.DTYPES[dtype]]
        key = f"cavity128_{dtype}_pull_trt"
        out[key] = {
            "MLUPS": round(fluid / ms / 1e3, 1), "bytes_per_update": b,
            "roofline_frac": round(fluid * b / (ms * 1e-3) / 1e9 / peak, 4)}
        traffic = profiled_traffic(key, fluid)
        if traffic is not None:
            out[key]["traffic"] = round(traffic)
        lat.close()
    # advection-diffusion, D3Q7 256^3 FP32, uniform velocity (7 x 4 x 2 = 56 B per update)
    try:
        n = 256
        a = olb.AdeLattice(olb.D3Q7, (n, n, n), "f32")
        a.set_tau(0.8)
        a.set_velocity((0.02, -0.01, 0.015))
        a.init(torch.ones(n ** 3, dtype=torch.float64, device="cuda"))
        a.step(10)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(a.stream)
        a.step(100)
        ev[1].record(a.stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / 100
        out["ade_d3q7_256_f32"] = {
            "MLUPS": round(n ** 3 / ms / 1e3, 1), "bytes_per_update": 56,
            "roofline_frac": round(n ** 3 * 56 / (ms * 1e-3) / 1e9 / peak, 4)}
        a.close()
    except Exception as e:  # an extra row: report, do not lose the bench line
        out["ade_d3q7_256_f32"] = {"error": str(e)[:200]}
    # 3D Taylor-Green vortex 512^3, periodic (no wall cells)
    n = 512
    for dtype in ("f32", "f16"):
        lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype=dtype, scheme="pull")
        lat.set_material(torch.ones(n ** 3, dtype=torch.uint8, device="cuda"), 7)
        lat.set_bgk(0.6)
        rho, u = I.tgv3d(n, 0.02, xp=torch, device="cuda")
        lat.init_equilibrium(rho.reshape(-1), u.reshape(-1))
        del rho, u
        lat.step(10)
        ms = time_step_kernel(torch, lat, 60)
        b = 19 * 2 * olb.STATE_ELEM[olb.DTYPES[dtype]]
        out[f"tgv512_{dtype}_pull"] = {
            "MLUPS": round(n ** 3 / ms / 1e3, 1), "bytes_per_update": b,
            "roofline_frac": round(n ** 3 * b / (ms * 1e-3) / 1e9 / peak, 4)}
        lat.close()
        torch.cuda.empty_cache()
    # adjoint, porous channel 256x128x128, FP32, 2000 steps, checkpoints every 100
    nx, ny, nz = 256, 128, 128
    lat, m = porous_channel(olb, torch, nx, ny, nz, "f32")
    lat.adjoint_run(20, 10, (0, nx - 1, 0))
    torch.cuda.synchronize()
    steps = 2000
    lat.init_equilibrium()
    t = time.perf_counter()
    loss, dg, dtau = lat.adjoint_run(steps, 100, (0, nx - 1, 0))
    torch.cuda.synchronize()
    sec = time.perf_counter() - t
    fl = int((m == I.FLUID).sum())
    mlups = fl * steps / sec / 1e6
    out["adjoint_channel256_f32"] = {
        "MLUPS": round(mlups, 1), "bytes_per_cell_step": 553,
        "roofline_frac": round(mlups * 1e6 * 553 / 1e9 / peak, 4),
        "loss": loss, "dL_dtau": dtau,
        "note": "forward + recompute + adjoint per cell-step (553 B), 2000 steps, K=100, wall time"}
    lat.close()
    return out


def porous_channel(olb, torch, nx, ny, nz, dtype, tau=0.8):
    """The differentiable channel: periodic x, walls on y and z, smoothed porosity
    (seed 2), Guo force for centre speed 0.05, at rest."""
    m = I.channel(nx, ny, nz)
    lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype=dtype, scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    lat.set_bgk(tau)
    lat.set_force((I.channel_force(ny, tau), 0, 0))
    lat.set_porosity(torch.from_numpy(I.smoothed_porosity(2, m).reshape(-1)).cuda())
    lat.init_equilibrium()
    return lat, m


def experiment_adjoint384(torch, olb, fd_cells=64, h=1e-3, fd_slice=None):
    """Adjoint at scale: channel 384x192x192, FP16 state (FP32 arithmetic, FP64
    gradient), 4000 steps, checkpoints every 200; compared per cell with the
    FP32-storage adjoint (checkpoints every 100) at every fluid cell, and both with
    central differences of FP64 forward runs at `fd_cells` seeded fluid cells
    (h = 1e-3 for gamma, the step experiment_fd256 explains) and tau (h = 1e-6).
    An FP64-storage adjoint does not fit at this size (the segment of 200 states
    alone would take 430 GB).

    One FP64 forward run takes ~24 s on a GB300, so the 2 x 64 runs of the differences
    take ~52 min: `fd_slice` = (a, b) differences only the seeded cells a .. b-1 (and tau
    only when a == 0), and the per-cell values are printed so that the slices of
    several runs can be put together."""
    nx, ny, nz, steps = 384, 192, 192, 4000
    obj = (0, nx - 1, 0)
    res = {"workload": "channel 384x192x192, 4000 steps, loss = mean u_x on x = 383"}
    grads = {}
    for dtype, K in (("f16", 200), ("f32", 100)):
        lat, m = porous_channel(olb, torch, nx, ny, nz, dtype)
        torch.cuda.synchronize()
        t = time.perf_counter()
        loss, dg, dtau = lat.adjoint_run(steps, K, obj)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t
        fl = int((m == I.FLUID).sum())
        grads[dtype] = (loss, dg.cpu().numpy().reshape(-1), dtau)
        res[dtype] = {"K": K, "seconds": round(sec, 2), "MLUPS": round(fl * steps / sec / 1e6, 1),
                      "loss": loss, "dL_dtau": dtau}
        lat.close()
        del dg
        torch.cuda.empty_cache()
    g16, g32 = grads["f16"][1], grads["f32"][1]
    flm = (m == I.FLUID).reshape(-1)
    r = np.abs(g16[flm] - g32[flm]) / np.abs(g32[flm])
    res["f16_vs_f32_all_fluid_cells"] = {
        "rel_l2": float(np.linalg.norm(g16[flm] - g32[flm]) / np.linalg.norm(g32[flm])),
        "rel_median": float(np.median(r)), "rel_p99": float(np.quantile(r, 0.99)),
        "abs_max_over_max_gradient": float(np.abs(g16[flm] - g32[flm]).max() / np.abs(g32[flm]).max())}
    res["f16_vs_f32_dtau_rel"] = abs(grads["f16"][2] - grads["f32"][2]) / abs(grads["f32"][2])
    # FP64 central differences
    gamma = I.smoothed_porosity(2, m)
    ref = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype="f64", scheme="pull")
    ref.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    ref.set_force((I.channel_force(ny, 0.8), 0, 0))
    plane = torch.from_numpy(m[:, :, nx - 1] == I.FLUID).cuda()

    def run(gam, tau):
        ref.set_bgk(tau)
        ref.set_porosity(torch.from_numpy(gam.reshape(-1)).cuda())
        ref.init_equilibrium()
        ref.step(steps)
        _, u = ref.moments()
        return float(u[0, :, :, nx - 1][plane].mean())

    t = time.perf_counter()
    a, b = fd_slice if fd_slice is not None else (0, fd_cells)
    sel = I.random_fluid_cells(3, m, fd_cells)[a:b]
    fd = []
    for c in sel:
        gp = gamma.reshape(-1).copy()
        gm = gp.copy()
        gp[c] += h
        gm[c] -= h
        fd.append((run(gp, 0.8) - run(gm, 0.8)) / (2 * h))
    fd = np.array(fd)
    d_tau = (run(gamma, 0.8 + 1e-6) - run(gamma, 0.8 - 1e-6)) / 2e-6 if a == 0 else None
    ref.close()
    res["fd_cells"] = {"slice": [a, b], "cell": [int(c) for c in sel], "fd": fd.tolist(),
                       "f16": g16[sel].tolist(), "f32": g32[sel].tolist()}
    for key, g in (("f16", g16), ("f32", g32)):
        rel = np.abs(g[sel] - fd) / np.abs(fd)
        res[f"{key}_vs_fd"] = {"cells": int(len(sel)), "h_gamma": h, "rel_max": float(rel.max()),
                               "rel_median": float(np.median(rel)),
                               "cells_within_1e-4": int((rel <= 1e-4).sum()),
                               "cells_within_1e-3": int((rel <= 1e-3).sum()),
                               "dtau_rel": None if d_tau is None else abs(grads[key][2] - d_tau) / abs(d_tau)}
    res["fd_seconds"] = round(time.perf_counter() - t, 1)
    return res


def experiment_fd256(torch, olb, cells=64, h=1e-3, richardson_cells=8):
    """The differentiable channel at its full size: 256x128x128, 2000 steps,
    checkpoints every 100, loss = mean u_x on the outlet plane x = 255.  The FP32- and
    FP64-storage adjoints' dL/dgamma at `cells` seeded random fluid cells and dL/dtau
    against central differences of FP64 forward runs on the GPU, and the FP32 adjoint
    against the FP64 adjoint at every fluid cell.

    Step of the differences: the loss is ~4e-6 and dL/dgamma ~1e-13 .. 1e-11 per cell,
    so at h = 1e-5 the two losses of a quotient differ only in their last ~5
    significant digits and the quotient carries FP64 rounding noise of 1e-5 .. 1e-3
    relative.  h = 1e-3 (gamma stays inside [0, 1]) moves the loss 100 times more; the
    truncation error of the central quotient is checked at `richardson_cells` cells by
    repeating them with h/2 (the two quotients differ by 3/4 of the h^2 error term)."""
    nx, ny, nz, steps, K = 256, 128, 128, 2000, 100
    obj = (0, nx - 1, 0)
    grads = {}
    secs = {}
    for dtype in ("f32", "f64"):
        lat, m = porous_channel(olb, torch, nx, ny, nz, dtype)
        torch.cuda.synchronize()
        t = time.perf_counter()
        loss, dg, dtau = lat.adjoint_run(steps, K, obj)
        torch.cuda.synchronize()
        secs[dtype] = round(time.perf_counter() - t, 2)
        grads[dtype] = (loss, dg.cpu().numpy().reshape(-1), dtau)
        lat.close()
        del dg
        torch.cuda.empty_cache()
    g32, g64 = grads["f32"][1], grads["f64"][1]
    gamma = I.smoothed_porosity(2, m)
    ref = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype="f64", scheme="pull")
    ref.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    ref.set_force((I.channel_force(ny, 0.8), 0, 0))
    plane = torch.from_numpy(m[:, :, nx - 1] == I.FLUID).cuda()

    def run(gam, tau):
        ref.set_bgk(tau)
        ref.set_porosity(torch.from_numpy(gam.reshape(-1)).cuda())
        ref.init_equilibrium()
        ref.step(steps)
        _, u = ref.moments()
        return float(u[0, :, :, nx - 1][plane].mean())

    def quotient(c, hh):
        gp = gamma.reshape(-1).copy()
        gm = gp.copy()
        gp[c] += hh
        gm[c] -= hh
        return (run(gp, 0.8) - run(gm, 0.8)) / (2 * hh)

    t = time.perf_counter()
    sel = I.random_fluid_cells(3, m, cells)
    fd = np.array([quotient(c, h) for c in sel])
    rich = [abs(quotient(c, h / 2) - d) / abs(d) for c, d in zip(sel[:richardson_cells], fd[:richardson_cells])]
    d_tau = (run(gamma, 0.8 + 1e-6) - run(gamma, 0.8 - 1e-6)) / 2e-6
    fd_sec = time.perf_counter() - t
    ref.close()
    r32 = np.abs(g32[sel] - fd) / np.abs(fd)
    r64 = np.abs(g64[sel] - fd) / np.abs(fd)
    fl = (m == I.FLUID).reshape(-1)
    rall = np.abs(g32[fl] - g64[fl]) / np.abs(g64[fl])
    return {
        "workload": f"porous channel {nx}x{ny}x{nz}, {steps} steps, K={K}, loss = mean u_x on x = {nx - 1}",
        "adjoint_seconds": secs, "loss": grads["f32"][0], "dL_dtau": grads["f32"][2],
        "fd": {"cells": int(len(sel)), "h_gamma": h, "h_tau": 1e-6, "seconds": round(fd_sec, 1),
               "truncation_check_h_vs_h/2_rel_max": float(max(rich)),
               "dgamma_abs_range": [float(np.abs(fd).min()), float(np.abs(fd).max())]},
        "f32_vs_fd": {"rel_max": float(r32.max()), "rel_median": float(np.median(r32)),
                      "cells_within_1e-4": int((r32 <= 1e-4).sum()),
                      "dtau_rel": abs(grads["f32"][2] - d_tau) / abs(d_tau)},
        "f64_vs_fd": {"rel_max": float(r64.max()), "rel_median": float(np.median(r64)),
                      "cells_within_1e-6": int((r64 <= 1e-6).sum()),
                      "dtau_rel": abs(grads["f64"][2] - d_tau) / abs(d_tau)},
        "f32_vs_f64_all_fluid_cells": {"rel_median": float(np.median(rall)),
                                       "rel_p99": float(np.quantile(rall, 0.99)),
                                       "rel_p9999": float(np.quantile(rall, 0.9999)),
                                       "abs_max_over_max_gradient": float(np.abs(g32[fl] - g64[fl]).max()
                                                                          / np.abs(g64[fl]).max())},
    }


def experiment_domain_id(torch, olb, dtype="f32", iterations=20):
    """Domain identification at scale (the guide's domainIdentification3d): a cube
    of porosity 0.05 (16^3 cells) in the forced channel 192x96x96 (periodic x, walls
    on y and z, tau 0.8), 1500 steps from rest.  The reference velocity u* comes
    from a forward run with the cube; the porosity of a 32^3 design box around it is
    then identified from u* on the fluid cells outside the box (velocity misfit,
    sigmoid projection, start 0.7, torch L-BFGS with strong Wolfe line search).
    Every evaluation is one checkpointed adjoint run (K = 100)."""
    from paper_2307_11752_gb300 import opti

    nx, ny, nz, steps, K, tau = 192, 96, 96, 1500, 100, 0.8
    m = I.channel(nx, ny, nz)
    lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype=dtype, scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    lat.set_bgk(tau)
    lat.set_force((I.channel_force(ny, tau), 0, 0))
    lat.init_equilibrium()
    f0 = lat.get_populations().clone()
    truth = torch.ones((nz, ny, nx), dtype=torch.float64, device="cuda")
    cz, cy, cx = nz // 2, ny // 2, nx // 3
    truth[cz - 8:cz + 8, cy - 8:cy + 8, cx - 8:cx + 8] = 0.05
    lat.set_porosity(truth.reshape(-1).contiguous())
    lat.step(steps)
    _, u_ref = lat.moments()
    fl = torch.from_numpy(m == I.FLUID).cuda()
    design = torch.zeros_like(fl)
    design[cz - 16:cz + 16, cy - 16:cy + 16, cx - 16:cx + 16] = True
    design &= fl
    region = (fl & ~design).to(torch.uint8)
    tau_t = torch.tensor(tau, dtype=torch.float64)
    times = []

    def evaluate(gamma):
        torch.cuda.synchronize()
        t = time.perf_counter()
        J = olb.velocity_misfit_loss(lat, gamma, tau_t, f0, steps, K, u_ref, region)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
        return J

    t0 = time.perf_counter()
    res = opti.identify_porosity(evaluate, torch.ones_like(truth), design, 0.7, iterations=iterations)
    wall = time.perf_counter() - t0
    inside = truth < 0.5
    core = torch.zeros_like(inside)
    core[cz - 7:cz + 7, cy - 7:cy + 7, cx - 7:cx + 7] = True
    shell = inside & ~core
    g = res.gamma
    fluid = int(fl.sum())
    ev = float(np.median(times))
    out = {
        "workload": f"domain identification, channel {nx}x{ny}x{nz} ({dtype} storage), {steps} steps, K={K}, "
                    f"cube 16^3 of porosity 0.05, design box 32^3 ({int(design.sum())} cells), "
                    f"objective on {int(region.sum())} fluid cells outside the box",
        "iterations": len(res.objective) - 1, "evaluations": res.evaluations, "seconds": round(wall, 2),
        "seconds_per_evaluation": round(ev, 3),
        "MLUPS_per_evaluation": round(fluid * steps / ev / 1e6, 1),
        "objective_first": res.objective[0], "objective_last": res.objective[-1],
        "objective_ratio": res.objective[-1] / res.objective[0],
        "objective": res.objective,
        "gamma_mean_in_cube": float(g[inside].mean()),
        "gamma_mean_cube_shell": float(g[shell].mean()),
        "gamma_mean_cube_core": float(g[core].mean()),
        "gamma_mean_design_outside_cube": float(g[design & ~inside].mean()),
        "gamma_min_design_outside_cube": float(g[design & ~inside].min()),
        "design_cells_below_half": int((g[design] < 0.5).sum()),
        "cube_shell_cells_below_half": int((g[shell] < 0.5).sum()), "cube_shell_cells": int(shell.sum()),
    }
    lat.close()
    return out


PROFILE_CASES = ("cavity128_{f32,f16,bf16}_{pull,aa}[_trt], tgv256_{f32,f16}_pull, "
                 "adjoint_channel128_f32")


def run_profile_case(torch, olb, case: str, launches: int):
    """A short run of one kernel configuration for an ncu capture: set-up, then
    `launches` step launches (or one adjoint run of `launches` steps).  Prints one
    line; times nothing."""
    parts = case.split("_")
    if parts[0] == "cavity128":
        dtype, scheme = parts[1], parts[2]
        lat, m, noise = make_cavity(olb, torch, dtype, scheme)
        if parts[-1] == "trt":
            lat.set_trt(TAU, 3.0 / 16.0)
        lat.init_equilibrium()
        lat.perturb(noise)
        lat.step(launches)
    elif parts[0] == "tgv256":
        n = 256
        lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype=parts[1], scheme=parts[2])
        lat.set_material(torch.ones(n ** 3, dtype=torch.uint8, device="cuda"), 7)
        lat.set_bgk(0.6)
        rho, u = I.tgv3d(n, 0.02, xp=torch, device="cuda")
        lat.init_equilibrium(rho.reshape(-1), u.reshape(-1))
        del rho, u
        lat.step(launches)
    elif case == "adjoint_channel128_f32":
        lat, m = porous_channel(olb, torch, 128, 64, 64, "f32")
        lat.adjoint_run(launches, 10, (0, 127, 0))
    else:
        raise SystemExit(f"unknown profile case {case!r}; cases: {PROFILE_CASES}")
    torch.cuda.synchronize()
    t, k = lat.counters()
    lat.close()
    print(json.dumps({"profile_case": case, "lbm_steps": t, "kernel_launches": k}), flush=True)


def reduce_over_ranks(torch, world: int, maxes, sums, device):
    """Whole-job figures of a multi-rank run: the max over ranks of each value in
    `maxes` (times) and the sum over ranks of each value in `sums` (counts), through
    the default process group on `device`.  On one rank both lists come back as given."""
    if world <= 1:
        return [float(v) for v in maxes], [float(v) for v in sums]
    import torch.distributed as dist

    a = torch.tensor([float(v) for v in maxes], dtype=torch.float64, device=device)
    s = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return a.tolist(), s.tolist()


def run_ours(args):
    import torch

    from paper_2307_11752_gb300 import build, olb

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    build.build()
    olb.load()
    scheme = "pull"
    lat, m, noise = make_cavity(olb, torch, "f32", scheme)
    fluid = int((m == I.FLUID).sum())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms, launches, stats = time_device(torch, lat, noise, args.steps, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    kernel_ms = time_step_kernel(torch, lat, 500)
    lat.close()
    e2e_sec, h2d, d2h = e2e_run(olb, torch, m, max(1, min(args.steps, 3)))
    # whole job: slowest rank's times, every rank's units and launches
    (ms_max, e2e_max), (launches_all,) = reduce_over_ranks(torch, world, [ms, e2e_sec], [launches], "cuda")
    units = fluid * LBM_STEPS * args.steps * world
    value = units / (ms_max * 1e-3) / 1e6
    peak, peak_kind = measured_peak_gbs()
    bytes_per_launch = fluid * 152
    achieved = bytes_per_launch / (kernel_ms * 1e-3) / 1e9
    traffic = profiled_traffic("cavity128_f32_pull", fluid)
    e2e_units = fluid * LBM_STEPS * max(1, min(args.steps, 3)) * world
    extra = variants(olb, torch) if (args.variants and rank == 0) else None
    if world > 1:
        dist.barrier()
    if rank != 0:
        return
    cfg = workload_config()
    cfg["scheme"] = scheme
    cfg["parallelism"] = f"replicas{world}" if world > 1 else "single-gpu"
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": cfg,
        "roofline": {"bound": "hbm", "kernel": "k_step_pair<D3Q19,float,G_PULL,S_OWN>", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "traffic": None if traffic is None else round(traffic),
                     # DRAM bytes (ncu) over the same launch time: the HBM-only fraction
                     "traffic_frac": None if traffic is None else round(traffic / (kernel_ms * 1e-3) / 1e9 / peak, 4),
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": round(kernel_ms, 5)},
        "e2e": {"value": round(e2e_units / e2e_max / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": h2d * world, "d2h_bytes_per_step": d2h * world},
        "gpu_launches": int(launches_all),
        "build": olb.build_info(),
        "clocks": clocks,
        "statistics_last_step": {"mass": stats[0], "max_u": stats[5], "nonfinite": stats[6]},
    }
    if extra is not None:
        line["variants"] = extra
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------
def _oracle_cavity():
    from oracle import oracle as orc

    orc.build()
    m = I.cavity(N_SIDE)
    wu = np.zeros((256, 3))
    wu[I.LID] = (LID, 0.0, 0.0)
    lat = orc.Lattice(orc.D3Q19, m, TAU, periodic=0, wall_u=wu)
    f = lat.init_equilibrium(*I.rest(m.shape)) + I.population_noise(SEED, 19, m, 1e-6)
    return lat, np.ascontiguousarray(f), int((m == I.FLUID).sum())


def _threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else len(os.sched_getaffinity(0))


def cpu_baseline(seconds: float = 12.0, single_thread_seconds: float = 4.0):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: as many LBM steps of the 128^3 cavity as fit in ~`seconds`; with
    `single_thread_seconds` > 0 also on one thread (a child process with
    OMP_NUM_THREADS=1, since the thread count is fixed when the oracle loads)."""
    lat, f, fluid = _oracle_cavity()
    t = time.perf_counter()
    lat.step(f, 1)
    one = time.perf_counter() - t
    n = max(1, min(LBM_STEPS, int(seconds / max(one, 1e-6))))
    t = time.perf_counter()
    lat.step(f, n)
    sec = time.perf_counter() - t
    out = {"value": round(fluid * n / sec / 1e6, 3), "unit": "MLUPS", "cores": _threads(),
           "kind": "oracle",
           "sample": f"{n} of the {LBM_STEPS} FP64 steps of the {N_SIDE}^3 cavity (after 1 warm-up step)"}
    if single_thread_seconds > 0:
        code = ("import json, bench; print(json.dumps(bench.cpu_baseline(%r, 0)))" % float(single_thread_seconds))
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                           env=dict(os.environ, OMP_NUM_THREADS="1"), timeout=600)
        if r.returncode == 0:
            one_thread = json.loads(r.stdout.strip().splitlines()[-1])
            out["single_thread"] = {k: one_thread[k] for k in ("value", "unit", "cores", "sample")}
        else:
            out["single_thread"] = {"error": r.stderr.strip().splitlines()[-1][:200] if r.stderr else "failed"}
    return out


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    lat, f, fluid = _oracle_cavity()
    sample = 2
    for _ in range(args.warmup):
        lat.step(f, 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        lat.step(f, sample)
    sec = time.perf_counter() - t
    value = fluid * sample * args.steps / sec / 1e6
    cfg = workload_config()
    cfg["storage"] = "f64"
    cfg["parallelism"] = "cpu"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3 / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": _threads(),
                             "kind": "oracle",
                             "sample": f"each step = {sample} of the {LBM_STEPS} LBM steps of the "
                                       f"{N_SIDE}^3 cavity in the FP64 CPU oracle"},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--experiment", choices=["adjoint384", "domain_id", "fd256"], default=None,
                    help="run a named experiment instead of the benchmark and print its JSON")
    ap.add_argument("--profile", default=None, metavar="CASE",
                    help="run one kernel configuration briefly for an ncu capture: " + PROFILE_CASES)
    ap.add_argument("--launches", type=int, default=6, help="step launches of --profile")
    ap.add_argument("--fd-slice", default=None, metavar="A:B",
                    help="adjoint384: difference only the seeded cells A .. B-1 of 64")
    args = ap.parse_args()
    if args.profile is not None:
        import torch

        from paper_2307_11752_gb300 import build, olb
        build.build()
        olb.load()
        run_profile_case(torch, olb, args.profile, args.launches)
        return
    if args.experiment is not None:
        import torch

        from paper_2307_11752_gb300 import build, olb
        build.build()
        olb.load()
        run = {"adjoint384": experiment_adjoint384, "domain_id": experiment_domain_id,
               "fd256": experiment_fd256}[args.experiment]
        kw = {}
        if args.fd_slice is not None:
            if args.experiment != "adjoint384":
                raise SystemExit("--fd-slice applies to --experiment adjoint384 only")
            a, b = (int(v) for v in args.fd_slice.split(":"))
            if not 0 <= a < b <= 64:
                raise SystemExit(f"--fd-slice {args.fd_slice}: want 0 <= A < B <= 64")
            kw["fd_slice"] = (a, b)
        print(json.dumps(run(torch, olb, **kw)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
