"""Benchmark of the GRMHD method-of-lines hot path on GB300.

One step = one full SSP-RK3 step of the 256^3 + 3-ghost block on the
Schwarzschild background (isotropic coordinates, M = 1, block [4, 12]^3)
with a planar jump along x ((rho, P) = (1, 1) | (0.125, 0.1), B^x = 0.5,
B^y flipping sign, 1% seeded perturbation), WENO5, HLLE, copy boundaries,
CFL 0.25: three stages of RHS with the stage update (FP64: face states, face
fluxes, then the per-cell pass; mixed: one fused kernel), con2prim and ghost
fill.  Metric: zone-cycles/s = steps * interior cells / time (the paper's
definition, Sec. 5).  The FP64 step is the headline `value`; the mixed step,
the adjoint/forward cost ratio, the 128^3 smooth Schwarzschild block and the
other sections are secondary keys.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grmhd|reference]

Under torchrun each rank runs an independent replica of the block (the
method shards by blocks with no collective on this path); the reported value
is the sum over ranks of the work divided by the slowest rank's time.
`--impl reference` times the CPU oracle (the only other implementation of
the method) on a bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2210_17509_gb300 import inputs as I  # noqa: E402

METRIC = "GRMHD zone-cycles/s (RHS+con2prim) FP64 vs mixed; adjoint/forward cost ratio"
UNIT = "zone-cycles/s"
N_HEADLINE = 256      # Riemann jump on the Schwarzschild background
N_SMOOTH = 128        # smooth state on the Schwarzschild background
CFL = 0.25
PAPER_V100_SETUPA = 0.47e8   # zone-cycles/s, 240^3, RK2, one V100 (Sec. 5.1) -- context only
WINDOW_LO = (104, 104, 104)  # a 48^3 window of the 256^3 block straddling the jump


def workload_config(n=N_HEADLINE):
    return {
        "workload": f"riemann-schwarzschild-{n}^3+3ghost-weno5-hlle-ssprk3",
        "block": [n, n, n], "ghosts": 3, "spacetime": "Schwarzschild isotropic M=1, block [4,12]^3",
        "initial_data": "planar jump along x: (rho, P) = (1, 1) | (0.125, 0.1), B^x = 0.5, B^y = +1 | -1, "
                        "1% seeded perturbation of rho and P",
        "recon": "WENO5", "riemann": "HLLE", "integrator": "SSP-RK3", "cfl": CFL, "bc": "copy",
        "gamma": I.GAMMA, "l2": f"inputs larger than L2 (prim+cons+metric ~ {26 * 8 * (n + 6) ** 3 / 1e9:.1f} GB)",
        "geometry_cache": "static metric: geometry caches built once (first step), reused (GRMHD_REUSE_GEOMETRY)",
    }


def headline_state(n=N_HEADLINE, seed=4):
    return I.riemann_schwarzschild(n, seed=seed)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.lines = []
        self.uuid = device_uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


# --------------------------------------------------------------- reference --
def run_reference(args):
    """The CPU oracle on a bounded sample of the workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    nthreads = os.cpu_count() or 1
    O.set_threads(nthreads)
    blk, prim, met = headline_state(args.n)
    # bounded sample: a 24^3 window of the block straddling the jump, its
    # ghosts by the copy condition
    sub = 24
    lo = tuple(v // 2 - sub // 2 for v in blk.n)
    sblk, sprim = I.window(blk, prim, lo, sub)
    smet = I.window(blk, met, lo, sub)[1]
    del prim, met
    g = O.Grid(sblk.n, 3, sblk.dx)
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_COPY)
    sprim = O.fill_ghosts(g, O.BC_COPY, sprim)
    cons = O.prim2con(g, par.gamma, sprim, smet)
    dt = CFL * min(sblk.dx)
    for _ in range(max(args.warmup, 0)):
        cons, sprim, _ = O.rk_step(g, par, O.RK3, dt, cons, sprim, smet)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cons, sprim, _ = O.rk_step(g, par, O.RK3, dt, cons, sprim, smet)
    t = time.perf_counter() - t0
    value = args.steps * sblk.ncells / t
    sample = (f"{args.steps} SSP-RK3 steps of a {sub}^3 window (interior cells {lo} ..) of the {args.n}^3 "
              f"Riemann-on-Schwarzschild workload straddling the jump (same cells, metric, WENO5/HLLE/copy BC), "
              f"oracle with {nthreads} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


FIELDS = ["D", "S_x", "S_y", "S_z", "tau", "B^x", "B^y", "B^z"]


def _errors(c, ref):
    """Per-field max |c - ref| / max |ref| (normwise), the same with vector
    components against their vector's largest length, and the cell-wise
    relative error of D and tau (floored at 1e-6 of the field's maximum)."""
    norm = [float(np.abs(c[q] - ref[q]).max() / np.abs(ref[q]).max()) for q in range(8)]
    vl = [np.sqrt((ref[sl] ** 2).sum(axis=0)).max() for sl in (slice(1, 4), slice(5, 8))]
    scale = [np.abs(ref[0]).max()] + [vl[0]] * 3 + [np.abs(ref[4]).max()] + [vl[1]] * 3
    vec = [float(np.abs(c[q] - ref[q]).max() / scale[q]) for q in range(8)]
    cell = {}
    for q in (0, 4):
        fl = np.maximum(np.abs(ref[q]), 1e-6 * np.abs(ref[q]).max())
        cell[FIELDS[q]] = float((np.abs(c[q] - ref[q]) / fl).max())
    return {"max_rel_err_per_field": norm, "max": max(norm), "vector_scaled_per_field": vec,
            "vector_scaled_max": max(vec), "cellwise_rel_D_tau": cell}


def _accuracy(G, O, blk, prim, met, lo, sub, steps=1):
    """One window of a workload stepped by the oracle and by the GPU's FP64
    and mixed paths; returns the oracle's (grid, params, cons, prim, metric,
    dt) for timing and the error report."""
    import torch
    sblk, sprim = I.window(blk, prim, lo, sub)
    smet = I.window(blk, met, lo, sub)[1]
    g = O.Grid(sblk.n, 3, sblk.dx)
    gp = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_COPY, rho_atm=gp.rho_atm, p_atm=gp.p_atm, weno_eps=gp.weno_eps)
    sprim = O.fill_ghosts(g, O.BC_COPY, sprim)
    cons = O.prim2con(g, par.gamma, sprim, smet)
    dt = CFL * min(sblk.dx)
    c1, p1, nf = cons, sprim, 0
    for _ in range(steps):
        c1, p1, k = O.rk_step(g, par, O.RK3, dt, c1, p1, smet)
        nf += k
    gg = G.Grid(sblk.n, 3, sblk.dx)
    inner = (slice(None),) + tuple(slice(3, -3) for _ in range(3))
    acc = {"sample": f"{steps} SSP-RK3 step(s) of the {sub}^3 window at interior cells {tuple(lo)}",
           "fields": FIELDS, "oracle_failed_cells": nf}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        tc = torch.from_numpy(cons).cuda()
        tp = torch.from_numpy(sprim).cuda()
        tm = torch.from_numpy(smet).cuda()
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
        ws = G.workspace(gg, G.RK3)
        for _ in range(steps):
            G.rk_step(gg, dataclasses.replace(gp, precision=prec), G.RK3, dt, tc, tp, tm, None, ws, nfail)
        acc[name] = _errors(tc.cpu().numpy()[inner], c1[inner])
        acc[name]["failed_cells"] = int(nfail.item())
    return (g, par, c1, p1, smet, dt, sblk), acc


def cpu_baseline_sample(G, n=N_HEADLINE, seconds_target=15.0):
    """Oracle throughput on a bounded sample (about 10-30 s of CPU work): a
    48^3 window of the headline block straddling the jump.  The same window
    gives the accuracy report: the errors of every conserved field of the
    FP64 and the mixed GPU paths against the FP64 oracle after two SSP-RK3
    steps; a 48^3 window of the smooth 128^3 Schwarzschild block (densities
    1e-3 .. 1) gives the same report for that workload."""
    import oracle as O
    O.build()
    nthreads = os.cpu_count() or 1
    O.set_threads(nthreads)
    blk, prim, met = headline_state(n)
    og = O.Grid(blk.n, 3, blk.dx)
    lo = tuple(v // 2 - 24 for v in blk.n)
    (g, par, cons, sprim, smet, dt, sblk), acc = _accuracy(G, O, blk, prim, met, lo, 48, steps=2)
    del prim, met, og
    sblk2, prim2, met2 = I.smooth_schwarzschild(N_SMOOTH, seed=1)
    _, acc128 = _accuracy(G, O, sblk2, prim2, met2, (40, 40, 40), 48, steps=2)
    del prim2, met2
    steps, t = 0, 0.0
    t0 = time.perf_counter()
    while t < seconds_target and steps < 400:
        cons, sprim, _ = O.rk_step(g, par, O.RK3, dt, cons, sprim, smet)
        steps += 1
        t = time.perf_counter() - t0
    return {
        "value": steps * sblk.ncells / t, "unit": UNIT, "cores": nthreads, "kind": "oracle",
        "sample": f"{steps} SSP-RK3 steps of a 48^3 window of the {n}^3 Riemann-on-Schwarzschild workload "
                  f"straddling the jump ({t:.1f} s of CPU work, {nthreads} OpenMP threads)",
        "accuracy_vs_oracle": acc,
        "accuracy_vs_oracle_smooth_128": acc128,
    }


# --------------------------------------------------------------- batched --
def batched_bench(G, steps, warmup, nbox=512):
    """512 AMR-like boxes (edges from {8..64}, 3 refinement levels, flat):
    recovery + ghost fill + RHS of every box as one library-owned CUDA graph
    of persistent launches (three kernels; five for the three-pass FP64 WENO5
    RHS), launched once per evaluation, against the same launches issued
    directly and against the plain form (three launches per box)."""
    import torch
    from paper_2210_17509_gb300 import autotune
    t0 = time.perf_counter()
    data = I.amr_boxes(nbox, seed=2)
    gen_s = time.perf_counter() - t0
    out = {"workload": f"{nbox} boxes, edges from {{8,16,24,32,48,64}}, levels 0-2, flat, WENO5+HLLE, "
                       "recovery+ghost fill+RHS", "input_generation_s": gen_s}
    ncells = sum(b.ncells for b, _ in data)
    out["interior_cells"] = ncells
    for precision, name in ((G.FP64, "fp64"), (G.MIXED, "mixed")):
        p = G.Params(recon=G.WENO5, bc=G.BC_PERIODIC, precision=precision)
        costs = autotune.tile_costs(p)
        boxes = []
        for blk, prim in data:
            g = G.Grid(blk.n, blk.ng, blk.dx)
            tp = torch.from_numpy(prim).cuda()
            G.fill_ghosts(g, G.BC_PERIODIC, tp)
            tc = G.prim2con(g, p, tp)
            boxes.append(G.Box(g, tc, tp, torch.zeros_like(tp), None, autotune.choose(blk.n, costs),
                               G.BC_PERIODIC))
        batch = G.Batch(boxes, p)
        for _ in range(max(warmup, 1)):
            batch.rhs(p)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            batch.rhs(p)
        e1.record()
        torch.cuda.synchronize()
        ms_direct = e0.elapsed_time(e1) / steps
        # the whole evaluation in one persistent launch (one-pass RHS tiles)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(max(warmup, 1)):
            batch.rhs_fused(p, None, status)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            batch.rhs_fused(p, None, status)
        e1.record()
        torch.cuda.synchronize()
        ms_fused = e0.elapsed_time(e1) / steps
        fused_status = int(status.item())
        # the library-owned graph of the phased launches: one launch per evaluation
        graph = batch.graph(p)
        for _ in range(warmup):
            graph.launch()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            graph.launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # plain form: per-box launches of the single-block entry points
        def plain():
            for b in boxes:
                G.con2prim(b.grid, p, b.cons, b.prim)
                G.fill_ghosts(b.grid, G.BC_PERIODIC, b.prim)
                G.rhs(b.grid, p, b.prim, None, None, b.rhs)
        plain()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            plain()
        e1.record()
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1) / steps
        tiles_used = {}
        for b in boxes:
            tiles_used[str(autotune.SHAPES[b.tile])] = tiles_used.get(str(autotune.SHAPES[b.tile]), 0) + 1
        out[name] = {"value": ncells / (ms * 1e-3), "unit": "cells/s (recovery+RHS per box, one evaluation)",
                     "ms_per_batch": ms, "form": "library graph (grmhd_batch_graph_launch), one launch per batch",
                     "direct_ms_per_batch": ms_direct,
                     "one_launch": {"ms_per_batch": ms_fused, "value": ncells / (ms_fused * 1e-3),
                                    "form": "grmhd_batch_rhs_fused: one memset + one persistent kernel "
                                            "(recovery, ghost fill, one-pass RHS tiles)",
                                    "status": fused_status},
                     "plain_per_box_ms": ms_plain,
                     "speedup_vs_plain": ms_plain / ms,
                     "kernels_per_batch": (3 + (batch.c.two_pass + batch.c.three_pass
                                                if precision == G.FP64 else 0)),
                     "multi_pass": ("three passes" if batch.c.three_pass and precision == G.FP64 else
                                    "two passes" if batch.c.two_pass and precision == G.FP64 else "one pass"),
                     "tile_shapes": tiles_used}
        graph.close()
        del boxes, batch, graph
        torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------- adjoint --
def adjoint_bench(G, n=64, nsteps=20, every=5, ndir=50):
    """64^3 periodic flat block, WENO5, 20 SSP-RK3 steps, L = sum rho^2 dV:
    time of the checkpointed adjoint (backward) against the forward pass, and
    the adjoint gradient against central differences along ndir smooth random
    directions (initial primitives and Gamma together)."""
    import dataclasses
    import torch
    from paper_2210_17509_gb300 import adjoint as A
    blk, prim_h, _ = I.smooth_flat(n, seed=3)
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_PERIODIC)
    dt = 0.25 * blk.dx[0]
    prim0 = torch.from_numpy(prim_h[:, 3:-3, 3:-3, 3:-3].copy()).cuda()

    def run(with_grad, det=False):
        x = prim0.clone().requires_grad_(with_grad)
        gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=with_grad)
        L = A.density_l2(A.evolve(x, gam, g, p, G.RK3, dt, nsteps, checkpoint_every=every, deterministic=det), g)
        return x, gam, L

    for _ in range(2):               # warm-up (module load, workspaces, the allocator's pools)
        run(True)[2].backward()
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    reps = []
    for _ in range(3):               # three forward + backward passes; the fastest backward counts
        e0.record()
        x, gam, L = run(True)
        e1.record()
        L.backward()
        e2.record()
        torch.cuda.synchronize()
        reps.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    # the backward is driven from Python (a few thousand launches); a stall of the
    # shared host's CPU leaves the GPU idle and adds tens of ms to single passes
    t_fwd, t_bwd = min(reps, key=lambda r: r[1])
    # the fixed-order reverse (GRMHD_DETERMINISTIC): one warm-up, two timed passes;
    # the two gradients must agree to the bit
    run(True, True)[2].backward()
    dreps, dgrads = [], []
    for _ in range(2):
        e0.record()
        xd, gd, Ld = run(True, True)
        e1.record()
        Ld.backward()
        e2.record()
        torch.cuda.synchronize()
        dreps.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        dgrads.append((xd.grad.clone(), float(gd.grad)))
    dfwd, dbwd = min(dreps, key=lambda r: r[1])
    deterministic = {
        "passes_ms": dreps, "forward_ms": dfwd, "backward_ms": dbwd, "adjoint_forward_ratio": dbwd / dfwd,
        "repeats_bitwise": bool(torch.equal(dgrads[0][0], dgrads[1][0]) and dgrads[0][1] == dgrads[1][1]),
        "max_rel_diff_vs_atomic": float((dgrads[0][0] - x.grad).abs().max() / x.grad.abs().max()),
    }
    # plain forward without checkpoint copies, for context
    e0.record()
    with torch.no_grad():
        run(False)
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1)
    # central differences along smooth random directions
    rng = np.random.default_rng(123)
    h = 1e-6
    errs = []
    for k in range(ndir):
        # smooth direction, not mean-free: a well-conditioned directional derivative
        d = I.smooth_prims(blk, 5000 + k)[:, 3:-3, 3:-3, 3:-3]
        d = d / np.abs(d).max(axis=(1, 2, 3), keepdims=True)
        dt_ = torch.from_numpy(np.ascontiguousarray(d)).cuda() * prim0.abs().amax(dim=(1, 2, 3), keepdim=True)
        dg = float(rng.normal())

        def loss(p0, gm):
            with torch.no_grad():
                pp = dataclasses.replace(p)
                return float(A.density_l2(A.evolve(p0, torch.tensor(gm, dtype=torch.float64), g, pp, G.RK3, dt,
                                                   nsteps), g))
        fd = (loss(prim0 + h * dt_, p.gamma + h * dg) - loss(prim0 - h * dt_, p.gamma - h * dg)) / (2 * h)
        ad = float((x.grad * dt_).sum()) + float(gam.grad) * dg
        errs.append(abs(fd - ad) / abs(ad))
    return {
        "workload": f"{n}^3 periodic flat, WENO5+HLLE, {nsteps} SSP-RK3 steps, checkpoint every {every}, "
                    "L = sum rho^2 dV, gradient w.r.t. initial primitives [8,64,64,64] and Gamma",
        "checkpointing": f"(U, P) every {every} steps; the last segment's stages recorded by the forward pass, "
                         "the earlier segments recomputed by the backward pass",
        "timing": "the pass with the fastest backward of 3 forward + backward passes after 2 warm-up passes",
        "passes_ms": reps,
        "forward_ms": t_fwd, "backward_ms": t_bwd, "forward_plain_ms": t_plain,
        "adjoint_forward_ratio": t_bwd / t_fwd, "adjoint_plain_forward_ratio": t_bwd / t_plain,
        "deterministic": deterministic,
        "fd_check": ({"directions": ndir, "h": h, "max_rel_err": max(errs), "median_rel_err": float(np.median(errs))}
                     if errs else None),
        "loss": float(L.item()),
    }


# ------------------------------------------------------------ shock tube --
def shocktube_bench(G, test=1, n=1600, transverse=8):
    """Balsara shock tube (Sec. 4.1) as the paper runs it: minmod + HLLE +
    RK4, CFL 0.8, copy boundaries, n cells on [-0.5, 0.5] along x and 8 x 8
    transverse cells, evolved to t_ref.  A 1600 x 8 x 8 block is too small to
    fill the GPU, so the 12 launches of a step are timed both as plain
    launches and replayed from one CUDA graph; the peak Lorentz factor at
    t_ref is reported against the paper's printed value."""
    import torch
    blk, prim_h, gamma, t_ref = I.shocktube(test, n, 0, transverse)
    g = G.Grid(blk.n, blk.ng, blk.dx)
    p = G.Params(gamma=gamma, recon=G.MINMOD, bc=G.BC_COPY)
    dt = 0.8 / n
    nsteps = int(round(t_ref / dt))
    ncells = blk.n[0] * blk.n[1] * blk.n[2]

    def setup():
        prim = torch.from_numpy(prim_h).cuda()
        cons = G.prim2con(g, p, prim)
        ws = G.workspace(g, G.RK4)
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
        return prim, cons, ws, nfail

    out = {"workload": f"Balsara {test}, {n}x{transverse}x{transverse}, minmod+HLLE, RK4, CFL 0.8, copy BC, "
                       f"{nsteps} steps to t_ref = {t_ref}"}
    # plain launches
    prim, cons, ws, nfail = setup()
    for _ in range(3):
        G.rk_step(g, p, G.RK4, dt, cons, prim, None, None, ws, nfail)
    prim, cons, ws, nfail = setup()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(nsteps):
        G.rk_step(g, p, G.RK4, dt, cons, prim, None, None, ws, nfail)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    v = prim[1:4, blk.ng:-blk.ng, blk.ng:-blk.ng, blk.ng:-blk.ng]
    wmax = float((1.0 / torch.sqrt(1.0 - (v * v).sum(dim=0))).max())
    out["plain"] = {"value": ncells * nsteps / (ms * 1e-3), "unit": "zone-cycles/s", "ms_total": ms,
                    "failed_cells": int(nfail.item())}
    # one step captured in a CUDA graph, replayed nsteps times from the initial state
    prim, cons, ws, nfail = setup()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        G.rk_step(g, p, G.RK4, dt, cons, prim, None, None, ws, nfail)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        G.rk_step(g, p, G.RK4, dt, cons, prim, None, None, ws, nfail)
    prim0, cons0, _, _ = setup()
    prim.copy_(prim0)
    cons.copy_(cons0)
    nfail.zero_()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(nsteps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    msg = e0.elapsed_time(e1)
    v = prim[1:4, blk.ng:-blk.ng, blk.ng:-blk.ng, blk.ng:-blk.ng]
    wmax_g = float((1.0 / torch.sqrt(1.0 - (v * v).sum(dim=0))).max())
    out["graph"] = {"value": ncells * nsteps / (msg * 1e-3), "unit": "zone-cycles/s", "ms_total": msg,
                    "failed_cells": int(nfail.item()), "launches_per_step": 12}
    out["peak_lorentz_factor"] = {"plain": wmax, "graph": wmax_g, "paper_printed": 1.458}
    return out


# ------------------------------------------------------------- two-level AMR --
def amr_bench(G, steps=5, warmup=2, nc=96, nfine=48):
    """Two-level block AMR without subcycling (Sec. 3): a 96^3 periodic flat
    coarse block with four 48^3 fine blocks (each covering 24^3 coarse cells,
    apart from one another), WENO5+HLLE, SSP-RK3 at CFL 0.25 of the fine
    spacing.  The composite step (fused RHS+update per block, flux
    restriction, restriction, recovery, ghost fill, prolongation) is timed
    against plain steps of the same five blocks, and the three transfer
    kernels are timed on their own."""
    import torch
    ng = 3
    cb = I.Block((nc,) * 3, ng, (1.0 / nc,) * 3, (0.0,) * 3)
    pc_h = I.smooth_prims(cb, 31)
    half = nfine // 2
    los = [(8, 8, 8), (8 + half + 24, 8, 8), (8, 8 + half + 24, 8 + half + 24), (8 + half + 24, 8 + half + 24, 8)]
    C = G.Grid(cb.n, ng, cb.dx)
    Fs = [G.Grid((nfine,) * 3, ng, (0.5 / nc,) * 3) for _ in los]
    p = G.Params(recon=G.WENO5, bc=G.BC_PERIODIC)
    pc = torch.from_numpy(pc_h).cuda()
    G.fill_ghosts(C, G.BC_PERIODIC, pc)
    pfs = []
    for F, lo in zip(Fs, los):
        pf = torch.zeros((8,) + F.shape, dtype=torch.float64, device="cuda")
        G.prolongate(C, pc, F, pf, lo, ghosts_only=False)
        pfs.append(pf)
    uc = G.prim2con(C, p, pc)
    ufs = [G.prim2con(F, p, pf) for F, pf in zip(Fs, pfs)]
    for F, uf, lo in zip(Fs, ufs, los):
        G.restrict(C, uc, F, uf, lo)
    ws = G.amr2_workspace(C, Fs, G.RK3)
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    dt = 0.25 * Fs[0].dx[0]
    ncells = nc ** 3 + len(Fs) * nfine ** 3

    def timed(fn, n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def composite():
        G.amr2_step(C, p, G.RK3, dt, uc, pc, Fs, ufs, pfs, los, ws=ws, nfail=nfail)

    for _ in range(warmup):
        composite()
    ms = timed(composite, steps)
    # the same five blocks stepped independently (no transfer)
    wsc = G.workspace(C, G.RK3, cached=False)
    wsf = [G.workspace(F, G.RK3, cached=False) for F in Fs]

    def plain():
        G.rk_step(C, p, G.RK3, dt, uc, pc, None, None, wsc, nfail)
        for F, uf, pf, w in zip(Fs, ufs, pfs, wsf):
            G.rk_step(F, p, G.RK3, dt, uf, pf, None, None, w, nfail)

    ms_plain = timed(plain, steps)
    out = torch.zeros_like(uc)
    t_restrict = timed(lambda: [G.restrict(C, uc, F, uf, lo) for F, uf, lo in zip(Fs, ufs, los)], 20)
    t_prolong = timed(lambda: [G.prolongate(C, pc, F, pf, lo) for F, pf, lo in zip(Fs, pfs, los)], 20)
    t_reflux = timed(lambda: [G.reflux(C, p, pc, F, pf, lo, out) for F, pf, lo in zip(Fs, pfs, los)], 20)
    # algorithmic bytes of one restriction pass: 8 fields x (8 fine reads + 1 coarse write) per covered cell
    cov = len(Fs) * half ** 3
    restrict_bytes = 8 * cov * 9 * 8
    hbm, _ = __import__("paper_2210_17509_gb300.roofline", fromlist=["hbm_peak_gbs"]).hbm_peak_gbs()
    return {
        "workload": f"{nc}^3 periodic flat coarse block + {len(Fs)} fine blocks of {nfine}^3 (each over {half}^3 "
                    f"coarse cells), WENO5+HLLE, SSP-RK3, dt = 0.25 dx_fine",
        "cells": ncells,
        "composite": {"value": ncells / (ms * 1e-3), "unit": "zone-cycles/s", "ms_per_step": ms,
                      "failed_cells": int(nfail.item())},
        "plain_blocks_ms_per_step": ms_plain,
        "transfer_overhead": ms / ms_plain - 1.0,
        "transfer_ms_per_pass": {"restrict": t_restrict, "prolongate_ghosts": t_prolong, "reflux": t_reflux},
        "restrict_gbs": restrict_bytes / (t_restrict * 1e-3) / 1e9,
        "restrict_hbm_frac": restrict_bytes / (t_restrict * 1e-3) / 1e9 / hbm,
    }


# ------------------------------------------------- constrained transport --
def ct_bench(G, steps=5, warmup=2, n=N_SMOOTH):
    """Constrained transport (Sec. 3: the field on staggered grids): the
    smooth 128^3 Schwarzschild block with a divergence-free face field (the
    discrete curl of a random edge potential, |sqrt(gamma) B| <= 0.03, so
    b^2/rho <= 0.2 on the density floor of 1e-3; cell field = mean of the
    faces), WENO5+HLLE, SSP-RK3 at CFL 0.25, FP64 and mixed.  Timed
    against plain steps of the same state; the largest |div B| after the
    timed steps is reported relative to max |B| / dx.  (At |B| <= 0.1 the
    cells with plasma beta ~ 2e-3 fall to the atmosphere under CT, in the
    oracle exactly as here: the face-averaged field differs from the
    cell-centred one by more than the thermal energy there.)"""
    import torch
    blk, prim_h, met_h = I.smooth_schwarzschild(n, seed=1)
    bf_h = I.face_curl(blk, I.edge_potential(blk, 101))
    inner = (slice(None),) + tuple(slice(blk.ng, s - blk.ng) for s in blk.shape)
    bf_h *= 0.03 / np.abs(bf_h[inner]).max()
    g = G.Grid(blk.n, blk.ng, blk.dx)
    met = torch.from_numpy(met_h).cuda()
    dt = CFL * min(blk.dx)
    out = {"workload": f"{n}^3 smooth Schwarzschild block with a divergence-free face field "
                       f"(|sqrt(gamma) B| <= 0.03), "
                       f"WENO5+HLLE, SSP-RK3, dt = {CFL} dx, copy boundaries"}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        res = {}
        for mode in ("plain", "ct"):
            p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec)
            prim = torch.from_numpy(prim_h).cuda()
            b = torch.from_numpy(bf_h).cuda()
            G.ct_cell_field(g, b, prim, met)        # cell field = face mean / sqrt(gamma)
            G.fill_ghosts(g, G.BC_COPY, prim)
            cons = G.prim2con(g, p, prim, met)
            ws = G.ct_workspace(g, G.RK3) if mode == "ct" else G.workspace(g, G.RK3)
            nfail = torch.zeros(1, dtype=torch.int32, device="cuda")

            def step(p):
                if mode == "ct":
                    G.ct_rk_step(g, p, G.RK3, dt, cons, prim, b, met, ws=ws, nfail=nfail)
                else:
                    G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)

            for _ in range(warmup):
                step(p)
                p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                step(p)
            e1.record()
            torch.cuda.synchronize()
            res[mode] = e0.elapsed_time(e1) / steps
            res[mode + "_failed"] = int(nfail.item())
            if mode == "ct":
                _, mx = G.ct_divergence(g, b, maxabs=torch.zeros(1, dtype=torch.float64, device="cuda"))
                div_rel = mx.item() * min(blk.dx) / b.abs().max().item()
        out[name] = {"value": blk.ncells / (res["ct"] * 1e-3), "unit": UNIT, "ms_per_step": res["ct"],
                     "plain_ms_per_step": res["plain"], "ct_overhead": res["ct"] / res["plain"] - 1.0,
                     "max_div_b_rel": div_rel, "steps": warmup + steps, "failed_cells": res["ct_failed"],
                     "plain_failed_cells": res["plain_failed"]}
    return out


# ------------------------------------------------------ polytropic EOS --
def poly_bench(G, steps=5, warmup=2, n=N_SMOOTH, K=100.0, gamma=2.0):
    """Polytropic EOS (Sec. 2.3; K = 100, Gamma = 2 as the paper's TOV star,
    Sec. 4.4): the 128^3 Schwarzschild block with a smooth state of
    density 1e-4 .. 1.28e-3 (the TOV central density), P = K rho^Gamma,
    |v| <= 0.5 and a weak field (|B| <= 1e-3), WENO5+HLLE, SSP-RK3 at the
    CFL 0.25, copy boundaries; FP64 and mixed."""
    import torch
    blk = I.Block((n,) * 3, 3, (8.0 / n,) * 3, (4.0,) * 3)
    met_h = I.schwarzschild_metric(blk)
    prim_h = I.smooth_prims(blk, 1, gamma, rho_range=(1e-4, 1.28e-3), metric=met_h, b_amp=1e-3)
    prim_h[4] = K * prim_h[0] ** gamma
    g = G.Grid(blk.n, blk.ng, blk.dx)
    met = torch.from_numpy(met_h).cuda()
    dt = CFL * min(blk.dx)
    out = {"workload": f"{n}^3 Schwarzschild block, polytrope K = {K}, Gamma = {gamma}, rho 1e-4..1.28e-3, "
                       f"|v| <= 0.5, |B| <= 1e-3, WENO5+HLLE, SSP-RK3, dt = {CFL} dx, copy boundaries"}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        p = G.Params(gamma=gamma, recon=G.WENO5, bc=G.BC_COPY, precision=prec, eos=G.EOS_POLYTROPE, poly_K=K)
        prim = torch.from_numpy(prim_h).cuda()
        G.fill_ghosts(g, G.BC_COPY, prim)
        cons = G.prim2con(g, p, prim, met)
        ws = G.workspace(g, G.RK3)
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
            p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": blk.ncells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "steps": warmup + steps, "failed_cells": int(nfail.item())}
    return out


# ------------------------------------------------------------------- GPU --
def _timer():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def block_state(G, blk, prim_h, met, precision, tile=0):
    import torch
    g = G.Grid(blk.n, blk.ng, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision, tile=tile)
    prim = torch.from_numpy(prim_h).cuda()
    G.fill_ghosts(g, G.BC_COPY, prim)
    cons = G.prim2con(g, p, prim, met)
    ws = G.workspace(g, G.RK3)
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    return g, p, prim, cons, ws, nfail


def time_steps(G, REP, blk, prim_h, met, precision, steps, warmup, tile=0, clocks=None):
    """warmup + steps SSP-RK3 steps of one block; the timed ones bracketed by a
    barrier and a synchronize on both sides, on the stream they run on.
    Returns (ms over the timed steps, max over ranks; failed cells; state)."""
    import torch
    g, p, prim, cons, ws, nfail = block_state(G, blk, prim_h, met, precision, tile)
    dt = CFL * min(blk.dx)
    for _ in range(warmup):
        G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
        # static metric: the geometry cache built by the first step is kept
        p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
    torch.cuda.synchronize()
    REP.barrier()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = _timer()
    e0.record(stream)
    for _ in range(steps):
        G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
    e1.record(stream)
    torch.cuda.synchronize()
    REP.barrier()
    clk = clocks.stop() if clocks is not None else None
    ms = REP.max_over_ranks(e0.elapsed_time(e1))
    return ms, int(nfail.item()), clk, (g, p, prim, cons, ws, nfail, dt)


def adjoint_step_ratio(G, g, p, prim, cons, met, ws, dt, ms_step):
    """Reverse of one SSP-RK3 step from recorded stages (the checkpointed
    backward's unit of work) against the forward FP64 step."""
    import torch
    stages = torch.empty((3, 8) + g.shape, dtype=torch.float64, device="cuda")
    c0, p0 = cons.clone(), prim.clone()
    G.rk_step_record(g, p, G.RK3, dt, cons, prim, stages, met, None, ws)
    wsa = G.adjoint_workspace(g, G.RK3)
    ub = torch.zeros_like(cons)
    pb = torch.zeros_like(prim)
    pb[0] = 1.0
    gb = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.rk_step_adjoint(g, p, G.RK3, dt, c0, p0, ub, pb, gb, met, None, wsa, stage_prims=stages)
    torch.cuda.synchronize()
    e0, e1 = _timer()
    e0.record()
    G.rk_step_adjoint(g, p, G.RK3, dt, c0, p0, ub, pb, gb, met, None, wsa, stage_prims=stages)
    e1.record()
    torch.cuda.synchronize()
    ams = e0.elapsed_time(e1)
    return {"ms": ams, "ratio_to_fp64_step": ams / ms_step,
            "value": blk_cells(g) / (ams * 1e-3),
            "unit": "zone-cycles/s (reverse step, recorded stages)"}


def blk_cells(g):
    return g.n[0] * g.n[1] * g.n[2]


def e2e_bench(G, REP, blk, prim_h, met, steps_e):
    """End to end through the public API with host buffers: every step uploads
    its inputs (U, primitives, metric) from pinned host memory, runs
    grmhd_rk_step and downloads its result (U, primitives).  Three device
    buffer sets let step k + 1's upload and step k - 1's download run on copy
    streams while step k computes (a user streaming steps would do the same);
    the serial figure (copies, then compute, then copies) is kept too."""
    import torch
    g, p, prim_d, cons_d, ws_e, nfail_e = block_state(G, blk, prim_h, met, G.FP64)
    dt = CFL * min(blk.dx)
    cons_h = cons_d.cpu().pin_memory()
    prim_h2 = prim_d.cpu().pin_memory()
    met_hp = met.cpu().pin_memory()
    del prim_d, cons_d
    # three buffer sets: step k + 3's upload waits for step k's download, so a
    # download and the next upload of the same set have two compute steps to run in
    nsets = 3
    bufs = []
    for _ in range(nsets):
        bufs.append({"cons": torch.empty_like(cons_h, device="cuda"), "prim": torch.empty_like(prim_h2, device="cuda"),
                     "met": torch.empty_like(met), "out_c": torch.empty_like(cons_h).pin_memory(),
                     "out_p": torch.empty_like(prim_h2).pin_memory()})
    s_comp = torch.cuda.current_stream()
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(nsets)] for k in ("up", "done", "down")}

    # the metric is static: the warm-up step builds the geometry caches and the
    # timed steps reuse them (GRMHD_REUSE_GEOMETRY), as the device-timed value
    # does; every step still uploads all of its inputs, the metric included
    p_reuse = dataclasses.replace(p, flags=p.flags | G.REUSE_GEOMETRY)

    def serial_step(b, pp=p_reuse):
        b["cons"].copy_(cons_h, non_blocking=True)
        b["prim"].copy_(prim_h2, non_blocking=True)
        b["met"].copy_(met_hp, non_blocking=True)
        G.rk_step(g, pp, G.RK3, dt, b["cons"], b["prim"], b["met"], None, ws_e, nfail_e)
        b["out_c"].copy_(b["cons"], non_blocking=True)
        b["out_p"].copy_(b["prim"], non_blocking=True)

    def pipelined(n):
        # uploads and downloads on streams of their own, so that step k + 1's
        # upload is not queued behind step k's download
        for k in range(n):
            i = k % nsets
            b = bufs[i]
            with torch.cuda.stream(s_up):
                if k >= nsets:
                    s_up.wait_event(ev["down"][i])
                b["cons"].copy_(cons_h, non_blocking=True)
                b["prim"].copy_(prim_h2, non_blocking=True)
                b["met"].copy_(met_hp, non_blocking=True)
                ev["up"][i].record(s_up)
            s_comp.wait_event(ev["up"][i])
            G.rk_step(g, p_reuse, G.RK3, dt, b["cons"], b["prim"], b["met"], None, ws_e, nfail_e, stream=s_comp)
            ev["done"][i].record(s_comp)
            with torch.cuda.stream(s_down):
                s_down.wait_event(ev["done"][i])
                b["out_c"].copy_(b["cons"], non_blocking=True)
                b["out_p"].copy_(b["prim"], non_blocking=True)
                ev["down"][i].record(s_down)
        s_comp.wait_stream(s_up)
        s_comp.wait_stream(s_down)

    def timed_e2e(fn):
        torch.cuda.synchronize()
        REP.barrier()
        q0, q1 = _timer()
        q0.record(s_comp)
        fn()
        q1.record(s_comp)
        torch.cuda.synchronize()
        REP.barrier()
        return REP.max_over_ranks(q0.elapsed_time(q1))

    serial_step(bufs[0], p)
    pipelined(nsets)
    ems_serial = timed_e2e(lambda: [serial_step(bufs[0]) for _ in range(steps_e)])
    ems = timed_e2e(lambda: pipelined(steps_e))
    h2d = cons_h.numel() * 8 + prim_h2.numel() * 8 + met_hp.numel() * 8
    d2h = bufs[0]["out_c"].numel() * 8 + bufs[0]["out_p"].numel() * 8
    ncells = blk.ncells
    return {"value": REP.job_rate(ncells * steps_e, ems), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "dtype": "f64", "steps": steps_e,
            "copies": "overlapped with the neighbouring steps' compute (three device buffer sets, upload and "
                      "download streams)",
            "geometry_cache": "built by the warm-up step from the uploaded static metric, reused by the timed steps "
                              "(GRMHD_REUSE_GEOMETRY), as for the device-timed value",
            "serial_value": REP.job_rate(ncells * steps_e, ems_serial)}


def mixed_tile(G, n, forced=-1):
    """RHS tile shape of the mixed path: the project's autotuner's choice for
    an n^3 curved block, unless one is forced (profiling runs)."""
    if forced >= 0:
        return forced
    from paper_2210_17509_gb300 import autotune
    return autotune.best_block_shape(G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=G.MIXED), (n, n, n),
                                     curved=True)


def smooth_block_bench(G, REP, steps, warmup, n=N_SMOOTH, tile_mx=-1):
    """The smooth 128^3 Schwarzschild block (densities 1e-3 .. 1, |v| <= 0.5,
    |B| <= 0.1, WENO5+HLLE, SSP-RK3, CFL 0.25, copy BC), FP64 and mixed."""
    import torch
    from paper_2210_17509_gb300 import autotune
    blk, prim_h, met_h = I.smooth_schwarzschild(n, seed=1)
    met = torch.from_numpy(met_h).cuda()
    tile = mixed_tile(G, n, tile_mx)
    out = {"workload": f"schwarzschild-block-{n}^3+3ghost-weno5-hlle-ssprk3 (smooth, rho 1e-3..1)"}
    for precision, name, t in ((G.FP64, "fp64", 0), (G.MIXED, "mixed", tile)):
        ms, nf, _, st = time_steps(G, REP, blk, prim_h, met, precision, steps, warmup, tile=t)
        out[name] = {"value": REP.job_rate(blk.ncells * steps, ms), "unit": UNIT, "ms_per_step": ms / steps,
                     "failed_cells": nf}
        del st
        torch.cuda.empty_cache()
    out["mixed"]["tile"] = autotune.BLOCK_SHAPES[tile]
    out["mixed_speedup"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grmhd", choices=["grmhd", "reference"])
    ap.add_argument("--n", type=int, default=N_HEADLINE)
    ap.add_argument("--smooth-n", type=int, default=N_SMOOTH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-smooth", action="store_true")
    ap.add_argument("--no-shocktube", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-ct", action="store_true")
    ap.add_argument("--no-poly", action="store_true")
    ap.add_argument("--section", default=None,
                    choices=["ct", "poly", "amr", "shocktube", "batched", "adjoint", "smooth"],
                    help="run only this section and print its JSON (profiling runs)")
    ap.add_argument("--mixed-tile", type=int, default=-1,
                    help="RHS tile shape of the mixed path (default: the autotuner's choice)")
    ap.add_argument("--adjoint-n", type=int, default=64)
    ap.add_argument("--adjoint-dirs", type=int, default=50)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2210_17509_gb300.replicas import Replicas
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    REP = Replicas("nccl", torch.device("cuda", local))
    world, rank = REP.world, REP.rank

    from paper_2210_17509_gb300 import grmhd as G
    from paper_2210_17509_gb300 import roofline as R

    if args.section:
        fns = {"ct": lambda: ct_bench(G, n=args.smooth_n), "poly": lambda: poly_bench(G, n=args.smooth_n),
               "amr": lambda: amr_bench(G), "shocktube": lambda: shocktube_bench(G),
               "batched": lambda: batched_bench(G, args.steps, args.warmup),
               "adjoint": lambda: adjoint_bench(G, n=args.adjoint_n, ndir=args.adjoint_dirs),
               "smooth": lambda: smooth_block_bench(G, REP, args.steps, args.warmup, args.smooth_n, args.mixed_tile)}
        out = fns[args.section]()
        if rank == 0:
            print(json.dumps({"section": args.section, args.section: out}), flush=True)
        return

    blk, prim_h, met_h = headline_state(args.n, seed=4 + rank)
    met = torch.from_numpy(met_h).cuda()
    del met_h
    ncells = blk.ncells
    hbm, hbm_src = R.hbm_peak_gbs()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    # FP64 (headline) -- clocks sampled during this timed region
    ms64, nfail64, clk, st = time_steps(G, REP, blk, prim_h, met, G.FP64, args.steps, args.warmup,
                                        clocks=ClockSampler(uuid))
    value64 = REP.job_rate(ncells * args.steps, ms64)
    # adjoint of one step against the forward step, on the same state
    g, p64, prim, cons, ws, _, dt = st
    adj_step = None
    if not args.no_adjoint:
        adj_step = adjoint_step_ratio(G, g, p64, prim, cons, met, ws, dt, ms64 / args.steps)
    del st, prim, cons, ws
    torch.cuda.empty_cache()

    # mixed precision path, on the RHS tile shape the project's autotuner picks
    from paper_2210_17509_gb300 import autotune
    tile_mx = mixed_tile(G, args.n, args.mixed_tile)
    msmx, nfailmx, _, st = time_steps(G, REP, blk, prim_h, met, G.MIXED, args.steps, args.warmup, tile=tile_mx)
    value_mx = REP.job_rate(ncells * args.steps, msmx)
    del st
    torch.cuda.empty_cache()

    # dominant kernel: the FP64 RHS (states, faces, cells), timed live with
    # events on its stream through grmhd_rhs_cached, which runs the same
    # kernels on the same FP64 geometry cache as the step
    g, p, prim_k, _, _, _ = block_state(G, blk, prim_h, met, G.FP64)
    rhs_out = torch.empty_like(prim_k)
    rws = G.rhs_workspace(g)
    G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
    for _ in range(3):
        G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    stream = torch.cuda.current_stream()
    nk = max(5, args.steps)
    k0, k1 = _timer()
    k0.record(stream)
    for _ in range(nk):
        G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    k1.record(stream)
    torch.cuda.synchronize()
    rhs_ms = k0.elapsed_time(k1) / nk
    roof = R.rhs_fp64_roofline(ncells, rhs_ms)
    del prim_k, rhs_out, rws
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        e2e = e2e_bench(G, REP, blk, prim_h, met, max(3, args.steps))
        torch.cuda.empty_cache()
    del met, prim_h
    torch.cuda.empty_cache()

    smooth = None
    if not args.no_smooth:
        smooth = smooth_block_bench(G, REP, args.steps, args.warmup, args.smooth_n, args.mixed_tile)
    batched = None
    if not args.no_batched:
        batched = batched_bench(G, args.steps, args.warmup)
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_bench(G, n=args.adjoint_n, ndir=args.adjoint_dirs)
    tube = None
    if not args.no_shocktube:
        tube = shocktube_bench(G)
    amr = None
    if not args.no_amr:
        amr = amr_bench(G)
    ct = None
    if not args.no_ct:
        ct = ct_bench(G, n=args.smooth_n)
    poly = None
    if not args.no_poly:
        poly = poly_bench(G, n=args.smooth_n)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_sample(G, args.n)
    floor = 512.0 * 3     # per-kernel byte floor per cell per SSP-RK3 step (three stages)
    zc_mx = value_mx / world
    mixed = {"value": value_mx, "unit": UNIT, "ms_per_step": msmx / args.steps,
             "dtype": "f32 reconstruct/HLLE/divergence + f64 con2prim/metric",
             "speedup_vs_fp64": value_mx / value64, "failed_cells": nfailmx,
             "tile": autotune.BLOCK_SHAPES[tile_mx],
             "hbm_frac_512B_floor": floor * zc_mx / (hbm * 1e9)}
    summary = {
        "fp64_zc_per_s": value64, "mixed_zc_per_s": value_mx, "fp64_failed_cells": nfail64,
        "mixed_failed_cells": nfailmx,
        "fp64_hbm_frac_512B_floor": floor * value64 / world / (hbm * 1e9),
        "mixed_hbm_frac_512B_floor": mixed["hbm_frac_512B_floor"],
        "adjoint_step_ratio_256": adj_step["ratio_to_fp64_step"] if adj_step else None,
        "adjoint_forward_ratio_64cube_20steps": adjoint["adjoint_forward_ratio"] if adjoint else None,
        "roofline_frac": roof["frac"],
        "mixed_max_err_vs_oracle": (cpu["accuracy_vs_oracle"]["mixed"]["vector_scaled_max"] if cpu else None),
        "fp64_max_err_vs_oracle": (cpu["accuracy_vs_oracle"]["fp64"]["max"] if cpu else None),
    }
    line = {
        "metric": METRIC, "value": value64, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args.n),
        # per SSP-RK3 stage: the three RHS passes, the recovery and the ghost fill
        "gpu_launches": args.steps * 15,
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "mixed": mixed,
        "failed_cells": nfail64,
        "hbm_peak_gbs": {"value": hbm, "source": hbm_src},
        "adjoint_step": adj_step,
        "smooth_128": smooth,
        "batched": batched,
        "adjoint": adjoint,
        "shocktube": tube,
        "amr2": amr,
        "ct": ct,
        "polytrope": poly,
        "context": {"paper_v100_setupA_zc_per_s": PAPER_V100_SETUPA,
                    "note": "paper: 240^3, RK2, FP64, V100 (Sec. 5.1); different hardware and setup"},
        "summary": summary,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
