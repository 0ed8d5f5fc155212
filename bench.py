"""Benchmark of the GRMHD method-of-lines hot path on GB300.

One step = one full SSP-RK3 step of the 128^3 + 3-ghost Schwarzschild block
(WENO5, HLLE, copy boundaries, CFL 0.25): three stages of RHS with the stage
update (FP64: face states, face fluxes, then the per-cell pass; mixed: one
fused kernel), con2prim and ghost fill.  Metric: zone-cycles/s =
steps * interior cells / time (the paper's definition, Sec. 5).

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
N_CELLS_SIDE = 128
CFL = 0.25
PAPER_V100_SETUPA = 0.47e8   # zone-cycles/s, 240^3, RK2, one V100 (Sec. 5.1) -- context only


def workload_config(n=N_CELLS_SIDE):
    return {
        "workload": f"schwarzschild-block-{n}^3+3ghost-weno5-hlle-ssprk3",
        "block": [n, n, n], "ghosts": 3, "spacetime": "Schwarzschild isotropic M=1, block [4,12]^3",
        "recon": "WENO5", "riemann": "HLLE", "integrator": "SSP-RK3", "cfl": CFL, "bc": "copy",
        "gamma": I.GAMMA, "l2": "inputs larger than L2 (prim+cons+metric ~ 500 MB per block)",
        "geometry_cache": "static metric: geometry caches built once (first step), reused (GRMHD_REUSE_GEOMETRY)",
    }


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
    blk, prim, met = I.smooth_schwarzschild(N_CELLS_SIDE, seed=1)
    # bounded sample: a 24^3 sub-block (cells [52, 76)^3 of the full block, with ghosts)
    sub = 24
    lo = 52
    sl = (slice(None),) + tuple(slice(lo, lo + sub + 6) for _ in range(3))
    sblk = I.Block((sub,) * 3, 3, blk.dx, tuple(blk.origin[d] + (lo - 3 + 3) * blk.dx[d] for d in range(3)))
    sprim = np.ascontiguousarray(prim[sl])
    smet = np.ascontiguousarray(met[sl])
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
    sample = (f"{args.steps} SSP-RK3 steps of a {sub}^3 sub-block of the {N_CELLS_SIDE}^3 Schwarzschild "
              f"workload (same cells, metric, WENO5/HLLE/copy BC), oracle with {nthreads} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(G, seconds_target=15.0):
    """Oracle throughput on a bounded sample (about 10-30 s of CPU work).
    Its first step also gives the accuracy report: the max relative error of
    every conserved field of the FP64 and the mixed GPU paths against the
    FP64 oracle after one SSP-RK3 step of the same sample."""
    import torch
    import oracle as O
    O.build()
    nthreads = os.cpu_count() or 1
    O.set_threads(nthreads)
    blk, prim, met = I.smooth_schwarzschild(N_CELLS_SIDE, seed=1)
    sub, lo = 48, 40
    sl = (slice(None),) + tuple(slice(lo, lo + sub + 6) for _ in range(3))
    sblk = I.Block((sub,) * 3, 3, blk.dx, blk.origin)
    sprim = np.ascontiguousarray(prim[sl])
    smet = np.ascontiguousarray(met[sl])
    g = O.Grid(sblk.n, 3, sblk.dx)
    gp = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_COPY, rho_atm=gp.rho_atm, p_atm=gp.p_atm, weno_eps=gp.weno_eps)
    sprim = O.fill_ghosts(g, O.BC_COPY, sprim)
    cons = O.prim2con(g, par.gamma, sprim, smet)
    dt = CFL * min(sblk.dx)
    cons0, prim0 = cons, sprim
    cons, sprim, _ = O.rk_step(g, par, O.RK3, dt, cons, sprim, smet)     # warm-up, and the reference step
    gg = G.Grid(sblk.n, 3, sblk.dx)
    inner = (slice(None),) + tuple(slice(3, -3) for _ in range(3))
    accuracy = {"sample": f"one SSP-RK3 step of the {sub}^3 sub-block",
                "fields": ["D", "S_x", "S_y", "S_z", "tau", "B^x", "B^y", "B^z"]}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        tc = torch.from_numpy(cons0).cuda()
        tp = torch.from_numpy(prim0).cuda()
        G.rk_step(gg, dataclasses.replace(gp, precision=prec), G.RK3, dt, tc, tp, torch.from_numpy(smet).cuda(),
                  None, G.workspace(gg, G.RK3))
        c = tc.cpu().numpy()[inner]
        ref = cons[inner]
        err = [float(np.abs(c[q] - ref[q]).max() / np.abs(ref[q]).max()) for q in range(8)]
        accuracy[name] = {"max_rel_err_per_field": err, "max": max(err)}
    steps, t = 0, 0.0
    t0 = time.perf_counter()
    while t < seconds_target and steps < 400:
        cons, sprim, _ = O.rk_step(g, par, O.RK3, dt, cons, sprim, smet)
        steps += 1
        t = time.perf_counter() - t0
    return {
        "value": steps * sblk.ncells / t, "unit": UNIT, "cores": nthreads, "kind": "oracle",
        "sample": f"{steps} SSP-RK3 steps of a {sub}^3 sub-block of the same Schwarzschild workload "
                  f"({t:.1f} s of CPU work, {nthreads} OpenMP threads)",
        "accuracy_vs_oracle": accuracy,
    }


# --------------------------------------------------------------- batched --
def batched_bench(G, steps, warmup, nbox=512):
    """512 AMR-like boxes (edges from {8..64}, 3 refinement levels, flat):
    recovery + ghost fill + RHS of every box as one graph of persistent
    launches (three; five for the three-pass FP64 WENO5 RHS), against the plain form
    (three launches per box)."""
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
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(max(warmup, 1)):
                batch.rhs(p)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            batch.rhs(p)
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            graph.replay()
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
                     "ms_per_batch": ms, "plain_per_box_ms": ms_plain, "speedup_vs_plain": ms_plain / ms,
                     "gpu_launches_per_batch": (3 + (batch.c.two_pass + batch.c.three_pass
                                                     if precision == G.FP64 else 0)),
                     "multi_pass": ("three passes" if batch.c.three_pass and precision == G.FP64 else
                                    "two passes" if batch.c.two_pass and precision == G.FP64 else "one pass"),
                     "tile_shapes": tiles_used}
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

    def run(with_grad):
        x = prim0.clone().requires_grad_(with_grad)
        gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=with_grad)
        L = A.density_l2(A.evolve(x, gam, g, p, G.RK3, dt, nsteps, checkpoint_every=every), g)
        return x, gam, L

    run(True)[2].backward()          # warm-up (module load, workspaces)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    x, gam, L = run(True)
    e1.record()
    L.backward()
    e2.record()
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1)
    t_bwd = e1.elapsed_time(e2)
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
        "forward_ms": t_fwd, "backward_ms": t_bwd, "forward_plain_ms": t_plain,
        "adjoint_forward_ratio": t_bwd / t_fwd, "adjoint_plain_forward_ratio": t_bwd / t_plain,
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
def ct_bench(G, steps=5, warmup=2, n=N_CELLS_SIDE):
    """Constrained transport (Sec. 3: the field on staggered grids): the
    headline 128^3 Schwarzschild block with a divergence-free face field (the
    discrete curl of a random edge potential, |sqrt(gamma) B| <= 0.03, so
    b^2/rho <= 0.2 on the density floor of 1e-3; cell field = mean of the
    faces), WENO5+HLLE, SSP-RK3 at the headline dt, FP64 and mixed.  Timed
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
    prim_h = I.ct_state(blk, prim_h, bf_h, met_h)
    g = G.Grid(blk.n, blk.ng, blk.dx)
    met = torch.from_numpy(met_h).cuda()
    dt = CFL * min(blk.dx)
    out = {"workload": f"{n}^3 Schwarzschild block (headline state) with a divergence-free face field "
                       f"(|sqrt(gamma) B| <= 0.03), "
                       f"WENO5+HLLE, SSP-RK3, dt = {CFL} dx, copy boundaries"}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        res = {}
        for mode in ("plain", "ct"):
            p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec)
            prim = torch.from_numpy(prim_h).cuda()
            G.fill_ghosts(g, G.BC_COPY, prim)
            cons = G.prim2con(g, p, prim, met)
            b = torch.from_numpy(bf_h).cuda()
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
def poly_bench(G, steps=5, warmup=2, n=N_CELLS_SIDE, K=100.0, gamma=2.0):
    """Polytropic EOS (Sec. 2.3; K = 100, Gamma = 2 as the paper's TOV star,
    Sec. 4.4): the headline 128^3 Schwarzschild block with a smooth state of
    density 1e-4 .. 1.28e-3 (the TOV central density), P = K rho^Gamma,
    |v| <= 0.5 and a weak field (|B| <= 1e-3), WENO5+HLLE, SSP-RK3 at the
    headline dt, copy boundaries; FP64 and mixed."""
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


# ------------------------------------------------------------ 256^3 block --
def large_block_bench(G, steps=3, warmup=1, n=256):
    """256^3 + 3 ghosts on the Schwarzschild background, planar Riemann jump
    along x with 1% perturbation, WENO5+HLLE, SSP-RK3: FP64, mixed and the
    adjoint step, each with its HBM fraction against the per-kernel
    algorithmic byte floor (512 B per cell per stage)."""
    import torch
    blk, prim_h, met_h = I.riemann_schwarzschild(n, seed=4)
    g = G.Grid(blk.n, blk.ng, blk.dx)
    dt = CFL * min(blk.dx)
    met = torch.from_numpy(met_h).cuda()
    from paper_2210_17509_gb300 import roofline as R
    hbm, _ = R.hbm_peak_gbs()
    out = {"workload": f"Riemann jump on Schwarzschild, {n}^3+3 ghosts, WENO5+HLLE, SSP-RK3, copy BC"}
    ncells = blk.ncells
    for precision, name in ((G.FP64, "fp64"), (G.MIXED, "mixed")):
        p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision)
        prim = torch.from_numpy(prim_h).cuda()
        G.fill_ghosts(g, G.BC_COPY, prim)
        cons = G.prim2con(g, p, prim, met)
        ws = G.workspace(g, G.RK3)
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
            p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        zc = ncells / (ms * 1e-3)
        out[name] = {"value": zc, "unit": UNIT, "ms_per_step": ms, "failed_cells": int(nfail.item()),
                     "hbm_frac_512B_floor": 512.0 * 3 * zc / (hbm * 1e9)}
        if precision == G.FP64:
            # adjoint of one step from recorded stages (the checkpointed backward's unit of work)
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
            e0.record()
            G.rk_step_adjoint(g, p, G.RK3, dt, c0, p0, ub, pb, gb, met, None, wsa, stage_prims=stages)
            e1.record()
            torch.cuda.synchronize()
            ams = e0.elapsed_time(e1)
            out["adjoint_step"] = {"ms": ams, "ratio_to_fp64_step": ams / ms, "value": ncells / (ams * 1e-3),
                                   "unit": "zone-cycles/s (reverse step, recorded stages)"}
            del stages, wsa, ub, pb, c0, p0
        del prim, cons, ws
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------- GPU --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grmhd", choices=["grmhd", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS_SIDE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-shocktube", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-ct", action="store_true")
    ap.add_argument("--no-poly", action="store_true")
    ap.add_argument("--section", default=None, choices=["ct", "poly", "amr", "shocktube", "batched", "adjoint", "large"],
                    help="run only this section and print its JSON (profiling runs)")
    ap.add_argument("--tile", type=int, default=-1, help="RHS tile shape (default: autotuned)")
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

    if args.section:
        fns = {"ct": lambda: ct_bench(G, n=args.n), "poly": lambda: poly_bench(G, n=args.n), "amr": lambda: amr_bench(G), "shocktube": lambda: shocktube_bench(G),
               "batched": lambda: batched_bench(G, args.steps, args.warmup),
               "adjoint": lambda: adjoint_bench(G, n=args.adjoint_n, ndir=args.adjoint_dirs),
               "large": lambda: large_block_bench(G)}
        out = fns[args.section]()
        if rank == 0:
            print(json.dumps({"section": args.section, args.section: out}), flush=True)
        return

    def barrier():
        REP.barrier()

    blk, prim_h, met_h = I.smooth_schwarzschild(args.n, seed=1 + rank)
    g = G.Grid(blk.n, blk.ng, blk.dx)
    dt = CFL * min(blk.dx)
    met = torch.from_numpy(met_h).cuda()
    stream = torch.cuda.current_stream()

    # tile shape of the single block from the project's autotuner (per precision)
    from paper_2210_17509_gb300 import autotune
    # (the FP64 RHS of the cached step runs in three passes, without tiles,
    # whatever the tile parameter says; the mixed RHS takes the tuned shape)
    if args.tile >= 0:
        tiles = {G.FP64: args.tile, G.MIXED: args.tile}
    else:
        tiles = {G.FP64: 0,
                 G.MIXED: autotune.best_block_shape(G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=G.MIXED), blk.n,
                                                    curved=True)}

    def setup(precision):
        p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision, tile=tiles[precision])
        prim = torch.from_numpy(prim_h).cuda()
        G.fill_ghosts(g, G.BC_COPY, prim)
        cons = G.prim2con(g, p, prim, met)
        ws = G.workspace(g, G.RK3)
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
        return p, prim, cons, ws, nfail

    def timed(precision, steps, warmup):
        p, prim, cons, ws, nfail = setup(precision)
        for i in range(warmup):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
            # static metric: the geometry cache built by the first step is kept
            p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            G.rk_step(g, p, G.RK3, dt, cons, prim, met, None, ws, nfail)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = REP.max_over_ranks(e0.elapsed_time(e1))
        return ms, int(nfail.item())

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    # FP64 (headline) -- clocks sampled during this timed region
    p64, prim, cons, ws, nfail = setup(G.FP64)
    for _ in range(args.warmup):
        G.rk_step(g, p64, G.RK3, dt, cons, prim, met, None, ws, nfail)
        p64 = dataclasses.replace(p64, flags=G.REUSE_GEOMETRY)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        G.rk_step(g, p64, G.RK3, dt, cons, prim, met, None, ws, nfail)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms64 = REP.max_over_ranks(e0.elapsed_time(e1))
    nfail64 = int(nfail.item())
    ncells = blk.ncells
    value64 = REP.job_rate(ncells * args.steps, ms64)

    # mixed precision path
    msmx, nfailmx = timed(G.MIXED, args.steps, args.warmup)
    value_mx = REP.job_rate(ncells * args.steps, msmx)

    # dominant kernel: the fused FP64 RHS, timed live with events on its stream
    # (the RK step's RHS reads the FP64 geometry cache of the static metric,
    # so the same kernel is timed here through grmhd_rhs_cached)
    p, prim_k, cons_k, _, _ = setup(G.FP64)
    rhs_out = torch.empty_like(prim_k)
    rws = G.rhs_workspace(g)
    G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    p = dataclasses.replace(p, flags=G.REUSE_GEOMETRY)
    for _ in range(3):
        G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    nk = max(5, args.steps)
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(nk):
        G.rhs_cached(g, p, prim_k, met, None, rhs_out, rws)
    k1.record(stream)
    torch.cuda.synchronize()
    rhs_ms = k0.elapsed_time(k1) / nk
    from paper_2210_17509_gb300 import roofline as R
    roof = R.rhs_fp64_roofline(ncells, rhs_ms)

    # end to end through the public API with host buffers: every step uploads
    # its inputs (U, primitives, metric) from pinned host memory, runs
    # grmhd_rk_step and downloads its result (U, primitives).  Two device
    # buffer sets let step k + 1's upload and step k - 1's download run on
    # copy streams while step k computes (a user streaming steps would do the
    # same); the serial figure (copies, then compute, then copies) is kept too.
    e2e = None
    if not args.no_e2e:
        p, prim_d, cons_d, ws_e, nfail_e = setup(G.FP64)
        cons_h = cons_d.cpu().pin_memory()
        prim_h2 = prim_d.cpu().pin_memory()
        met_hp = met.cpu().pin_memory()
        steps_e = max(3, args.steps // 2)
        bufs = []
        for _ in range(2):
            bufs.append({"cons": torch.empty_like(cons_d), "prim": torch.empty_like(prim_d),
                         "met": torch.empty_like(met), "out_c": torch.empty_like(cons_h).pin_memory(),
                         "out_p": torch.empty_like(prim_h2).pin_memory()})
        s_comp = stream
        s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
        ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("up", "done", "down")}

        def serial_step(b):
            b["cons"].copy_(cons_h, non_blocking=True)
            b["prim"].copy_(prim_h2, non_blocking=True)
            b["met"].copy_(met_hp, non_blocking=True)
            G.rk_step(g, p, G.RK3, dt, b["cons"], b["prim"], b["met"], None, ws_e, nfail_e)
            b["out_c"].copy_(b["cons"], non_blocking=True)
            b["out_p"].copy_(b["prim"], non_blocking=True)

        def pipelined(n):
            # uploads and downloads on streams of their own, so that step
            # k + 1's upload is not queued behind step k's download
            for k in range(n):
                i = k % 2
                b = bufs[i]
                with torch.cuda.stream(s_up):
                    if k >= 2:
                        s_up.wait_event(ev["down"][i])
                    b["cons"].copy_(cons_h, non_blocking=True)
                    b["prim"].copy_(prim_h2, non_blocking=True)
                    b["met"].copy_(met_hp, non_blocking=True)
                    ev["up"][i].record(s_up)
                s_comp.wait_event(ev["up"][i])
                G.rk_step(g, p, G.RK3, dt, b["cons"], b["prim"], b["met"], None, ws_e, nfail_e, stream=s_comp)
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
            barrier()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(s_comp)
            fn()
            q1.record(s_comp)
            torch.cuda.synchronize()
            barrier()
            return REP.max_over_ranks(q0.elapsed_time(q1))

        serial_step(bufs[0])
        pipelined(2)
        ems_serial = timed_e2e(lambda: [serial_step(bufs[0]) for _ in range(steps_e)])
        ems = timed_e2e(lambda: pipelined(steps_e))
        h2d = cons_h.numel() * 8 + prim_h2.numel() * 8 + met_hp.numel() * 8
        d2h = bufs[0]["out_c"].numel() * 8 + bufs[0]["out_p"].numel() * 8
        e2e = {"value": REP.job_rate(ncells * steps_e, ems), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "dtype": "f64", "steps": steps_e,
               "copies": "overlapped with the neighbouring steps' compute (two device buffer sets, upload and "
                         "download streams)",
               "serial_value": REP.job_rate(ncells * steps_e, ems_serial)}

    batched = None
    if not args.no_batched:
        batched = batched_bench(G, args.steps, args.warmup)
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_bench(G, n=args.adjoint_n, ndir=args.adjoint_dirs)
    large = None
    if not args.no_large:
        large = large_block_bench(G)
    tube = None
    if not args.no_shocktube:
        tube = shocktube_bench(G)
    amr = None
    if not args.no_amr:
        amr = amr_bench(G)
    ct = None
    if not args.no_ct:
        ct = ct_bench(G, n=args.n)
    poly = None
    if not args.no_poly:
        poly = poly_bench(G, n=args.n)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_sample(G)
    line = {
        "metric": METRIC, "value": value64, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args.n),
        "mixed": {"value": value_mx, "unit": UNIT, "ms_per_step": msmx / args.steps,
                  "dtype": "f32 reconstruct/HLLE/divergence + f64 con2prim/metric",
                  "speedup_vs_fp64": value_mx / value64, "failed_cells": nfailmx},
        "failed_cells": nfail64,
        "tile_shapes": {"fp64": "none (three-pass RHS: states, faces, cells)",
                        "mixed": autotune.BLOCK_SHAPES[tiles[G.MIXED]]},
        # per SSP-RK3 stage: the three RHS passes, the recovery and the ghost fill
        "gpu_launches": args.steps * 15,
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
        "batched": batched,
        "adjoint": adjoint,
        "block_256": large,
        "shocktube": tube,
        "amr2": amr,
        "ct": ct,
        "polytrope": poly,
        "cpu_baseline": cpu,
        "context": {"paper_v100_setupA_zc_per_s": PAPER_V100_SETUPA,
                    "note": "paper: 240^3, RK2, FP64, V100 (Sec. 5.1); different hardware and setup"},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
