"""Tile-shape autotuner for the RHS kernels.

Measures, on the current GPU, the cost of one RHS tile for every tile shape
(by timing grmhd_rhs on a block that all shapes cut without waste), then
picks for each box the shape that minimises  n_tiles(shape, box) * cost(shape)
-- the shape that wastes the fewest idle threads on ragged box edges weighted
by how fast that shape runs.  Costs are cached per GPU model, precision,
reconstruction and metric type in a JSON file next to the library.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import grmhd as G

SHAPES = {0: (8, 8, 4), 1: (16, 4, 4), 2: (32, 4, 2), 3: (4, 8, 8)}   # batched boxes
BLOCK_SHAPES = {**SHAPES, 4: (8, 8, 8)}                               # single blocks
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".autotune_cache.json")


def n_tiles(shape_id: int, n) -> int:
    s = BLOCK_SHAPES[shape_id]
    return math.prod((n[d] + s[d] - 1) // s[d] for d in range(3))


def _key(params: G.Params, curved: bool) -> str:
    name = torch.cuda.get_device_name()
    return f"{name}|prec{params.precision}|recon{params.recon}|curved{int(curved)}"


def measure_tile_costs(params: G.Params, curved: bool = False, n: int = 64, reps: int = 5, shapes=None) -> dict:
    """Seconds per tile for each shape, timed with CUDA events on the current stream."""
    shapes = SHAPES if shapes is None else shapes
    from . import inputs as I
    blk = I.Block((n, n, n), 3, (1.0 / n,) * 3, (4.0, 4.0, 4.0))
    met = I.schwarzschild_metric(blk) if curved else None
    prim_h = I.smooth_prims(blk, 7, rho_range=(0.1, 1.0), metric=met)
    g = G.Grid(blk.n, 3, blk.dx)
    prim = torch.from_numpy(prim_h).cuda()
    metric = None if met is None else torch.from_numpy(met).cuda()
    out = torch.empty_like(prim)
    ws = G.rhs_workspace(g)
    costs = {}
    # on a metric the steps read the geometry caches: time that kernel
    run = (lambda pp: G.rhs_cached(g, pp, prim, metric, None, out, ws)) if curved else \
        (lambda pp: G.rhs(g, pp, prim, metric, None, out))
    for sid in shapes:
        p = G.Params(**{**params.__dict__, "tile": sid})
        run(p)
        p = G.Params(**{**params.__dict__, "tile": sid, "flags": G.REUSE_GEOMETRY})
        run(p)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run(p)
        e1.record()
        torch.cuda.synchronize()
        costs[sid] = e0.elapsed_time(e1) * 1e-3 / reps / n_tiles(sid, blk.n)
    return costs


def tile_costs(params: G.Params, curved: bool = False, refresh: bool = False) -> dict:
    key = _key(params, curved)
    cache = {}
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not refresh and key in cache:
        return {int(k): v for k, v in cache[key].items()}
    costs = measure_tile_costs(params, curved)
    cache[key] = {str(k): v for k, v in costs.items()}
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)
    return costs


def choose(n, costs: dict) -> int:
    """Best tile shape (0..3) for a box of interior extent n = (nx, ny, nz)."""
    return min((sid for sid in costs if sid in SHAPES), key=lambda sid: (n_tiles(sid, n) * costs[sid], sid))


def best_block_shape(params: G.Params, n, curved: bool = False) -> int:
    """Tile shape for one large block of extent n (all five shapes timed)."""
    costs = measure_tile_costs(params, curved, shapes=BLOCK_SHAPES)
    return min(costs, key=lambda sid: (n_tiles(sid, n) * costs[sid], sid))
