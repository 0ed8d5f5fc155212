"""grmhd_rk_step_static: the step for callers that cannot allocate device memory.

Such callers (a host code whose device memory belongs to another allocator, a
callback where allocation is forbidden, a binding with no device allocator)
pass only their state buffers; the library lays the step's workspace over a
fixed device array of its own.  The step must give the same result as
grmhd_rk_step with a caller workspace of the same size class, call after
call: the shared array keeps the previous call's contents -- possibly another
block's geometry caches -- and nothing may depend on them.  Both entry points
then run the same kernels on the same data, so the results are compared bit
for bit (which implies the FP64 tolerance of the other tests).

This file is collected last, so a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, MIXED_TOL, interior, normwise

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2210_17509_gb300 import build
    build.build()
    from paper_2210_17509_gb300 import grmhd
    return grmhd


def _state(G, n, seed, origin=4.0, extent=8.0):
    blk = I.Block((n, n, n), 3, (extent / n,) * 3, (origin,) * 3)
    met = I.schwarzschild_metric(blk)
    prim = I.smooth_prims(blk, seed, rho_range=(0.1, 1.0), metric=met)
    g = G.Grid(blk.n, 3, blk.dx)
    tp = torch.from_numpy(prim).cuda()
    tm = torch.from_numpy(met).cuda()
    G.fill_ghosts(g, G.BC_COPY, tp)
    tc = G.prim2con(g, G.Params(recon=G.WENO5, bc=G.BC_COPY), tp, tm)
    return g, tc, tp, tm, blk


def _assert_same(st, ref, tol):
    a, b = st.cpu().numpy(), ref.cpu().numpy()
    assert np.all(normwise(interior(a, 3), interior(b, 3)) < tol)
    assert np.array_equal(a, b)


def _workspace(G, g, scheme, cached):
    n = G.rk_workspace_bytes_cached(g, scheme) if cached else G.rk_workspace_bytes(g, scheme)
    return torch.empty(n, dtype=torch.uint8, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_static_scratch_step_matches_workspace_step(G, scheme, precision):
    """A 24^3 block: its cached workspace fits in the array, so both entry
    points take the cached paths; two calls in a row through each."""
    prec = G.FP64 if precision == "fp64" else G.MIXED
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec)
    g, tc, tp, tm, blk = _state(G, 24, 3)
    assert G.rk_workspace_bytes_cached(g, scheme) <= G.STATIC_SCRATCH_BYTES
    dt = 0.25 * blk.dx[0]
    ref_c, ref_p = tc.clone(), tp.clone()
    st_c, st_p = tc.clone(), tp.clone()
    ws = _workspace(G, g, scheme, cached=True)
    so = ctypes.CDLL(G.LIB_PATH)
    assert hasattr(so, "grmhd_rk_step_static")
    tol = FP64_TOL if prec == G.FP64 else MIXED_TOL
    for _ in range(2):
        G.rk_step(g, p, scheme, dt, ref_c, ref_p, tm, None, ws)
        G.rk_step_static(g, p, scheme, dt, st_c, st_p, tm)
        torch.cuda.synchronize()
        _assert_same(st_c, ref_c, tol)
        _assert_same(st_p, ref_p, tol)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_scratch_uncached_block(G, precision):
    """A 64^3 block: the plain workspace fits in the array, the cached one does
    not, so the step takes the uncached paths, as grmhd_rk_step does with a
    workspace of grmhd_rk_workspace_bytes."""
    prec = G.FP64 if precision == "fp64" else G.MIXED
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec)
    g, tc, tp, tm, blk = _state(G, 64, 5)
    assert G.rk_workspace_bytes(g, G.RK3) <= G.STATIC_SCRATCH_BYTES < G.rk_workspace_bytes_cached(g, G.RK3)
    dt = 0.25 * blk.dx[0]
    ref_c, ref_p = tc.clone(), tp.clone()
    st_c, st_p = tc.clone(), tp.clone()
    ws = _workspace(G, g, G.RK3, cached=False)
    tol = FP64_TOL if prec == G.FP64 else MIXED_TOL
    for _ in range(2):
        G.rk_step(g, p, G.RK3, dt, ref_c, ref_p, tm, None, ws)
        G.rk_step_static(g, p, G.RK3, dt, st_c, st_p, tm)
        torch.cuda.synchronize()
        _assert_same(st_c, ref_c, tol)
        _assert_same(st_p, ref_p, tol)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_scratch_alternating_blocks_with_reuse_flag(G, precision):
    """Two blocks with different grids and metrics stepped in turn, with
    GRMHD_REUSE_GEOMETRY set: the static step ignores the flag (the shared
    array holds the other block's caches), so each block gets the result of
    its own workspace step, whose workspace really does keep its caches."""
    prec = G.FP64 if precision == "fp64" else G.MIXED
    first = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec)
    reuse = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=prec, flags=G.REUSE_GEOMETRY)
    blocks = []
    for n, seed, origin, extent in ((24, 3, 4.0, 8.0), (20, 8, 6.0, 5.0)):
        g, tc, tp, tm, blk = _state(G, n, seed, origin, extent)
        blocks.append(dict(g=g, tm=tm, dt=0.25 * blk.dx[0], ws=_workspace(G, g, G.RK3, cached=True),
                           ref=[tc.clone(), tp.clone()], st=[tc.clone(), tp.clone()]))
    tol = FP64_TOL if prec == G.FP64 else MIXED_TOL
    for it in range(3):
        for b in blocks:
            G.rk_step(b["g"], first if it == 0 else reuse, G.RK3, b["dt"], *b["ref"], b["tm"], None, b["ws"])
            G.rk_step_static(b["g"], reuse, G.RK3, b["dt"], *b["st"], b["tm"])
        torch.cuda.synchronize()
        for b in blocks:
            _assert_same(b["st"][0], b["ref"][0], tol)
            _assert_same(b["st"][1], b["ref"][1], tol)


@pytest.mark.gpu
def test_static_scratch_rejects_blocks_beyond_its_size(G):
    # 100^3 interior + ghosts needs 8 * 106^3 * 8 B > 64 MiB for RK3: refused before any launch
    grid = G.Grid((100, 100, 100), 3, (0.1, 0.1, 0.1))
    assert G.rk_workspace_bytes(grid, G.RK3) > G.STATIC_SCRATCH_BYTES
    fake = ctypes.c_void_p(0x1000)
    rc = G._lib.grmhd_rk_step_static(ctypes.byref(grid.c()), ctypes.byref(G.Params().c()), G.RK3, 0.01,
                                     fake, fake, None, None, None, None)
    assert rc == -4
