"""grmhd_rk_step_static: the step for callers that cannot allocate device memory.

It must give the same result as grmhd_rk_step with a caller workspace, call
after call (the shared library-owned scratch keeps the previous call's
contents, which the step must not depend on).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, interior, normwise

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2210_17509_gb300 import build
    build.build()
    from paper_2210_17509_gb300 import grmhd
    return grmhd


def _state(G, n, seed):
    blk = I.Block((n, n, n), 3, (8.0 / n,) * 3, (4.0, 4.0, 4.0))
    met = I.schwarzschild_metric(blk)
    prim = I.smooth_prims(blk, seed, rho_range=(0.1, 1.0), metric=met)
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    tp = torch.from_numpy(prim).cuda()
    tm = torch.from_numpy(met).cuda()
    G.fill_ghosts(g, G.BC_COPY, tp)
    tc = G.prim2con(g, p, tp, tm)
    return g, p, tc, tp, tm, blk


@pytest.mark.gpu
@pytest.mark.parametrize("scheme", [3, 4])
def test_static_scratch_step_matches_workspace_step(G, scheme):
    g, p, tc, tp, tm, blk = _state(G, 24, 3)
    dt = 0.25 * blk.dx[0]
    ref_c, ref_p = tc.clone(), tp.clone()
    st_c, st_p = tc.clone(), tp.clone()
    ws = G.workspace(g, scheme)
    for _ in range(2):       # two calls in a row through each entry point
        G.rk_step(g, p, scheme, dt, ref_c, ref_p, tm, None, ws)
        so = ctypes.CDLL(G.LIB_PATH)
        assert hasattr(so, "grmhd_rk_step_static")
        G.rk_step_static(g, p, scheme, dt, st_c, st_p, tm)
        torch.cuda.synchronize()
        a, b = st_c.cpu().numpy(), ref_c.cpu().numpy()
        assert np.all(normwise(interior(a, 3), interior(b, 3)) < FP64_TOL)
        a, b = st_p.cpu().numpy(), ref_p.cpu().numpy()
        assert np.all(normwise(interior(a, 3), interior(b, 3)) < FP64_TOL)


@pytest.mark.gpu
def test_static_scratch_rejects_blocks_beyond_its_size(G):
    # 100^3 interior + ghosts needs 8 * 106^3 * 8 B > 64 MiB for RK3: refused before any launch
    grid = G.Grid((100, 100, 100), 3, (0.1, 0.1, 0.1))
    assert G.rk_workspace_bytes(grid, G.RK3) > G.STATIC_SCRATCH_BYTES
    fake = ctypes.c_void_p(0x1000)
    rc = G._lib.grmhd_rk_step_static(ctypes.byref(grid.c()), ctypes.byref(G.Params().c()), G.RK3, 0.01,
                                     fake, fake, None, None, None, None)
    assert rc == -4
