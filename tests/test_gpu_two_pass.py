"""The RHS of the cached paths in several passes against the single-pass
tile kernel (GRMHD_SINGLE_PASS).  FP64: WENO5 in three passes (the face states
of every cell into a state buffer, every face flux once into a face buffer,
then a per-cell pass), minmod in two (tiled faces, per-cell pass): the same
reconstruction, face routine and per-cell operations, so the results are
bit-identical.  Blocks that end inside a tile (ragged) and exactly at a tile
boundary are both covered, with and without constrained transport, and blocks
one cell thick along each axis.  The mixed path keeps the fused single pass.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2210_17509_gb300 import build
    build.build()
    from paper_2210_17509_gb300 import grmhd
    return grmhd


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def state(n):
    h = 8.0 / max(n)
    blk = I.Block(tuple(n), 3, (h, h, h), (4.0, 4.0, 4.0))
    m = I.schwarzschild_metric(blk)
    prim = I.smooth_prims(blk, 3, rho_range=(0.05, 1.0), metric=m)
    prim = O.fill_ghosts(O.Grid(blk.n, 3, blk.dx), O.BC_COPY, prim)
    return blk, m, prim


@pytest.mark.parametrize("n", [(19, 13, 11), (16, 16, 8), (8, 24, 12), (9, 7, 1), (1, 10, 6), (8, 1, 5)])
@pytest.mark.parametrize("recon", ["weno5", "minmod"])
def test_rk_steps_bit_identical(G, n, recon):
    blk, m, prim = state(n)
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5 if recon == "weno5" else G.MINMOD, bc=G.BC_COPY)
    gm = cuda(m)
    out = []
    for flags in (0, G.SINGLE_PASS):
        pp = dataclasses.replace(p, flags=flags)
        gp = cuda(prim)
        gc = G.prim2con(g, pp, gp, gm)
        ws = G.workspace(g, G.RK3)
        for _ in range(2):
            G.rk_step(g, pp, G.RK3, 0.25 * blk.dx[0], gc, gp, gm, ws=ws)
        out.append((host(gc), host(gp)))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_rhs_cached_bit_identical(G):
    blk, m, prim = state((24, 16, 12))
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    gm, gp = cuda(m), cuda(prim)
    ws = G.rhs_workspace(g)
    a = host(G.rhs_cached(g, p, gp, gm, ws=ws))
    b = host(G.rhs_cached(g, dataclasses.replace(p, flags=G.SINGLE_PASS), gp, gm, ws=ws))
    assert np.array_equal(a, b)
    assert np.abs(a).max() > 0.0


@pytest.mark.parametrize("n", [(19, 13, 11), (16, 16, 8)])
def test_ct_step_bit_identical(G, n):
    blk, m, prim = state(n)
    bf = I.face_curl(blk, I.edge_potential(blk, 5))
    inner = (slice(None),) + tuple(slice(3, s - 3) for s in blk.shape)
    bf *= 0.05 / np.abs(bf[inner]).max()
    prim = O.fill_ghosts(O.Grid(blk.n, 3, blk.dx), O.BC_COPY, O.ct_cell_field(prim, bf, m))
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    gm = cuda(m)
    out = []
    for flags in (0, G.SINGLE_PASS):
        pp = dataclasses.replace(p, flags=flags)
        gp, gb = cuda(prim), cuda(bf)
        gc = G.prim2con(g, pp, gp, gm)
        G.ct_rk_step(g, pp, G.RK3, 0.25 * blk.dx[0], gc, gp, gb, gm)
        out.append((host(gc), host(gp), host(gb)))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_rk_steps_multi_pass_against_oracle(G, precision):
    """SSP-RK3 steps on the cached paths (FP64 in several passes, mixed in
    the fused pass) against the oracle, ragged block."""
    from tests.helpers import FP64_TOL, MIXED_TOL, normwise
    blk, m, prim = state((19, 13, 11))
    og = O.Grid(blk.n, 3, blk.dx)
    op = O.make_params(recon=O.REC_WENO5, bc=O.BC_COPY)
    cons = O.prim2con(og, op.gamma, prim, m)
    dt = 0.25 * blk.dx[0]
    c, pr = cons, prim
    for _ in range(2):
        c, pr, nf = O.rk_step(og, op, O.RK3, dt, c, pr, m)
        assert nf == 0
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision)
    gc, gp, gm = cuda(cons), cuda(prim), cuda(m)
    ws = G.workspace(g, G.RK3)
    for _ in range(2):
        G.rk_step(g, p, G.RK3, dt, gc, gp, gm, ws=ws)
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    assert np.all(normwise(host(gc)[inner], c[inner]) <= tol)
