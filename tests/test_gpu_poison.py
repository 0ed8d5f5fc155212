"""Scratch poisoning: every workspace, face buffer and field-flux register is
filled with NaN before the call, and the results must be finite and
bit-identical to a run whose scratch was zeroed.  A kernel that read scratch
it had not written first (a face of the two-pass buffer no tile computed, an
edge field outside the ring, a stale cache) would carry a NaN into the
output.  The ghost entries of U, which no step reads, are poisoned too.
"""
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


def fill(t, poison):
    if poison:
        t.view(torch.uint8).fill_(0xFF)  # all-ones bytes: a NaN in every double and float
    else:
        t.zero_()
    return t


def poison_ghosts(a, ng=3):
    out = np.full_like(a, np.nan)
    sl = (slice(None),) + tuple(slice(ng, s - ng) for s in a.shape[1:])
    out[sl] = a[sl]
    return out


def state(n, curved=True, seed=3):
    n = tuple(n)
    h = 8.0 / max(n)
    blk = I.Block(n, 3, (h, h, h), (4.0, 4.0, 4.0))
    m = I.schwarzschild_metric(blk) if curved else None
    prim = I.smooth_prims(blk, seed, rho_range=(0.05, 1.0), metric=m)
    og = O.Grid(blk.n, 3, blk.dx)
    prim = O.fill_ghosts(og, O.BC_COPY, prim)
    return blk, m, prim


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [(19, 13, 11), (16, 16, 8)])
def test_rk_step_with_poisoned_workspace(G, precision, n):
    blk, m, prim = state(n)
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision)
    gm = cuda(m)
    cons = host(G.prim2con(g, p, cuda(prim), gm))
    out = []
    for poison in (False, True):
        gc, gp = cuda(poison_ghosts(cons) if poison else cons), cuda(prim)
        ws = fill(G.workspace(g, G.RK3), poison)
        for _ in range(2):
            G.rk_step(g, p, G.RK3, 0.25 * blk.dx[0], gc, gp, gm, ws=ws)
        out.append((host(gc), host(gp)))
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    assert np.all(np.isfinite(out[1][0][inner])) and np.all(np.isfinite(out[1][1]))
    assert np.array_equal(out[0][0][inner], out[1][0][inner])
    assert np.array_equal(out[0][1], out[1][1])


def test_rhs_cached_with_poisoned_workspace(G):
    blk, m, prim = state((24, 16, 12))
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY)
    gm, gp = cuda(m), cuda(prim)
    a = host(G.rhs_cached(g, p, gp, gm, ws=fill(G.rhs_workspace(g), False)))
    b = host(G.rhs_cached(g, p, gp, gm, ws=fill(G.rhs_workspace(g), True)))
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    assert np.all(np.isfinite(b[inner]))
    assert np.array_equal(a[inner], b[inner])


@pytest.mark.parametrize("precision", [0, 1])
def test_ct_step_with_poisoned_workspace(G, precision):
    blk, m, prim = state((19, 13, 11))
    bf = I.face_curl(blk, I.edge_potential(blk, 7))
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    bf *= 0.05 / np.abs(bf[inner]).max()
    prim = O.fill_ghosts(O.Grid(blk.n, 3, blk.dx), O.BC_COPY, O.ct_cell_field(prim, bf, m))
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_COPY, precision=precision)
    gm = cuda(m)
    cons = host(G.prim2con(g, p, cuda(prim), gm))
    out = []
    for poison in (False, True):
        gc, gp, gb = cuda(cons), cuda(prim), cuda(bf)
        ws = fill(G.ct_workspace(g, G.RK3), poison)
        G.ct_rk_step(g, p, G.RK3, 0.25 * blk.dx[0], gc, gp, gb, gm, ws=ws)
        out.append((host(gc), host(gp), host(gb)))
    for a, b in zip(out[0], out[1]):
        assert np.all(np.isfinite(b[inner]))
        assert np.array_equal(a[inner], b[inner])


def test_batch_with_poisoned_face_and_state_buffers(G):
    p = G.Params(recon=G.WENO5, bc=G.BC_PERIODIC)
    shapes = I.amr_box_shapes(8, 3)
    out = []
    for poison in (False, True):
        boxes = []
        for b, (n, lev) in enumerate(shapes):
            h = 1.0 / 2 ** lev
            blk = I.Block(n, 3, (h, h, h), (0.0, 0.0, 0.0))
            prim = I.smooth_prims(blk, 300 + b)
            g = G.Grid(blk.n, 3, blk.dx)
            tp = cuda(prim)
            G.fill_ghosts(g, G.BC_PERIODIC, tp)
            tc = G.prim2con(g, p, tp)
            faces = fill(torch.empty((24,) + g.shape, dtype=torch.float64, device="cuda"), poison)
            states = fill(torch.empty((48,) + g.shape, dtype=torch.float64, device="cuda"), poison)
            boxes.append(G.Box(g, tc, tp.clone(), torch.zeros_like(tp), None, b % 4, G.BC_PERIODIC, faces, states))
        batch = G.Batch(boxes, p, two_pass=True)
        assert batch.c.three_pass == 1
        batch.rhs(p)
        out.append([host(b.rhs)[:, 3:-3, 3:-3, 3:-3] for b in boxes])
    for a, b in zip(out[0], out[1]):
        assert np.all(np.isfinite(b))
        assert np.array_equal(a, b)
