"""Edge cases of the CUDA path through the C ABI, against the FP64 oracle:
a single-cell periodic block (every stencil sees one value: RHS exactly 0),
one-cell-thick blocks along each axis (ragged tiles with a degenerate
extent), the unmagnetised (hydro) limit and a fluid at rest in a curved
metric (where the RHS is the hydrostatic source balance)."""
import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, interior, normwise

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


def rhs_both(G, blk, prim, met, recon, bc):
    g = G.Grid(blk.n, blk.ng, blk.dx)
    og = O.Grid(blk.n, blk.ng, blk.dx)
    gp = G.Params(recon=recon, bc=bc)
    op = O.make_params(recon=recon, bc=bc, rho_atm=gp.rho_atm, p_atm=gp.p_atm, weno_eps=gp.weno_eps)
    prim = O.fill_ghosts(og, bc, prim)
    r = G.rhs(g, gp, cuda(prim), None if met is None else cuda(met)).cpu().numpy()
    ro = O.rhs(og, op, prim, met)
    return interior(r, blk.ng), interior(ro, blk.ng)


@pytest.mark.parametrize("recon", [0, 1])
def test_single_cell_periodic_block_has_zero_rhs(G, recon):
    blk = I.Block((1, 1, 1), 3, (0.1, 0.1, 0.1), (0.0, 0.0, 0.0))
    prim = np.zeros((8,) + blk.shape)
    prim[:, 3, 3, 3] = [0.7, 0.3, -0.2, 0.1, 0.4, 0.2, -0.1, 0.3]
    r, ro = rhs_both(G, blk, prim, None, recon, G.BC_PERIODIC)
    assert np.all(r == 0.0)
    assert np.all(np.abs(ro) < 1e-14)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("recon", [0, 1])
def test_one_cell_thick_blocks(G, axis, recon):
    n = [1, 1, 1]
    n[axis] = 37
    n[(axis + 1) % 3] = 5
    blk = I.Block(tuple(n), 3, tuple(1.0 / max(n) for _ in range(3)), (0.0, 0.0, 0.0))
    prim = I.smooth_prims(blk, 12)
    r, ro = rhs_both(G, blk, prim, None, recon, G.BC_COPY)
    assert normwise(r, ro, floor=1e-12).max() <= FP64_TOL


def test_hydro_limit_no_field(G):
    blk = I.Block((12, 10, 9), 3, (0.1, 0.1, 0.1), (0.0, 0.0, 0.0))
    prim = I.smooth_prims(blk, 13)
    prim[5:] = 0.0
    r, ro = rhs_both(G, blk, prim, None, 1, G.BC_PERIODIC)
    assert np.all(r[5:] == 0.0)
    assert normwise(r[:5], ro[:5]).max() <= FP64_TOL


def test_fluid_at_rest_in_schwarzschild(G):
    """v = 0, B = 0, uniform rho and P on the curved background: the RHS is the pressure-gradient-free
    gravitational source (plus the flux divergence of the non-uniform lapse and volume element)."""
    n = 14
    h = 8.0 / n
    blk = I.Block((n,) * 3, 3, (h,) * 3, (4.0,) * 3)
    met = I.schwarzschild_metric(blk)
    prim = np.zeros((8,) + blk.shape)
    prim[0] = 0.5
    prim[4] = 0.2
    r, ro = rhs_both(G, blk, prim, met, 1, G.BC_COPY)
    # no mass flux at rest (both face states equal, zero shift): D's RHS is exactly 0
    assert np.all(r[0] == 0.0)
    assert normwise(r[1:5], ro[1:5], floor=1e-12).max() <= FP64_TOL
