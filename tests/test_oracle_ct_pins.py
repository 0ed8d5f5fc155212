"""Pins of the oracle's constrained transport (reading R19: face field,
edge electric field averaged from the four face fluxes around each edge,
Sec. 3's staggered grids) against what the mathematics fixes:

* the discrete curl of an edge potential has zero discrete divergence, and
  CT steps keep it zero to round-off;
* a uniform state stays uniform; with no field, a CT step is the plain step;
* on a periodic block the field flux through every coordinate plane is
  conserved (the edge fields telescope);
* advecting a weak field with a uniform flow converges to the exactly
  advected face field (the edge fields carry the right signs and centring).
"""
import numpy as np

import oracle as O
from paper_2210_17509_gb300 import inputs as I


def block(n):
    if isinstance(n, int):
        n = (n, n, n)
    return I.Block(tuple(n), 3, tuple(1.0 / v for v in n), (0.0, 0.0, 0.0))


def ct_setup(blk, seed=1, bmax=0.1, prim=None):
    g = O.Grid(blk.n, blk.ng, blk.dx)
    if prim is None:
        prim = I.smooth_prims(blk, seed)
    A = I.edge_potential(blk, seed + 100)
    bf = I.face_curl(blk, A)
    bf *= bmax / np.abs(bf[:, 3:-3, 3:-3, 3:-3]).max()
    prim = O.ct_cell_field(prim, bf)
    prim = O.fill_ghosts(g, O.BC_PERIODIC, prim)
    return g, prim, bf


def max_div(g, bf):
    return np.abs(O.ct_divergence(g, bf)).max()


def test_face_curl_is_divergence_free():
    blk = block((12, 10, 8))
    A = I.edge_potential(blk, 3)
    bf = I.face_curl(blk, A)
    scale = np.abs(bf).max() / min(blk.dx)
    assert max_div(O.Grid(blk.n, 3, blk.dx), bf) <= 1e-14 * scale


def test_ct_steps_keep_the_divergence_at_round_off():
    blk = block(12)
    g, prim, bf = ct_setup(blk)
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_PERIODIC)
    cons = O.prim2con(g, par.gamma, prim)
    scale = np.abs(bf).max() / blk.dx[0]
    for scheme in (O.RK2, O.RK3, O.RK4):
        c, p, b, nf = cons, prim, bf, 0
        for _ in range(3):
            c, p, b, n = O.ct_rk_step(g, par, scheme, 0.25 * blk.dx[0], c, p, b)
            nf += n
        assert nf == 0
        assert np.abs(b - bf).max() > 1e-6 * np.abs(bf).max()     # the field did evolve
        assert max_div(g, b) <= 1e-13 * scale, scheme


def test_ct_uniform_state_and_no_field_limit():
    blk = block(8)
    g = O.Grid(blk.n, 3, blk.dx)
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_PERIODIC)
    # uniform state with a uniform field: nothing changes
    state = np.array([1.0, 0.2, -0.1, 0.3, 0.7, 0.05, -0.02, 0.03])
    prim = np.broadcast_to(state[:, None, None, None], (8,) + g.shape).copy()
    bf = np.broadcast_to(state[5:, None, None, None], (3,) + g.shape).copy()
    cons = O.prim2con(g, par.gamma, prim)
    c, p, b, nf = O.ct_rk_step(g, par, O.RK3, 0.02, cons, prim, bf)
    assert nf == 0
    assert np.abs(b - bf)[:, 3:-3, 3:-3, 3:-3].max() <= 1e-15
    assert np.abs(c - cons)[:, 3:-3, 3:-3, 3:-3].max() <= 1e-14
    # no field: the CT step is the plain step
    prim = I.smooth_prims(blk, 4)
    prim[5:] = 0.0
    prim = O.fill_ghosts(g, O.BC_PERIODIC, prim)
    cons = O.prim2con(g, par.gamma, prim)
    c1, p1, b1, _ = O.ct_rk_step(g, par, O.RK3, 0.02, cons, prim, np.zeros((3,) + g.shape))
    c2, p2, _ = O.rk_step(g, par, O.RK3, 0.02, cons, prim)
    assert np.all(b1 == 0.0)
    assert np.array_equal(c1[:, 3:-3, 3:-3, 3:-3], c2[:, 3:-3, 3:-3, 3:-3])


def test_ct_conserves_the_flux_through_every_plane():
    blk = block((10, 8, 12))
    g, prim, bf = ct_setup(blk, seed=5)
    par = O.make_params(recon=O.REC_MINMOD, bc=O.BC_PERIODIC)
    cons = O.prim2con(g, par.gamma, prim)
    c, p, b, nf = O.ct_rk_step(g, par, O.RK3, 0.25 * min(blk.dx), cons, prim, bf)
    assert nf == 0
    for a in range(3):
        # flux of B^a through each a-plane (sum over the transverse interior faces)
        ax = 2 - a
        inner = [slice(3, -3)] * 3
        inner[ax] = slice(3, 3 + blk.n[a] + 1)
        f0 = bf[a][tuple(inner)].sum(axis=tuple(e for e in range(3) if e != ax))
        f1 = b[a][tuple(inner)].sum(axis=tuple(e for e in range(3) if e != ax))
        assert np.abs(f1 - f0).max() <= 1e-13 * np.abs(bf[a]).max() * blk.n[(a + 1) % 3] * blk.n[(a + 2) % 3]


def test_weak_field_advection_converges():
    """Uniform flow v, uniform rho and P, a weak field: the induction equation advects the field,
    so the face field should approach the discrete curl of the advected potential."""
    v = np.array([0.3, 0.2, 0.1])
    errs = []
    for n in (12, 24):
        blk = block(n)
        g = O.Grid(blk.n, 3, blk.dx)
        prim = np.zeros((8,) + g.shape)
        prim[0] = 1.0
        prim[4] = 1.0
        prim[1:4] = v[:, None, None, None]
        A = I.edge_potential(blk, 9, nmodes=2)
        scale = 1e-4 / np.abs(I.face_curl(blk, A)).max()
        bf = scale * I.face_curl(blk, A)
        prim = O.ct_cell_field(prim, bf)
        prim = O.fill_ghosts(g, O.BC_PERIODIC, prim)
        par = O.make_params(recon=O.REC_WENO5, bc=O.BC_PERIODIC)
        cons = O.prim2con(g, par.gamma, prim)
        dt = 0.25 / n
        nsteps = n // 4
        c, p, b = cons, prim, bf
        for _ in range(nsteps):
            c, p, b, nf = O.ct_rk_step(g, par, O.RK3, dt, c, p, b)
            assert nf == 0
        W = 1.0 / np.sqrt(1.0 - v @ v)
        ref = scale * I.face_curl(blk, I.edge_potential(blk, 9, shift=tuple(v * nsteps * dt), nmodes=2))
        inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
        errs.append(np.abs(b[inner] - ref[inner]).mean() / np.abs(ref[inner]).mean())
        del W
    assert errs[1] < errs[0] / 3.0, errs
