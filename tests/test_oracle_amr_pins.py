"""Pins of the oracle's two-level AMR transfer (Sec. 3; readings R14-R17 in
the oracle header) against what the mathematics fixes:

* prolongation reproduces linear fields exactly, leaves children equal to the
  parent at an extremum (minmod), and its 8 children average to the parent,
  so restriction after prolongation returns the coarse field;
* restriction conserves the integral;
* with flux restriction, the composite RHS (uncovered coarse cells plus fine
  cells) telescopes to zero on a periodic coarse block; without it, it does
  not;
* a composite step keeps a uniform state uniform and conserves the composite
  totals to round-off.
"""
import numpy as np

import oracle as O
from paper_2210_17509_gb300 import inputs as I


def coords(g, origin):
    ax = [origin[d] + (np.arange(g.n[d] + 2 * g.ng) - g.ng + 0.5) * g.dx[d] for d in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


def two_level(nc=16, nf=8, lo=(4, 4, 4), ng=3):
    C = O.Grid((nc,) * 3, ng, (1.0 / nc,) * 3)
    F = O.Grid((nf,) * 3, ng, (0.5 / nc,) * 3)
    return C, F, lo


def test_prolongation_exact_for_linear_fields():
    C, F, lo = two_level(8, 8, (2, 2, 2))
    x, y, z = coords(C, (0, 0, 0))
    uc = np.stack([1 + 2 * x - 3 * y + 0.5 * z, x + y + z - 0.25])
    uf = O.prolongate(C, uc, F, np.zeros((2,) + F.shape), lo, ghosts_only=False)
    xf, yf, zf = coords(F, tuple(lo[d] * C.dx[d] for d in range(3)))
    ref = np.stack([1 + 2 * xf - 3 * yf + 0.5 * zf, xf + yf + zf - 0.25])
    assert np.abs(uf - ref).max() < 1e-14


def test_prolongation_flat_at_extremum_and_ghosts_only():
    C, F, lo = two_level(8, 8, (2, 2, 2))
    x, y, z = coords(C, (0, 0, 0))
    uc = (-((x - 0.3125) ** 2) - (y - 0.3125) ** 2 - (z - 0.3125) ** 2)[None]   # maximum at cell (2, 2, 2)
    uf = O.prolongate(C, uc, F, np.zeros((1,) + F.shape), lo, ghosts_only=False)
    par = uc[0, 5, 5, 5]
    assert np.all(uf[0, 3:5, 3:5, 3:5] == par)          # the 8 children of the extremum
    marker = np.full((1,) + F.shape, 7.0)
    g = O.prolongate(C, uc, F, marker, lo, ghosts_only=True)
    assert np.all(g[0, 3:-3, 3:-3, 3:-3] == 7.0)          # interior untouched
    assert np.all(g[0, :3] == uf[0, :3])                   # ghosts as in the full prolongation


def test_children_average_to_parent():
    C, F, lo = two_level(12, 8, (3, 2, 4))
    rng = np.random.default_rng(5)
    uc = rng.normal(size=(8,) + C.shape)
    uf = O.prolongate(C, uc, F, np.zeros((8,) + F.shape), lo, ghosts_only=False)
    back = O.restrict(C, np.zeros_like(uc), F, uf, lo)
    sl = (slice(None),) + tuple(slice(3 + lo[d], 3 + lo[d] + 4) for d in (2, 1, 0))
    assert np.abs(back[sl] - uc[sl]).max() < 1e-14


def test_restriction_conserves_the_integral():
    C, F, lo = two_level(16, 12, (5, 3, 2))
    rng = np.random.default_rng(6)
    uf = rng.uniform(0.5, 2.0, size=(8,) + F.shape)
    uc = O.restrict(C, np.zeros((8,) + C.shape), F, uf, lo)
    dvc, dvf = np.prod(C.dx), np.prod(F.dx)
    cov = uc[:, 3 + lo[2]:3 + lo[2] + 6, 3 + lo[1]:3 + lo[1] + 6, 3 + lo[0]:3 + lo[0] + 6]
    tot_c = cov.sum(axis=(1, 2, 3)) * dvc
    tot_f = uf[:, 3:-3, 3:-3, 3:-3].sum(axis=(1, 2, 3)) * dvf
    assert np.all(np.abs(tot_c - tot_f) <= 1e-13 * np.abs(tot_f))


def _composite_setup(recon=O.REC_WENO5):
    C, F, lo = two_level(16, 8, (4, 5, 6))
    blk = I.Block(C.n, C.ng, C.dx, (0.0, 0.0, 0.0))
    pc = I.smooth_prims(blk, 11)
    pf = O.prolongate(C, pc, F, np.zeros((8,) + F.shape), lo, ghosts_only=False)
    # fine data that differs from the coarse parents (smooth, periodic-free perturbation)
    xf, yf, zf = coords(F, tuple(lo[d] * C.dx[d] for d in range(3)))
    pf[0] *= 1.0 + 0.05 * np.sin(40 * xf) * np.cos(30 * yf)
    pf[4] *= 1.0 + 0.05 * np.cos(35 * zf)
    pf = O.prolongate(C, pc, F, pf, lo, ghosts_only=True)
    par = O.make_params(recon=recon, bc=O.BC_PERIODIC)
    return C, F, lo, pc, pf, par


def test_flux_restriction_makes_the_composite_rhs_telescope():
    C, F, lo, pc, pf, par = _composite_setup()
    Lc = O.rhs(C, par, pc)
    Lf = O.rhs(F, par, pf)
    dL = O.reflux(C, par, pc, F, pf, lo)
    covered = np.zeros(C.shape, dtype=bool)
    covered[3 + lo[2]:3 + lo[2] + 4, 3 + lo[1]:3 + lo[1] + 4, 3 + lo[0]:3 + lo[0] + 4] = True
    inner = np.zeros(C.shape, dtype=bool)
    inner[3:-3, 3:-3, 3:-3] = True
    unc = inner & ~covered
    dvc, dvf = np.prod(C.dx), np.prod(F.dx)
    fine_sum = Lf[:, 3:-3, 3:-3, 3:-3].sum(axis=(1, 2, 3)) * dvf
    scale = np.abs(Lc[:, unc]).sum(axis=1) * dvc + np.abs(Lf[:, 3:-3, 3:-3, 3:-3]).sum(axis=(1, 2, 3)) * dvf
    with_flux = (Lc + dL)[:, unc].sum(axis=1) * dvc + fine_sum
    without = Lc[:, unc].sum(axis=1) * dvc + fine_sum
    assert np.all(np.abs(with_flux) <= 1e-13 * scale), with_flux / scale
    # dL is non-zero only next to the fine grid, and without it the sum does not vanish
    assert np.all(dL[:, ~unc] == 0.0)
    assert np.abs(without[0]) > 1e-6 * scale[0]


def test_composite_step_keeps_a_uniform_state():
    C, F, lo = two_level(12, 8, (2, 3, 4))
    state = np.array([1.0, 0.2, -0.1, 0.05, 0.5, 0.1, 0.02, -0.03])
    pc = np.broadcast_to(state[:, None, None, None], (8,) + C.shape).copy()
    pf = np.broadcast_to(state[:, None, None, None], (8,) + F.shape).copy()
    par = O.make_params(recon=O.REC_WENO5, bc=O.BC_PERIODIC)
    uc = O.prim2con(C, par.gamma, pc)
    uf = O.prim2con(F, par.gamma, pf)
    uc2, pc2, (uf2,), (pf2,), nf = O.amr2_step(C, par, O.RK3, 0.25 * F.dx[0], uc, pc, [F], [uf], [pf], [lo])
    assert nf == 0
    assert np.abs(uc2[:, 3:-3, 3:-3, 3:-3] - uc[:, 3:-3, 3:-3, 3:-3]).max() <= 1e-14
    assert np.abs(uf2[:, 3:-3, 3:-3, 3:-3] - uf[:, 3:-3, 3:-3, 3:-3]).max() <= 1e-14


def test_composite_step_conserves_the_totals():
    C, F, lo, pc, pf, par = _composite_setup()
    uc = O.prim2con(C, par.gamma, pc)
    uf = O.prim2con(F, par.gamma, pf)
    uc = O.restrict(C, uc, F, uf, lo)
    covered = np.zeros(C.shape, dtype=bool)
    covered[3 + lo[2]:3 + lo[2] + 4, 3 + lo[1]:3 + lo[1] + 4, 3 + lo[0]:3 + lo[0] + 4] = True
    inner = np.zeros(C.shape, dtype=bool)
    inner[3:-3, 3:-3, 3:-3] = True
    unc = inner & ~covered
    dvc, dvf = np.prod(C.dx), np.prod(F.dx)

    def total(uc_, uf_):
        return uc_[:, unc].sum(axis=1) * dvc + uf_[:, 3:-3, 3:-3, 3:-3].sum(axis=(1, 2, 3)) * dvf

    t0 = total(uc, uf)
    for scheme in (O.RK2, O.RK3, O.RK4):
        uc2, pc2, (uf2,), (pf2,), nf = O.amr2_step(C, par, scheme, 0.25 * F.dx[0], uc, pc, [F], [uf], [pf], [lo])
        assert nf == 0
        t1 = total(uc2, uf2)
        # the integral over the covered region equals the fine integral (restriction)
        assert np.all(np.abs(uc2[:, covered].sum(axis=1) * dvc - uf2[:, 3:-3, 3:-3, 3:-3].sum(axis=(1, 2, 3)) * dvf)
                      <= 1e-13 * np.abs(t0).max())
        scale = np.abs(uc[:, inner]).sum(axis=1) * dvc
        assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (scheme, (t1 - t0) / scale)
