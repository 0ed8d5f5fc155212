"""Two-level AMR transfer on the CUDA path (through the C ABI) against the
oracle (Sec. 3; readings R14-R17 of the oracle header).

* restriction and prolongation: bit-exact (the same additions in the same
  order; the prolongation offsets are powers of two, so fused and unfused
  multiply-adds agree);
* flux restriction: 1e-12 of the largest RHS change, flat and Schwarzschild,
  minmod and WENO5;
* composite steps (one and two fine grids, SSP-RK3 and RK4, flat periodic and
  Schwarzschild with copy boundaries): 1e-12 normwise per field on every
  block; the composite totals are conserved to round-off on a periodic
  coarse block.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, normwise

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


def levels(nc, fine_specs, curved=False, ng=3):
    """Coarse block (flat on [0,1]^3, or Schwarzschild on [4,12]^3) and fine blocks
    (n, lo); returns blocks, metrics and primitives (fine from the coarse by
    prolongation, plus a smooth perturbation so that the levels differ)."""
    if curved:
        h = 8.0 / nc
        cb = I.Block((nc,) * 3, ng, (h,) * 3, (4.0,) * 3)
        cm = I.schwarzschild_metric(cb)
        pc = I.smooth_prims(cb, 21, rho_range=(0.1, 1.0), metric=cm)
    else:
        h = 1.0 / nc
        cb = I.Block((nc,) * 3, ng, (h,) * 3, (0.0,) * 3)
        cm = None
        pc = I.smooth_prims(cb, 21)
    Cg = O.Grid(cb.n, ng, cb.dx)
    fbs, fms, pfs = [], [], []
    for n, lo in fine_specs:
        fb = I.Block(tuple(n), ng, tuple(d / 2 for d in cb.dx),
                     tuple(cb.origin[d] + lo[d] * cb.dx[d] for d in range(3)))
        fm = I.schwarzschild_metric(fb) if curved else None
        Fg = O.Grid(fb.n, ng, fb.dx)
        pf = O.prolongate(Cg, pc, Fg, np.zeros((8,) + Fg.shape), lo, ghosts_only=False)
        x, y, z = fb.centres()
        pf[0] *= 1.0 + 0.03 * np.sin(2 * np.pi * x / fb.dx[0] / 16) * np.cos(2 * np.pi * y / fb.dx[1] / 12)
        pf[4] *= 1.0 + 0.03 * np.cos(2 * np.pi * z / fb.dx[2] / 10)
        pf = O.prolongate(Cg, pc, Fg, pf, lo, ghosts_only=True)
        fbs.append(fb)
        fms.append(fm)
        pfs.append(pf)
    return cb, cm, pc, fbs, fms, pfs


def test_restrict_and_prolongate_bit_exact(G):
    rng = np.random.default_rng(3)
    C = G.Grid((12, 10, 14), 3, (0.1, 0.1, 0.1))
    F = G.Grid((8, 6, 10), 3, (0.05, 0.05, 0.05))
    OC, OF = O.Grid(C.n, 3, C.dx), O.Grid(F.n, 3, F.dx)
    lo = (2, 3, 1)
    uf = rng.normal(size=(8,) + F.shape)
    uc = rng.normal(size=(8,) + C.shape)
    got = host(G.restrict(C, cuda(uc), F, cuda(uf), lo))
    assert np.array_equal(got, O.restrict(OC, uc, OF, uf, lo))
    for ghosts_only in (True, False):
        base = rng.normal(size=(5,) + F.shape)
        got = host(G.prolongate(C, cuda(uc[:5]), F, cuda(base), lo, ghosts_only))
        assert np.array_equal(got, O.prolongate(OC, uc[:5], OF, base, lo, ghosts_only))


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("recon", [0, 1])
def test_reflux_matches_oracle(G, curved, recon):
    cb, cm, pc, fbs, fms, pfs = levels(16, [((8, 10, 6), (4, 3, 5))], curved=curved)
    fb, fm, pf = fbs[0], fms[0], pfs[0]
    lo = (4, 3, 5)
    C, F = G.Grid(cb.n, 3, cb.dx), G.Grid(fb.n, 3, fb.dx)
    gp = G.Params(recon=recon, bc=G.BC_COPY)
    op = O.make_params(recon=recon, bc=O.BC_COPY, rho_atm=gp.rho_atm, p_atm=gp.p_atm, weno_eps=gp.weno_eps)
    out = torch.zeros((8,) + C.shape, dtype=torch.float64, device="cuda")
    got = host(G.reflux(C, gp, cuda(pc), F, cuda(pf), lo, out, scale=0.5,
                        coarse_metric=None if cm is None else cuda(cm), fine_metric=None if fm is None else cuda(fm)))
    ref = O.reflux(O.Grid(cb.n, 3, cb.dx), op, pc, O.Grid(fb.n, 3, fb.dx), pf, lo, scale=0.5,
                   coarse_metric=cm, fine_metric=fm)
    assert np.array_equal(got != 0.0, ref != 0.0)
    err = np.abs(got - ref).max(axis=(1, 2, 3)) / np.maximum(np.abs(ref).max(axis=(1, 2, 3)), 1e-300)
    assert err.max() <= FP64_TOL, err


def run_both(G, cb, cm, pc, fbs, fms, pfs, los, scheme, nsteps, bc, recon=1, cfl=0.25):
    C = G.Grid(cb.n, 3, cb.dx)
    Fs = [G.Grid(fb.n, 3, fb.dx) for fb in fbs]
    gp = G.Params(recon=recon, bc=bc)
    op = O.make_params(recon=recon, bc=bc, rho_atm=gp.rho_atm, p_atm=gp.p_atm, weno_eps=gp.weno_eps)
    OC = O.Grid(cb.n, 3, cb.dx)
    OFs = [O.Grid(fb.n, 3, fb.dx) for fb in fbs]
    dt = cfl * fbs[0].dx[0]
    # consistent start: U from the primitives, covered coarse cells restricted
    uc = O.prim2con(OC, gp.gamma, pc, cm)
    ufs = [O.prim2con(OFs[i], gp.gamma, pfs[i], fms[i]) for i in range(len(fbs))]
    for i in range(len(fbs)):
        uc = O.restrict(OC, uc, OFs[i], ufs[i], los[i])
    pc0, _, _ = O.con2prim(OC, op, uc, cm, pc)
    pc0 = O.fill_ghosts(OC, bc, pc0)
    pfs0 = [O.prolongate(OC, pc0, OFs[i], pfs[i], los[i], ghosts_only=True) for i in range(len(fbs))]
    # GPU
    d_uc, d_pc = cuda(uc), cuda(pc0)
    d_uf = [cuda(u) for u in ufs]
    d_pf = [cuda(p) for p in pfs0]
    d_cm = None if cm is None else cuda(cm)
    d_fm = None if cm is None else [cuda(m) for m in fms]
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = G.amr2_workspace(C, Fs, scheme)
    for _ in range(nsteps):
        G.amr2_step(C, gp, scheme, dt, d_uc, d_pc, Fs, d_uf, d_pf, los, coarse_metric=d_cm, fine_metrics=d_fm,
                    ws=ws, nfail=nfail)
    # oracle
    o_uc, o_pc, o_uf, o_pf = uc, pc0, ufs, pfs0
    onf = 0
    for _ in range(nsteps):
        o_uc, o_pc, o_uf, o_pf, nf = O.amr2_step(OC, op, scheme, dt, o_uc, o_pc, OFs, o_uf, o_pf, los,
                                                 coarse_metric=cm, fine_metrics=fms if cm is not None else None)
        onf += nf
    return (host(d_uc), host(d_pc), [host(t) for t in d_uf], [host(t) for t in d_pf], int(nfail.item()),
            (o_uc, o_pc, o_uf, o_pf, onf), (OC, OFs))


def interior(a, ng=3):
    return a[:, ng:-ng, ng:-ng, ng:-ng]


@pytest.mark.parametrize("case", ["flat-rk3-one", "flat-rk4-two", "curved-rk3-one"])
def test_composite_step_matches_oracle(G, case):
    if case == "flat-rk3-one":
        specs, scheme, curved, bc = [((8, 8, 8), (4, 5, 6))], G.RK3, False, G.BC_PERIODIC
    elif case == "flat-rk4-two":
        specs, scheme, curved, bc = [((8, 6, 8), (2, 2, 3)), ((6, 8, 10), (9, 8, 8))], G.RK4, False, G.BC_PERIODIC
    else:
        specs, scheme, curved, bc = [((10, 8, 8), (5, 4, 4))], G.RK3, True, G.BC_COPY
    cb, cm, pc, fbs, fms, pfs = levels(16, specs, curved=curved)
    los = [lo for _, lo in specs]
    uc, pcg, ufs, pfg, nf, (o_uc, o_pc, o_uf, o_pf, onf), _ = run_both(G, cb, cm, pc, fbs, fms, pfs, los, scheme,
                                                                       3, bc)
    assert nf == 0 and onf == 0
    assert normwise(interior(uc), interior(o_uc)).max() <= FP64_TOL
    assert normwise(interior(pcg), interior(o_pc), floor=1e-3).max() <= FP64_TOL
    for i in range(len(fbs)):
        assert normwise(interior(ufs[i]), interior(o_uf[i])).max() <= FP64_TOL, i
        # fine primitives including the prolongated ghosts
        assert normwise(pfg[i], o_pf[i], floor=1e-3).max() <= FP64_TOL, i


def test_composite_totals_conserved_on_gpu(G):
    specs = [((8, 8, 8), (4, 5, 6))]
    cb, cm, pc, fbs, fms, pfs = levels(16, specs)
    los = [specs[0][1]]
    uc, pcg, ufs, pfg, nf, (o_uc, _, o_uf, _, _), (OC, OFs) = run_both(G, cb, cm, pc, fbs, fms, pfs, los, G.RK3, 5,
                                                                        G.BC_PERIODIC)
    lo = los[0]
    covered = np.zeros(OC.shape, dtype=bool)
    covered[3 + lo[2]:7 + lo[2], 3 + lo[1]:7 + lo[1], 3 + lo[0]:7 + lo[0]] = True
    inner = np.zeros(OC.shape, dtype=bool)
    inner[3:-3, 3:-3, 3:-3] = True
    unc = inner & ~covered
    dvc, dvf = np.prod(cb.dx), np.prod(fbs[0].dx)
    # initial totals from the oracle's starting state (run_both restricts before stepping)
    gp = G.Params()
    u0c = O.prim2con(OC, gp.gamma, pc)
    u0f = O.prim2con(OFs[0], gp.gamma, pfs[0])
    t0 = u0c[:, unc].sum(axis=1) * dvc + interior(u0f).sum(axis=(1, 2, 3)) * dvf
    t1 = uc[:, unc].sum(axis=1) * dvc + interior(ufs[0]).sum(axis=(1, 2, 3)) * dvf
    scale = np.abs(u0c[:, inner]).sum(axis=1) * dvc
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale
