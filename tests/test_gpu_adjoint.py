"""The hand-written adjoint: transposition (dot-product) tests of every
reverse kernel against central differences of its forward kernel, the full
checkpointed gradient against the oracle's forward-mode dual numbers, and the
64^3 / 20-step SSP-RK3 gradient against central finite differences."""
import math

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


@pytest.fixture(scope="module")
def A(G):
    from paper_2210_17509_gb300 import adjoint
    return adjoint


def dot(a, b):
    return float((a * b).sum().item())


def state(G, n, curved, seed=3, recon=1):
    if curved:
        blk = I.Block((n, n, n), 3, (8.0 / n,) * 3, (4.0, 4.0, 4.0))
        met = I.schwarzschild_metric(blk)
        prim = I.smooth_prims(blk, seed, rho_range=(0.1, 1.0), metric=met)
        bc = G.BC_COPY
    else:
        blk = I.Block((n, n, n), 3, (1.0 / n,) * 3, (0.0, 0.0, 0.0))
        met = None
        prim = I.smooth_prims(blk, seed)
        bc = G.BC_PERIODIC
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=recon, bc=bc)
    tp = torch.from_numpy(prim).cuda()
    G.fill_ghosts(g, bc, tp)
    tm = None if met is None else torch.from_numpy(met).cuda()
    return g, p, tp, tm, blk, met


def interior_mask(g):
    m = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    m[3:-3, 3:-3, 3:-3] = 1.0
    return m


def test_ghost_fill_adjoint_is_the_transpose(G):
    gen = torch.Generator(device="cuda").manual_seed(0)
    for bc in (0, 1):
        for n in ((6, 5, 4), (1, 3, 2), (12, 9, 8)):
            g = G.Grid(n, 3, (0.1, 0.1, 0.1))
            v = torch.randn((8,) + g.shape, dtype=torch.float64, device="cuda", generator=gen)
            w = torch.randn((8,) + g.shape, dtype=torch.float64, device="cuda", generator=gen)
            gv = v.clone()
            G.fill_ghosts(g, bc, gv)
            gtw = w.clone()
            G.fill_ghosts_adjoint(g, bc, gtw)
            torch.cuda.synchronize()
            lhs, rhs = dot(gv, w), dot(v, gtw)
            assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
            assert float(gtw[:, :3].abs().max()) == 0.0


def smooth_direction(G, blk, like, seed):
    """A smooth random direction with each component scaled to its field's size
    (central differences along rough directions cross the kinks of min/max
    and WENO weights far more often)."""
    d = I.smooth_prims(blk, seed)
    d = d - d.mean(axis=(1, 2, 3), keepdims=True)
    d = d / np.abs(d).max(axis=(1, 2, 3), keepdims=True)
    t = torch.from_numpy(d).cuda()
    if like.shape != t.shape:
        t = t[:, 3:-3, 3:-3, 3:-3].contiguous()
    return t * like.abs().amax(dim=(1, 2, 3), keepdim=True)


@pytest.mark.parametrize("curved,recon,tol", [(False, 1, 1e-6), (True, 1, 1e-6), (False, 0, 1e-4)])
def test_rhs_adjoint_dot_product(G, curved, recon, tol):
    """<w, J v> (central differences of grmhd_rhs) == <J^T w, v> (grmhd_rhs_adjoint).
    Minmod is piecewise linear with kinks, so its check is looser."""
    g, p, prim, met, blk, _ = state(G, 10, curved, recon=recon)
    gen = torch.Generator(device="cuda").manual_seed(1)
    v = smooth_direction(G, blk, prim, 11)
    w = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * interior_mask(g)
    h = 1e-7
    fd = dot(w, (G.rhs(g, p, prim + h * v, met) - G.rhs(g, p, prim - h * v, met)) / (2 * h))
    pbar = torch.zeros_like(prim)
    gbar = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.rhs_adjoint(g, p, prim, w, pbar, gbar, met)
    ad = dot(pbar, v)
    assert abs(fd - ad) <= tol * abs(ad), (fd, ad)
    import dataclasses
    hg = 1e-7
    rp = G.rhs(g, dataclasses.replace(p, gamma=p.gamma + hg), prim, met)
    rm = G.rhs(g, dataclasses.replace(p, gamma=p.gamma - hg), prim, met)
    fdg = dot(w, (rp - rm) / (2 * hg))
    assert abs(fdg - float(gbar.item())) <= tol * abs(fdg), (fdg, float(gbar.item()))


@pytest.mark.parametrize("curved", [False, True])
def test_recovery_adjoints_dot_product(G, curved):
    import dataclasses
    g, p, prim, met, blk, _ = state(G, 8, curved)
    cons = G.prim2con(g, p, prim, met)
    gen = torch.Generator(device="cuda").manual_seed(2)
    mask = interior_mask(g)
    # prim2con: dU = J dP
    v = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * prim.abs().amax(
        dim=(1, 2, 3), keepdim=True) * mask
    w = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * mask
    h = 1e-6
    fd = dot(w, (G.prim2con(g, p, prim + h * v, met) - G.prim2con(g, p, prim - h * v, met)) / (2 * h))
    pbar = torch.zeros_like(prim)
    gbar = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.prim2con_adjoint(g, p, prim, w, pbar, gbar, met)
    assert abs(fd - dot(pbar, v)) <= 1e-8 * abs(fd)
    fdg = dot(w, (G.prim2con(g, dataclasses.replace(p, gamma=p.gamma + h), prim, met)
                  - G.prim2con(g, dataclasses.replace(p, gamma=p.gamma - h), prim, met)) / (2 * h))
    assert abs(fdg - float(gbar.item())) <= 1e-8 * abs(fdg)
    # con2prim: dP = J^{-1} dU
    vu = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * cons.abs().amax(
        dim=(1, 2, 3), keepdim=True) * mask * 1e-2

    def c2p(u, pp):
        out = prim.clone()
        G.con2prim(g, pp, u, out, met)
        return out
    fd = dot(w, (c2p(cons + h * vu, p) - c2p(cons - h * vu, p)) / (2 * h))
    ubar = torch.zeros_like(prim)
    gbar.zero_()
    G.con2prim_adjoint(g, p, prim, w, ubar, gbar, met)
    assert abs(fd - dot(ubar, vu)) <= 1e-7 * abs(fd), (fd, dot(ubar, vu))
    fdg = dot(w, (c2p(cons, dataclasses.replace(p, gamma=p.gamma + h))
                  - c2p(cons, dataclasses.replace(p, gamma=p.gamma - h))) / (2 * h))
    assert abs(fdg - float(gbar.item())) <= 1e-7 * abs(fdg), (fdg, float(gbar.item()))


@pytest.mark.parametrize("scheme", [2, 3])
def test_rk_step_adjoint_dot_product(G, scheme):
    g, p, prim, met, blk, _ = state(G, 10, False)
    cons = G.prim2con(g, p, prim, met)
    gen = torch.Generator(device="cuda").manual_seed(4)
    mask = interior_mask(g)
    # smooth perturbation directions (rough ones cross the HLLE min/max kinks)
    vu = smooth_direction(G, blk, cons, 21) * mask * 1e-2
    vp = smooth_direction(G, blk, prim, 22) * 1e-2
    wu = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * mask
    wp = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen)
    dt = 0.3 * blk.dx[0]
    h = 1e-6

    def step(u, pp):
        u, pp = u.clone(), pp.clone()
        G.rk_step(g, p, scheme, dt, u, pp, met)
        return u, pp
    up, pp_ = step(cons + h * vu, prim + h * vp)
    um, pm = step(cons - h * vu, prim - h * vp)
    fd = dot(wu, (up - um) / (2 * h)) + dot(wp, (pp_ - pm) / (2 * h))
    ubar, pbar = wu.clone(), wp.clone()
    gbar = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.rk_step_adjoint(g, p, scheme, dt, cons, prim, ubar, pbar, gbar, met)
    ad = dot(ubar, vu) + dot(pbar, vp)
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("curved", [False, True])
def test_gradient_matches_oracle_dual_numbers(G, A, curved):
    """Checkpointed adjoint gradient of L = sum rho^2 dV after 3 SSP-RK3 steps
    against the oracle's forward-mode derivative along random directions."""
    n = 10
    g, p, prim, met, blk, met_h = state(G, n, curved, seed=5)
    prim0 = prim[:, 3:-3, 3:-3, 3:-3].clone().requires_grad_(True)
    gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=True)
    dt = 0.25 * blk.dx[0]
    out = A.evolve(prim0, gam, g, p, G.RK3, dt, 3, checkpoint_every=2, metric=met)
    L = A.density_l2(out, g, met)
    L.backward()
    og = O.Grid(blk.n, 3, blk.dx)
    op = O.make_params(recon=O.REC_WENO5, bc=p.bc, rho_atm=p.rho_atm, p_atm=p.p_atm)
    prim_h = prim.cpu().numpy()
    rng = np.random.default_rng(6)
    for _ in range(3):
        d = rng.normal(size=prim_h.shape) * np.abs(prim_h).max(axis=(1, 2, 3), keepdims=True) * 1e-2
        dg = float(rng.normal())
        Lo, dLo, nf = O.loss_jvp(og, op, O.RK3, dt, 3, prim_h, d, dg, met_h)
        assert nf == 0
        assert abs(float(L.item()) - Lo) <= 1e-12 * abs(Lo)
        ad = float((prim0.grad.cpu().numpy() * d[:, 3:-3, 3:-3, 3:-3]).sum()) + float(gam.grad.item()) * dg
        assert abs(ad - dLo) <= 1e-10 * abs(dLo), (ad, dLo)


def test_config3_gradient_matches_central_differences(G, A):
    """64^3 periodic flat block, WENO5, 20 SSP-RK3 steps, checkpoint every 5:
    the adjoint gradient (initial primitives and Gamma) against central
    differences along random directions, to 1e-6 relative."""
    blk, prim_h, _ = I.smooth_flat(64, seed=3)
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=G.WENO5, bc=G.BC_PERIODIC)
    dt = 0.25 * blk.dx[0]
    prim0 = torch.from_numpy(prim_h[:, 3:-3, 3:-3, 3:-3].copy()).cuda()
    x = prim0.clone().requires_grad_(True)
    gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=True)
    L = A.density_l2(A.evolve(x, gam, g, p, G.RK3, dt, 20, checkpoint_every=5), g)
    L.backward()

    def loss(p0, gm):
        with torch.no_grad():
            return float(A.density_l2(A.evolve(p0, torch.tensor(gm, dtype=torch.float64), g, p, G.RK3, dt, 20), g))
    gen = torch.Generator(device="cuda").manual_seed(7)
    h = 1e-6
    for k in range(4):
        d = smooth_direction(G, blk, prim0, 100 + k)
        dg = float(torch.randn(1, generator=gen, device="cuda").item())
        fd = (loss(prim0 + h * d, p.gamma + h * dg) - loss(prim0 - h * d, p.gamma - h * dg)) / (2 * h)
        ad = dot(x.grad, d) + float(gam.grad.item()) * dg
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("nsteps,every", [(7, 3), (6, 3), (1, 5)])
def test_kept_last_segment_gives_the_recomputed_gradient(G, A, nsteps, every):
    """The forward pass that records its last segment (keep_last_segment, the
    default) gives the gradient of the one that recomputes it, to round-off
    (the reverse's atomic scatter varies in the last bits from run to run),
    and the same end state to the bit."""
    g, p, prim, met, blk, _ = state(G, 10, True, seed=8)
    dt = 0.25 * blk.dx[0]
    res = []
    for keep in (True, False):
        x = prim[:, 3:-3, 3:-3, 3:-3].clone().requires_grad_(True)
        gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=True)
        out = A.evolve(x, gam, g, p, G.RK3, dt, nsteps, checkpoint_every=every, metric=met, keep_last_segment=keep)
        A.density_l2(out, g, met).backward()
        res.append((out.detach().cpu().numpy(), x.grad.cpu().numpy(), float(gam.grad.item())))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    scale = np.abs(res[1][1]).max()
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-13 * scale
    assert abs(res[0][2] - res[1][2]) <= 1e-13 * abs(res[1][2])


def test_rk_step_adjoint_with_recorded_stages_is_identical(G):
    g, p, prim, met, blk, _ = state(G, 8, True)
    cons = G.prim2con(g, p, prim, met)
    dt = 0.25 * blk.dx[0]
    gen = torch.Generator(device="cuda").manual_seed(9)
    ub0 = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen) * interior_mask(g)
    pb0 = torch.randn(prim.shape, dtype=torch.float64, device="cuda", generator=gen)
    stages = torch.empty((3, 8) + g.shape, dtype=torch.float64, device="cuda")
    c1, p1 = cons.clone(), prim.clone()
    G.rk_step_record(g, p, G.RK3, dt, c1, p1, stages, met)
    c2, p2 = cons.clone(), prim.clone()
    G.rk_step(g, p, G.RK3, dt, c2, p2, met)
    torch.cuda.synchronize()
    assert torch.equal(c1, c2) and torch.equal(p1, p2) and torch.equal(stages[2], p1)
    outs = []
    for sp in (None, stages):
        ub, pb = ub0.clone(), pb0.clone()
        gb = torch.zeros(1, dtype=torch.float64, device="cuda")
        G.rk_step_adjoint(g, p, G.RK3, dt, cons, prim, ub, pb, gb, met, stage_prims=sp)
        torch.cuda.synchronize()
        outs.append((ub, pb, gb))
    # atomics make the summation order vary: compare to round-off
    for a, b in zip(outs[0], outs[1]):
        assert float((a - b).abs().max()) <= 1e-12 * float(a.abs().max())
