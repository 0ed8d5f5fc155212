"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Seeded synthetic inputs from paper_2210_17509_gb300.inputs feed both sides.
Tolerances: FP64 path 1e-12 relative (normwise per field), mixed path 1e-5
relative on conserved fields; index/byte work (ghost fill) bit-exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, MIXED_TOL, interior, normwise, vector_normwise

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


def grids(G, blk):
    return G.Grid(blk.n, blk.ng, blk.dx), O.Grid(blk.n, blk.ng, blk.dx)


def params(G, recon, bc=0, precision=0, gamma=I.GAMMA):
    gp = G.Params(gamma=gamma, recon=recon, bc=bc, precision=precision)
    op = O.make_params(gamma=gamma, recon=recon, bc=bc, rho_atm=gp.rho_atm, p_atm=gp.p_atm,
                       weno_eps=gp.weno_eps)
    return gp, op


def block_flat(n, seed=0, ng=3):
    if isinstance(n, int):
        n = (n, n, n)
    blk = I.Block(tuple(n), ng, tuple(1.0 / v for v in n), (0.0, 0.0, 0.0))
    return blk, I.smooth_prims(blk, seed), None


def block_curved(n, seed=1, ng=3, rho_range=(1e-3, 1.0)):
    if isinstance(n, int):
        n = (n, n, n)
    h = 8.0 / max(n)
    blk = I.Block(tuple(n), ng, (h, h, h), (4.0, 4.0, 4.0))
    met = I.schwarzschild_metric(blk)
    return blk, I.smooth_prims(blk, seed, rho_range=rho_range, metric=met), met


# ------------------------------------------------------------- ghost fill --
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [(8, 8, 8), (13, 7, 5), (1, 4, 2)])
def test_fill_ghosts_bit_exact(G, bc, n):
    blk, prim, _ = block_flat(n)
    g, og = grids(G, blk)
    rng = np.random.default_rng(0)
    arr = rng.normal(size=prim.shape)
    t = cuda(arr)
    G.fill_ghosts(g, bc, t)
    np.testing.assert_array_equal(host(t), O.fill_ghosts(og, bc, arr))


# --------------------------------------------------------- prim <-> cons --
@pytest.mark.parametrize("curved", [False, True])
def test_prim2con_parity(G, curved):
    blk, prim, met = (block_curved if curved else block_flat)(12)
    g, og = grids(G, blk)
    gp, op = params(G, 1)
    U = host(G.prim2con(g, gp, cuda(prim), None if met is None else cuda(met)))
    Uo = O.prim2con(og, op.gamma, prim, met)
    assert np.all(normwise(U, Uo) < 1e-13)


@pytest.mark.parametrize("curved", [False, True])
def test_con2prim_parity_and_round_trip(G, curved):
    blk, prim, met = (block_curved if curved else block_flat)(16, seed=4)
    g, og = grids(G, blk)
    gp, op = params(G, 1)
    Uo = O.prim2con(og, op.gamma, prim, met)
    rng = np.random.default_rng(1)
    guess = prim * (1.0 + 0.01 * rng.uniform(-1, 1, size=prim.shape))
    tp = cuda(guess)
    status = torch.zeros(g.shape, dtype=torch.int8, device="cuda")
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.con2prim(g, gp, cuda(Uo), tp, None if met is None else cuda(met), status, nfail)
    P = host(tp)
    Po, st, nf = O.con2prim(og, op, Uo, met, guess)
    assert nf == 0 and int(nfail.item()) == 0
    assert np.all(interior(host(status)[None], 3) == 0)
    assert np.all(normwise(interior(P, 3), interior(Po, 3)) < FP64_TOL)
    assert np.all(normwise(interior(P, 3), interior(prim, 3)) < FP64_TOL)
    # ghost entries untouched
    gmask = np.ones(g.shape, bool)
    gmask[3:-3, 3:-3, 3:-3] = False
    np.testing.assert_array_equal(P[:, gmask], guess[:, gmask])


@pytest.mark.parametrize("curved", [False, True])
def test_con2prim_newman_hamlin_first(G, curved):
    """GRMHD_NEWMAN_HAMLIN: the Newman-Hamlin iteration (Sec. 2.3) as the primary recovery, from
    a pressure guess 30% off, against the oracle's bracketed recovery."""
    blk, prim, met = (block_curved if curved else block_flat)(16, seed=6)
    g, og = grids(G, blk)
    gp, op = params(G, 1)
    gp.flags = G.NEWMAN_HAMLIN
    Uo = O.prim2con(og, op.gamma, prim, met)
    guess = prim.copy()
    guess[4] *= 1.3
    tp = cuda(guess)
    status = torch.zeros(g.shape, dtype=torch.int8, device="cuda")
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.con2prim(g, gp, cuda(Uo), tp, None if met is None else cuda(met), status, nfail)
    P = host(tp)
    Po, st, nf = O.con2prim(og, op, Uo, met, guess)
    assert nf == 0 and int(nfail.item()) == 0
    assert np.all(interior(host(status)[None], 3) == 0)
    assert np.all(normwise(interior(P, 3), interior(Po, 3)) < FP64_TOL)


def test_con2prim_failures_set_atmosphere(G):
    """Host-injected faults: tau + D < 0, NaN, and an impossible momentum."""
    blk, prim, _ = block_flat(8, seed=2)
    g, og = grids(G, blk)
    gp, op = params(G, 1)
    Uo = O.prim2con(og, op.gamma, prim)
    bad = [(3, 3, 3), (5, 6, 7), (9, 4, 5)]
    Uo[4, 3, 3, 3] = -10.0 * Uo[0, 3, 3, 3]
    Uo[:5, 7, 6, 5] = np.nan
    Uo[1, 5, 4, 9] = 50.0 * (Uo[4, 5, 4, 9] + Uo[0, 5, 4, 9])
    tp = cuda(prim)
    status = torch.zeros(g.shape, dtype=torch.int8, device="cuda")
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.con2prim(g, gp, cuda(Uo), tp, None, status, nfail)
    P, S = host(tp), host(status)
    assert int(nfail.item()) == 3
    for (i, j, k) in bad:
        assert S[k, j, i] == 2
        assert P[0, k, j, i] == gp.rho_atm and P[4, k, j, i] == gp.p_atm
        assert np.all(P[1:4, k, j, i] == 0.0)
    S[3, 3, 3] = S[7, 6, 5] = S[5, 4, 9] = 0
    assert np.all(S[3:-3, 3:-3, 3:-3] == 0)


# ------------------------------------------------------------------ RHS --
RHS_CASES = [
    ("flat-minmod-32", lambda: block_flat(32, seed=0), 0),           # config 0 at full size
    ("flat-weno5-ragged", lambda: block_flat((20, 12, 9), seed=3), 1),
    ("flat-weno5-tiny", lambda: block_flat((1, 2, 3), seed=5), 1),
    ("curved-weno5-20", lambda: block_curved(20, seed=1), 1),
    ("curved-minmod-ragged", lambda: block_curved((11, 17, 6), seed=6), 0),
]


@pytest.mark.parametrize("name,make,recon", RHS_CASES, ids=[c[0] for c in RHS_CASES])
def test_rhs_fp64_parity(G, name, make, recon):
    blk, prim, met = make()
    g, og = grids(G, blk)
    bc = 1 if met is not None else 0
    gp, op = params(G, recon, bc=bc)
    prim = O.fill_ghosts(og, bc, prim)
    r = host(G.rhs(g, gp, cuda(prim), None if met is None else cuda(met)))
    ro = O.rhs(og, op, prim, met)
    err = normwise(interior(r, 3), interior(ro, 3))
    assert np.all(err < FP64_TOL), err


def test_rhs_fp64_parity_with_shift_and_extrinsic_curvature(G):
    """Static lapse/shift with a given K_ij: the covariant oracle builds d_t gamma
    from K_ij, the kernel uses the 3+1 source form; both must agree."""
    blk, prim, met = block_curved(12, seed=8)
    g, og = grids(G, blk)
    x, y, z = blk.centres()
    met = met.copy()
    met[1] = 0.05 * np.sin(x)
    met[2] = -0.03 * np.cos(y)
    met[3] = 0.02 * np.sin(z + x)
    met[5] = 0.01 * np.cos(x + y)
    rng = np.random.default_rng(2)
    kij = 0.02 * rng.normal(size=(6,) + g.shape)
    gp, op = params(G, 1, bc=1)
    prim = O.fill_ghosts(og, 1, prim)
    r = host(G.rhs(g, gp, cuda(prim), cuda(met), cuda(kij)))
    ro = O.rhs(og, op, prim, met, kij)
    err = normwise(interior(r, 3), interior(ro, 3))
    assert np.all(err < FP64_TOL), err


def test_rhs_uniform_state_exactly_zero(G):
    blk, prim, _ = block_flat((9, 10, 11))
    for q, v in enumerate([1.3, 0.2, -0.4, 0.1, 0.7, 0.3, -0.2, 0.5]):
        prim[q] = v
    g, _ = grids(G, blk)
    for recon in (0, 1):
        for prec in (0, 1):
            gp, _ = params(G, recon, precision=prec)
            r = host(G.rhs(g, gp, cuda(prim)))
            assert np.all(interior(r, 3) == 0.0)


def test_rhs_periodic_telescoping(G):
    blk, prim, _ = block_flat(24, seed=11)
    g, og = grids(G, blk)
    gp, _ = params(G, 1)
    prim = O.fill_ghosts(og, 0, prim)
    r = interior(host(G.rhs(g, gp, cuda(prim))), 3)
    for q in range(8):
        assert abs(r[q].sum()) < 1e-13 * np.abs(r[q]).sum()


@pytest.mark.parametrize("path", ["rhs", "rhs_cached"])
def test_rhs_full_size_schwarzschild_sampled(G, path):
    """128^3 WENO5 on the Schwarzschild block, the benchmark's launch (the
    cached path is the two-pass RHS the benchmark times): sampled cells
    (random, faces, edges, corners) against the oracle one by one."""
    blk, prim, met = I.smooth_schwarzschild(128, seed=1)
    g, og = grids(G, blk)
    gp, op = params(G, 1, bc=1)
    tp = cuda(prim)
    G.fill_ghosts(g, 1, tp)
    prim = host(tp)
    if path == "rhs":
        r = host(G.rhs(g, gp, tp, cuda(met)))
    else:
        r = host(G.rhs_cached(g, gp, tp, cuda(met)))
    rng = np.random.default_rng(5)
    n = 128
    pick = [rng.integers(0, n, size=3) for _ in range(400)]
    for a in (0, n - 1):
        for b in (0, n - 1):
            for c in (0, n - 1):
                pick.append(np.array([a, b, c]))
    cells = np.array(pick) + 3
    ro = O.rhs_cells(og, op, prim, cells, met)
    rg = np.array([r[:, k, j, i] for (i, j, k) in cells])
    scale = np.max(np.abs(interior(r, 3)), axis=(1, 2, 3))
    err = np.max(np.abs(rg - ro), axis=0) / scale
    assert np.all(err < FP64_TOL), err


@pytest.mark.parametrize("curved", [False, True])
def test_rhs_mixed_close_to_fp64_oracle(G, curved):
    blk, prim, met = (block_curved if curved else block_flat)(20, seed=3)
    g, og = grids(G, blk)
    bc = 1 if curved else 0
    gp, op = params(G, 1, bc=bc, precision=1)
    prim = O.fill_ghosts(og, bc, prim)
    r = host(G.rhs(g, gp, cuda(prim), None if met is None else cuda(met)))
    ro = O.rhs(og, op, prim, met)
    err = normwise(interior(r, 3), interior(ro, 3))
    print("mixed RHS vs oracle, normwise", err, "vector-scaled", vector_normwise(interior(r, 3), interior(ro, 3)))
    assert np.all(err < MIXED_TOL), err


# ------------------------------------------------------------- RK steps --
def _evolve_both(G, blk, prim, met, recon, bc, scheme, nsteps, cfl, precision=0):
    g, og = grids(G, blk)
    gp, op = params(G, recon, bc=bc, precision=precision)
    prim = O.fill_ghosts(og, bc, prim)
    cons = O.prim2con(og, op.gamma, prim, met)
    dt = cfl * min(blk.dx)
    tc, tp = cuda(cons), cuda(prim)
    tm = None if met is None else cuda(met)
    ws = G.workspace(g, scheme)
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(nsteps):
        G.rk_step(g, gp, scheme, dt, tc, tp, tm, None, ws, nfail)
    co, po = cons, prim
    for _ in range(nsteps):
        co, po, nf = O.rk_step(og, op, scheme, dt, co, po, met)
        assert nf == 0
    assert int(nfail.item()) == 0
    return host(tc), host(tp), co, po


def test_rk2_config0_full_size(G):
    """Config shape 0: 32^3 periodic flat, minmod, one RK2 step."""
    blk, prim, met = I.smooth_flat(32, seed=0)
    c, p, co, po = _evolve_both(G, blk, prim, met, 0, 0, G.RK2, 1, 0.4)
    assert np.all(normwise(interior(c, 3), interior(co, 3)) < FP64_TOL)
    assert np.all(normwise(interior(p, 3), interior(po, 3)) < FP64_TOL)
    # ghost planes are exact periodic copies of the device's own interior
    np.testing.assert_array_equal(p[:, :3], p[:, 32:35])
    np.testing.assert_array_equal(p[:, :, :, 35:], p[:, :, :, 3:6])


@pytest.mark.parametrize("scheme", [3, 4])
def test_rk_curved_weno5(G, scheme):
    blk, prim, met = block_curved(16, seed=1, rho_range=(0.1, 1.0))
    c, p, co, po = _evolve_both(G, blk, prim, met, 1, 1, scheme, 2, 0.25)
    assert np.all(normwise(interior(c, 3), interior(co, 3)) < FP64_TOL)
    assert np.all(normwise(interior(p, 3), interior(po, 3)) < FP64_TOL)


def test_rk3_mixed_conserved_error(G):
    """Mixed path: every conserved field within 1e-5 (normwise) of the FP64 oracle."""
    blk, prim, met = block_curved(16, seed=1, rho_range=(0.1, 1.0))
    c, p, co, po = _evolve_both(G, blk, prim, met, 1, 1, 3, 3, 0.25, precision=1)
    err = normwise(interior(c, 3), interior(co, 3))
    assert np.all(err < MIXED_TOL), err


@pytest.mark.parametrize("seed,rho_range", [(1, (0.1, 1.0)), (4, (1e-3, 1.0))])
def test_mixed_recovery_is_an_fp64_solve(G, seed, rho_range):
    """Mixed path with dt = 1e-9 dx: the FP32 right-hand side changes U by
    round-off only, so the step's FP64 primitives are the recovery's root
    from the FP32 guess.  The FP32 predictor alone would leave about 1e-7;
    its FP64-residual refinement must reach the FP64 oracle's root."""
    blk, prim, met = block_curved(16, seed=seed, rho_range=rho_range)
    c, p, co, po = _evolve_both(G, blk, prim, met, 1, 1, 3, 1, 1e-9, precision=1)
    err = normwise(interior(p, 3), interior(po, 3))
    assert np.all(err < 1e-10), err


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_rk3_full_size_schwarzschild_step(G, precision, tol):
    '''The benchmark's workload and launch (128^3 Schwarzschild, WENO5, SSP-RK3,
    CFL 0.25): one full step compared element by element with the oracle.'''
    blk, prim, met = I.smooth_schwarzschild(128, seed=1)
    c, p, co, po = _evolve_both(G, blk, prim, met, 1, 1, 3, 1, 0.25, precision=precision)
    c, co = interior(c, 3), interior(co, 3)
    err = normwise(c, co)
    assert np.all(err < tol), err
    # rho spans [1e-3, 1]: D and tau also cell by cell, relative to each cell's
    # own value (floored at 1e-6 of the field's maximum)
    for q in (0, 4):
        s = np.maximum(np.abs(co[q]), 1e-6 * np.max(np.abs(co[q])))
        cell = np.max(np.abs(c[q] - co[q]) / s)
        assert cell < tol, (q, cell)


def test_rk3_periodic_conserves_totals(G):
    blk, prim, met = block_flat(24, seed=12)
    g, og = grids(G, blk)
    gp, op = params(G, 1)
    prim = O.fill_ghosts(og, 0, prim)
    cons = O.prim2con(og, op.gamma, prim)
    tc, tp = cuda(cons), cuda(prim)
    tot0 = interior(cons, 3).sum(axis=(1, 2, 3))
    for _ in range(3):
        G.rk_step(g, gp, G.RK3, 0.25 / 24, tc, tp)
    c = interior(host(tc), 3)
    scale = np.abs(c).sum(axis=(1, 2, 3))
    assert np.all(np.abs(c.sum(axis=(1, 2, 3)) - tot0) <= 1e-13 * scale)


def test_rk3_mixed_without_cache_workspace(G):
    """With only the minimum workspace the mixed path reads the FP64 inputs
    (no FP32 caches); it must meet the same 1e-5 bound."""
    blk, prim, met = block_curved(16, seed=1, rho_range=(0.1, 1.0))
    g, og = grids(G, blk)
    gp, op = params(G, 1, bc=1, precision=1)
    prim = O.fill_ghosts(og, 1, prim)
    cons = O.prim2con(og, op.gamma, prim, met)
    dt = 0.25 * blk.dx[0]
    tc, tp, tm = cuda(cons), cuda(prim), cuda(met)
    ws = G.workspace(g, G.RK3, cached=False)
    assert ws.numel() < G.rk_workspace_bytes_cached(g, G.RK3)
    for _ in range(3):
        G.rk_step(g, gp, G.RK3, dt, tc, tp, tm, None, ws)
    co, po = cons, prim
    for _ in range(3):
        co, po, _ = O.rk_step(og, op, O.RK3, dt, co, po, met)
    err = normwise(interior(host(tc), 3), interior(co, 3))
    assert np.all(err < MIXED_TOL), err


def test_mixed_geometry_reuse_flag(G):
    """Reusing the geometry cache of a static metric gives the same steps."""
    import dataclasses
    blk, prim, met = block_curved(12, seed=2, rho_range=(0.1, 1.0))
    g, og = grids(G, blk)
    gp, op = params(G, 1, bc=1, precision=1)
    prim = O.fill_ghosts(og, 1, prim)
    cons = O.prim2con(og, op.gamma, prim, met)
    dt = 0.25 * blk.dx[0]
    res = []
    for reuse in (False, True):
        tc, tp, tm = cuda(cons), cuda(prim), cuda(met)
        ws = G.workspace(g, G.RK3)
        p = gp
        for _ in range(3):
            G.rk_step(g, p, G.RK3, dt, tc, tp, tm, None, ws)
            if reuse:
                p = dataclasses.replace(gp, flags=G.REUSE_GEOMETRY)
        res.append(host(tc))
    np.testing.assert_array_equal(res[0], res[1])


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_independent_of_tile_shape(G, precision):
    """Every tile shape cuts the same face fluxes: bit-identical RHS."""
    import dataclasses
    blk, prim, met = block_curved((19, 13, 10), seed=6, rho_range=(0.1, 1.0))
    g, og = grids(G, blk)
    gp, _ = params(G, 1, bc=1, precision=precision)
    prim = O.fill_ghosts(og, 1, prim)
    tp, tm = cuda(prim), cuda(met)
    ref = host(G.rhs(g, gp, tp, tm))
    for shape in (1, 2, 3, 4):
        r = host(G.rhs(g, dataclasses.replace(gp, tile=shape), tp, tm))
        np.testing.assert_array_equal(interior(r, 3), interior(ref, 3))


@pytest.mark.parametrize("precision", [0, 1])
def test_cached_and_direct_paths_agree(G, precision):
    """The workspace size selects geometry caches (cached) or direct FP64 reads;
    both are the same method and agree with each other and the oracle."""
    blk, prim, met = block_curved(14, seed=3, rho_range=(0.1, 1.0))
    g, og = grids(G, blk)
    gp, op = params(G, 1, bc=1, precision=precision)
    prim = O.fill_ghosts(og, 1, prim)
    cons = O.prim2con(og, op.gamma, prim, met)
    dt = 0.25 * blk.dx[0]
    outs = []
    for cached in (True, False):
        tc, tp, tm = cuda(cons), cuda(prim), cuda(met)
        ws = G.workspace(g, G.RK3, cached=cached)
        for _ in range(2):
            G.rk_step(g, gp, G.RK3, dt, tc, tp, tm, None, ws)
        outs.append(host(tc))
    co, po = cons, prim
    for _ in range(2):
        co, po, _ = O.rk_step(og, op, O.RK3, dt, co, po, met)
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    for o in outs:
        assert np.all(normwise(interior(o, 3), interior(co, 3)) < tol)
    assert np.all(normwise(interior(outs[0], 3), interior(outs[1], 3)) < (1e-14 if precision == 0 else MIXED_TOL))


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_cached_matches_rhs(G, precision):
    import dataclasses
    blk, prim, met = block_curved((13, 11, 9), seed=4, rho_range=(0.1, 1.0))
    g, og = grids(G, blk)
    gp, op = params(G, 1, bc=1, precision=precision)
    prim = O.fill_ghosts(og, 1, prim)
    tp, tm = cuda(prim), cuda(met)
    ws = G.rhs_workspace(g)
    r1 = host(G.rhs_cached(g, gp, tp, tm, None, None, ws))
    r2 = host(G.rhs_cached(g, dataclasses.replace(gp, flags=G.REUSE_GEOMETRY), tp, tm, None, None, ws))
    np.testing.assert_array_equal(r1, r2)
    ro = O.rhs(og, op, prim, met)
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    err = normwise(interior(r1, 3), interior(ro, 3))
    print("cached RHS vs oracle, precision", precision, "normwise", err)
    assert np.all(err < tol), err
