"""Constrained transport on the CUDA path (through the C ABI) against the
oracle (Sec. 3, staggered-grid field evolution; reading R19 of the oracle
header).

* face rate -curl E: 1e-12 of its largest magnitude per component, flat
  periodic and Schwarzschild with copy boundaries, minmod and WENO5, on
  blocks that span several tiles with ragged tails;
* steps (SSP-RK2, SSP-RK3, RK4; cached and uncached workspaces): 1e-12
  normwise per field for U, the primitives and the interior faces;
* discrete divergence: bit-exact against the oracle's (the same divisions
  and additions in the same order), and kept at round-off by many steps;
* mixed precision: within the mixed bound of the FP64 oracle, with the
  divergence still at round-off (the face update is FP64 whatever the
  flux precision);
* one-cell-thick blocks along each axis;
* no field: the CT step equals the plain step bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, MIXED_TOL, normwise

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


def ct_case(n, seed=1, curved=False, bmax=0.1, ng=3):
    """Smooth primitives with a divergence-free face field (the discrete curl
    of a random edge potential) whose cell means set the primitive field."""
    n = tuple(n)
    if curved:
        h = 8.0 / max(n)
        blk = I.Block(n, ng, (h, h, h), (4.0, 4.0, 4.0))
        metric = I.schwarzschild_metric(blk)
        prim = I.smooth_prims(blk, seed, rho_range=(0.1, 1.0), metric=metric)
        bc = O.BC_COPY
    else:
        blk = I.Block(n, ng, tuple(1.0 / v for v in n), (0.0, 0.0, 0.0))
        metric = None
        prim = I.smooth_prims(blk, seed)
        bc = O.BC_PERIODIC
    bf = I.face_curl(blk, I.edge_potential(blk, seed + 100))
    inner = (slice(None),) + tuple(slice(ng, s - ng) for s in blk.shape)
    bf *= bmax / np.abs(bf[inner]).max()
    prim = O.ct_cell_field(prim, bf, metric)
    og = O.Grid(blk.n, ng, blk.dx)
    prim = O.fill_ghosts(og, bc, prim)
    return blk, og, metric, prim, bf, bc


def faces(bf, n, ng):
    """The interior faces of each component, flattened."""
    out = []
    for a in range(3):
        sl = [slice(ng, ng + n[2]), slice(ng, ng + n[1]), slice(ng, ng + n[0])]
        sl[2 - a] = slice(ng, ng + n[a] + 1)
        out.append(bf[a][tuple(sl)].ravel())
    return out


def face_normwise(a, b, n, ng):
    fa, fb = faces(a, n, ng), faces(b, n, ng)
    return np.array([np.abs(x - y).max() / max(np.abs(y).max(), 1e-300) for x, y in zip(fa, fb)])


def interior(a, ng):
    return a[(slice(None),) + tuple(slice(ng, s - ng) for s in a.shape[1:])]


def gpu_params(G, recon, bc, precision=None):
    p = G.Params(recon=recon, bc=bc)
    if precision is not None:
        p.precision = precision
    return p


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("recon", ["minmod", "weno5"])
def test_ct_rate_parity(G, curved, recon):
    blk, og, metric, prim, bf, bc = ct_case((19, 13, 11), seed=3, curved=curved)
    orec = O.REC_WENO5 if recon == "weno5" else O.REC_MINMOD
    grec = G.WENO5 if recon == "weno5" else G.MINMOD
    ref = O.ct_rate(og, O.make_params(recon=orec, bc=bc), prim, metric)
    gg = G.Grid(blk.n, 3, blk.dx)
    out = host(G.ct_rate(gg, gpu_params(G, grec, bc), cuda(prim), None if metric is None else cuda(metric)))
    err = normwise(out, ref)
    assert np.all(err <= FP64_TOL), err
    # nothing outside the interior faces
    mask = np.zeros_like(ref, dtype=bool)
    for a in range(3):
        sl = [slice(3, 3 + blk.n[2]), slice(3, 3 + blk.n[1]), slice(3, 3 + blk.n[0])]
        sl[2 - a] = slice(3, 3 + blk.n[a] + 1)
        mask[a][tuple(sl)] = True
    assert np.all(out[~mask] == 0.0)


def run_ct_steps(G, blk, og, metric, prim, bf, bc, scheme, nsteps, recon=O.REC_WENO5, cached=True, dt_frac=0.25,
                 precision=None):
    op = O.make_params(recon=recon, bc=bc)
    cons = O.prim2con(og, op.gamma, prim, metric)
    dt = dt_frac * min(blk.dx)
    c, p, b = cons, prim, bf
    for _ in range(nsteps):
        c, p, b, nf = O.ct_rk_step(og, op, scheme, dt, c, p, b, metric)
        assert nf == 0
    gg = G.Grid(blk.n, 3, blk.dx)
    gp = gpu_params(G, G.WENO5 if recon == O.REC_WENO5 else G.MINMOD, bc, precision)
    gc, gpr, gb = cuda(cons), cuda(prim), cuda(bf)
    gm = None if metric is None else cuda(metric)
    ws = G.ct_workspace(gg, scheme, cached=cached)
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(nsteps):
        G.ct_rk_step(gg, gp, scheme, dt, gc, gpr, gb, gm, ws=ws, nfail=nfail)
    assert int(host(nfail)[0]) == 0
    return (c, p, b), (host(gc), host(gpr), host(gb))


@pytest.mark.parametrize("scheme", ["rk2", "rk3", "rk4"])
def test_ct_step_parity_flat(G, scheme):
    sch = {"rk2": O.RK2, "rk3": O.RK3, "rk4": O.RK4}[scheme]
    blk, og, metric, prim, bf, bc = ct_case((19, 13, 11), seed=5)
    (c, p, b), (gc, gp, gb) = run_ct_steps(G, blk, og, metric, prim, bf, bc, sch, 2)
    assert np.all(normwise(interior(gc, 3), interior(c, 3)) <= FP64_TOL)
    assert np.all(normwise(interior(gp, 3), interior(p, 3)) <= FP64_TOL)
    assert np.all(face_normwise(gb, b, blk.n, 3) <= FP64_TOL)
    assert np.abs(gb - bf).max() > 1e-6 * np.abs(bf).max()     # the field did evolve


@pytest.mark.parametrize("cached", [True, False])
@pytest.mark.parametrize("recon", [O.REC_MINMOD, O.REC_WENO5])
def test_ct_step_parity_schwarzschild(G, cached, recon):
    blk, og, metric, prim, bf, bc = ct_case((18, 12, 10), seed=7, curved=True)
    (c, p, b), (gc, gp, gb) = run_ct_steps(G, blk, og, metric, prim, bf, bc, O.RK3, 2, recon=recon, cached=cached)
    assert np.all(normwise(interior(gc, 3), interior(c, 3)) <= FP64_TOL)
    assert np.all(normwise(interior(gp, 3), interior(p, 3)) <= FP64_TOL)
    assert np.all(face_normwise(gb, b, blk.n, 3) <= FP64_TOL)


@pytest.mark.parametrize("n", [(9, 7, 1), (1, 10, 6), (8, 1, 5)])
def test_ct_thin_blocks(G, n):
    blk, og, metric, prim, bf, bc = ct_case(n, seed=11)
    (c, p, b), (gc, gp, gb) = run_ct_steps(G, blk, og, metric, prim, bf, bc, O.RK3, 2)
    assert np.all(normwise(interior(gc, 3), interior(c, 3), floor=1e-12) <= FP64_TOL)
    assert np.all(face_normwise(gb, b, blk.n, 3) <= FP64_TOL)


def test_ct_divergence_bit_exact_and_preserved(G):
    blk, og, metric, prim, bf, bc = ct_case((40, 36, 32), seed=13)
    gg = G.Grid(blk.n, 3, blk.dx)
    # a field with divergence: the oracle's divergence reproduced bit for bit
    rng = np.random.default_rng(1)
    noisy = bf + 1e-3 * rng.standard_normal(bf.shape)
    div, mx = G.ct_divergence(gg, cuda(noisy), maxabs=torch.zeros(1, dtype=torch.float64, device="cuda"),
                              div=torch.empty(gg.shape, dtype=torch.float64, device="cuda"))
    ref = O.ct_divergence(og, noisy)
    assert np.array_equal(host(div), ref)
    assert host(mx)[0] == np.abs(ref).max()
    # many steps keep the discrete divergence of a curl at round-off
    gp = gpu_params(G, G.WENO5, bc)
    op = O.make_params(recon=O.REC_WENO5, bc=bc)
    gc, gpr, gb = cuda(O.prim2con(og, op.gamma, prim)), cuda(prim), cuda(bf)
    ws = G.ct_workspace(gg, G.RK3)
    dt = 0.3 * min(blk.dx)
    for _ in range(40):
        G.ct_rk_step(gg, gp, G.RK3, dt, gc, gpr, gb, ws=ws)
    _, mx = G.ct_divergence(gg, gb, maxabs=torch.zeros(1, dtype=torch.float64, device="cuda"))
    scale = np.abs(host(gb)).max() / min(blk.dx)
    assert host(mx)[0] <= 1e-13 * scale
    assert np.abs(host(gb) - bf).max() > 1e-3 * np.abs(bf).max()


def test_ct_mixed_precision(G):
    blk, og, metric, prim, bf, bc = ct_case((24, 20, 16), seed=17, curved=True)
    (c, p, b), (gc, gp, gb) = run_ct_steps(G, blk, og, metric, prim, bf, bc, O.RK3, 2, precision=G.MIXED)
    assert np.all(normwise(interior(gc, 3), interior(c, 3)) <= MIXED_TOL)
    assert np.all(face_normwise(gb, b, blk.n, 3) <= MIXED_TOL)
    gg = G.Grid(blk.n, 3, blk.dx)
    _, mx = G.ct_divergence(gg, cuda(gb), maxabs=torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert host(mx)[0] <= 1e-13 * np.abs(gb).max() / min(blk.dx)


def test_ct_without_field_is_the_plain_step(G):
    blk, og, metric, prim, bf, bc = ct_case((19, 13, 11), seed=19, curved=True)
    prim[5:] = 0.0
    bf[:] = 0.0
    gg = G.Grid(blk.n, 3, blk.dx)
    gp = gpu_params(G, G.WENO5, bc)
    cons = O.prim2con(og, gp.gamma, prim, metric)
    gm = cuda(metric)
    c1, p1, b1 = cuda(cons), cuda(prim), cuda(bf)
    c2, p2 = cuda(cons), cuda(prim)
    for _ in range(2):
        G.ct_rk_step(gg, gp, G.RK3, 0.02, c1, p1, b1, gm)
        G.rk_step(gg, gp, G.RK3, 0.02, c2, p2, gm)
    assert np.array_equal(host(c1), host(c2))
    assert np.array_equal(host(p1), host(p2))
    assert np.all(host(b1) == 0.0)


@pytest.mark.parametrize("curved", [False, True])
def test_cell_field_from_faces_matches_oracle(G, curved):
    """grmhd_ct_cell_field: the primitive field of every interior cell is the
    mean of its two faces over sqrt(gamma), as the oracle forms it; nothing
    else of prim changes."""
    blk, og, metric, prim, bf, bc = ct_case((13, 7, 5), seed=4, curved=curved)
    rng = np.random.default_rng(3)
    start = prim + rng.normal(size=prim.shape) * 0.01      # a field not yet matching the faces
    g = G.Grid(blk.n, blk.ng, blk.dx)
    tp = cuda(start)
    G.ct_cell_field(g, cuda(bf), tp, None if metric is None else cuda(metric))
    got = host(tp)
    ref = O.ct_cell_field(start, bf, metric)
    inner = (slice(None),) + tuple(slice(blk.ng, s - blk.ng) for s in blk.shape)
    np.testing.assert_allclose(got[inner][5:], ref[inner][5:], rtol=4e-16, atol=0)
    np.testing.assert_array_equal(got[inner][:5], start[inner][:5])
    outer = np.ones(got.shape[1:], bool)
    outer[inner[1:]] = False
    np.testing.assert_array_equal(got[:, outer], start[:, outer])
