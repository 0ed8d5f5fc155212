"""Polytropic EOS (Sec. 2.3, P = K rho^gamma; reading R20 of the oracle
header) on the CUDA path, through the C ABI, against the oracle:

* prim -> cons (the input pressure replaced by K rho^gamma) and the
  recovery from D, S_i and B^i: 1e-12 per field, flat and Schwarzschild,
  magnetised states up to v = 0.9, from guesses 20% off;
* the recovery does not read tau (bit-identical results);
* RHS (face pressure from the face density): 1e-12 FP64, 1e-5 mixed, for
  minmod and WENO5, flat periodic and Schwarzschild with copy boundaries;
* SSP-RK3 steps, FP64 cached and uncached and mixed, and a
  constrained-transport step.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_17509_gb300 import inputs as I
from tests.helpers import FP64_TOL, MIXED_TOL, normwise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K, GAM = 100.0, 2.0


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


def interior(a, ng=3):
    return a[(slice(None),) + tuple(slice(ng, s - ng) for s in a.shape[1:])]


def case(n, seed, curved, vmax=0.9, b_scale=1.0, log_rho=(-4.0, -2.5), K=K, GAM=GAM):
    n = tuple(n)
    if curved:
        h = 8.0 / max(n)
        blk = I.Block(n, 3, (h, h, h), (4.0, 4.0, 4.0))
        m = I.schwarzschild_metric(blk)
    else:
        blk = I.Block(n, 3, tuple(1.0 / v for v in n), (0.0, 0.0, 0.0))
        m = None
    prim = I.polytrope_prims(blk, seed, K, GAM, m, vmax=vmax, log_rho=log_rho, b_scale=b_scale)
    return blk, m, prim


def params(G, recon=None, bc=None, precision=None, K=K, GAM=GAM):
    p = G.Params(gamma=GAM, eos=G.EOS_POLYTROPE, poly_K=K)
    if recon is not None:
        p.recon = recon
    if bc is not None:
        p.bc = bc
    if precision is not None:
        p.precision = precision
    return p


def oparams(recon=O.REC_WENO5, bc=O.BC_PERIODIC, K=K, GAM=GAM):
    return O.make_params(gamma=GAM, recon=recon, bc=bc, eos=O.EOS_POLYTROPE, poly_K=K)


# gamma = 2 takes the product form of K rho^(gamma - 1) on the GPU, other gammas pow
EOS_CASES = [(100.0, 2.0), (10.0, 5.0 / 3.0)]


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("eos", EOS_CASES)
def test_prim2con_and_recovery(G, curved, eos):
    Kc, Gc = eos
    blk, m, prim = case((12, 10, 9), 3, curved, K=Kc, GAM=Gc)
    og = O.Grid(blk.n, 3, blk.dx)
    gg = G.Grid(blk.n, 3, blk.dx)
    junk = prim.copy()
    junk[4] *= np.random.default_rng(2).uniform(0.2, 5.0, junk[4].shape)
    op = oparams(K=Kc, GAM=Gc)
    gpp = params(G, K=Kc, GAM=Gc)
    ref_cons = O.prim2con(og, Gc, prim, m, params=op)
    gm = None if m is None else cuda(m)
    gcons = host(G.prim2con(gg, gpp, cuda(junk), gm))
    assert np.all(normwise(gcons, ref_cons) <= FP64_TOL)
    ref, st, nf = O.con2prim(og, op, ref_cons, m, prim)
    assert nf == 0
    guess = prim.copy()
    guess[1:4] *= 0.8
    gp = cuda(guess)
    status = torch.zeros(gg.shape, dtype=torch.int8, device="cuda")
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.con2prim(gg, gpp, cuda(ref_cons), gp, gm, status=status, nfail=nfail)
    assert int(host(nfail)[0]) == 0
    assert np.all(normwise(interior(host(gp)), interior(ref)) <= FP64_TOL)
    # tau is not read
    c2 = ref_cons.copy()
    c2[4] *= 3.0
    gp2 = cuda(guess)
    G.con2prim(gg, gpp, cuda(c2), gp2, gm)
    assert np.array_equal(host(gp2), host(gp))


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("recon", ["minmod", "weno5"])
@pytest.mark.parametrize("mixed", [False, True])
def test_rhs(G, curved, recon, mixed):
    blk, m, prim = case((19, 13, 11), 5, curved, vmax=0.5, b_scale=0.3, log_rho=(-3.5, -3.0))
    og = O.Grid(blk.n, 3, blk.dx)
    bc = O.BC_COPY if curved else O.BC_PERIODIC
    prim = O.fill_ghosts(og, bc, prim)
    orec = O.REC_WENO5 if recon == "weno5" else O.REC_MINMOD
    ref = O.rhs(og, oparams(orec, bc), prim, m)
    gg = G.Grid(blk.n, 3, blk.dx)
    p = params(G, G.WENO5 if recon == "weno5" else G.MINMOD, bc, G.MIXED if mixed else None)
    out = host(G.rhs(gg, p, cuda(prim), None if m is None else cuda(m)))
    err = normwise(interior(out), interior(ref))
    assert np.all(err <= (MIXED_TOL if mixed else FP64_TOL)), err


@pytest.mark.parametrize("mode", ["fp64_cached", "fp64_uncached", "mixed"])
@pytest.mark.parametrize("eos", EOS_CASES)
def test_rk3_steps(G, mode, eos):
    Kc, Gc = eos
    blk, m, prim = case((18, 12, 10), 7, True, vmax=0.5, b_scale=0.3, log_rho=(-3.5, -3.0), K=Kc, GAM=Gc)
    og = O.Grid(blk.n, 3, blk.dx)
    prim = O.fill_ghosts(og, O.BC_COPY, prim)
    op = oparams(O.REC_WENO5, O.BC_COPY, K=Kc, GAM=Gc)
    cons = O.prim2con(og, Gc, prim, m, params=op)
    dt = 0.25 * blk.dx[0]
    c, pr = cons, prim
    for _ in range(2):
        c, pr, nf = O.rk_step(og, op, O.RK3, dt, c, pr, m)
        assert nf == 0
    gg = G.Grid(blk.n, 3, blk.dx)
    p = params(G, G.WENO5, G.BC_COPY, G.MIXED if mode == "mixed" else None, K=Kc, GAM=Gc)
    gc, gp, gm = cuda(cons), cuda(prim), cuda(m)
    ws = G.workspace(gg, G.RK3, cached=(mode != "fp64_uncached"))
    nfail = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        G.rk_step(gg, p, G.RK3, dt, gc, gp, gm, ws=ws, nfail=nfail)
    assert int(host(nfail)[0]) == 0
    tol = MIXED_TOL if mode == "mixed" else FP64_TOL
    assert np.all(normwise(interior(host(gc)), interior(c)) <= tol)
    assert np.all(normwise(interior(host(gp)), interior(pr)) <= tol)


def test_ct_step(G):
    blk = I.Block((16, 12, 10), 3, (1 / 16, 1 / 12, 1 / 10), (0.0, 0.0, 0.0))
    og = O.Grid(blk.n, 3, blk.dx)
    prim = I.polytrope_prims(blk, 9, K, GAM, vmax=0.4, b_scale=0.0, log_rho=(-3.5, -3.0))
    bf = I.face_curl(blk, I.edge_potential(blk, 109))
    bf *= 0.3 * np.sqrt(10 ** -3.5) / np.abs(interior(bf)).max()
    prim = O.fill_ghosts(og, O.BC_PERIODIC, O.ct_cell_field(prim, bf))
    op = oparams()
    cons = O.prim2con(og, GAM, prim, None, params=op)
    dt = 0.25 * min(blk.dx)
    c, pr, b, nf = O.ct_rk_step(og, op, O.RK3, dt, cons, prim, bf)
    assert nf == 0
    gg = G.Grid(blk.n, 3, blk.dx)
    gc, gp, gb = cuda(cons), cuda(prim), cuda(bf)
    G.ct_rk_step(gg, params(G), G.RK3, dt, gc, gp, gb)
    assert np.all(normwise(interior(host(gp)), interior(pr)) <= FP64_TOL)
    fb, rb = host(gb), b
    sl = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    assert np.abs(fb[sl] - rb[sl]).max() <= FP64_TOL * np.abs(rb[sl]).max()
