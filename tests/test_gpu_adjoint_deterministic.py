"""GRMHD_DETERMINISTIC: the reverse calls add in a fixed order (each
direction's face adjoint in six launches by face index mod 6, the Gamma sums
through per-warp slots added in slot order), so two runs give the same bits;
and the fixed order changes nothing but rounding against the atomic adds,
whose correctness the transposition tests of test_gpu_adjoint.py pin."""
import numpy as np
import pytest

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


def block(G, n, curved, recon, seed=3):
    if curved:
        blk = I.Block(n, 3, tuple(8.0 / max(n) for _ in range(3)), (4.0, 4.0, 4.0))
        met = I.schwarzschild_metric(blk)
        prim = I.smooth_prims(blk, seed, rho_range=(0.1, 1.0), metric=met)
        bc = G.BC_COPY
    else:
        blk = I.Block(n, 3, tuple(1.0 / max(n) for _ in range(3)), (0.0, 0.0, 0.0))
        met = None
        prim = I.smooth_prims(blk, seed)
        bc = G.BC_PERIODIC
    g = G.Grid(blk.n, 3, blk.dx)
    p = G.Params(recon=recon, bc=bc)
    tp = torch.from_numpy(prim).cuda()
    G.fill_ghosts(g, bc, tp)
    tm = None if met is None else torch.from_numpy(met).cuda()
    return g, p, tp, tm, blk


def det(G, p):
    import dataclasses
    return dataclasses.replace(p, flags=p.flags | G.DETERMINISTIC)


def seeds(G, g, seed):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    mask = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    mask[3:-3, 3:-3, 3:-3] = 1.0
    ub = torch.randn((8,) + g.shape, dtype=torch.float64, device="cuda", generator=gen) * mask
    pb = torch.randn((8,) + g.shape, dtype=torch.float64, device="cuda", generator=gen)
    return ub, pb


def close(a, b, rel):
    scale = float(b.abs().max())
    return float((a - b).abs().max()) <= rel * scale


@pytest.mark.parametrize("curved,recon,n,scheme", [(True, 1, (12, 10, 9), 3), (False, 1, (16, 7, 13), 3),
                                                  (False, 0, (13, 4, 7), 3), (True, 1, (9, 11, 8), 2)])
def test_deterministic_step_adjoint_repeats_to_the_bit(G, curved, recon, n, scheme):
    """SSP-RK3 / RK2 reverse step (WENO5: the buffered face pass; minmod: the
    per-face pass, one direction and one residue per launch) twice with the
    flag: the same bits; against the atomic adds: rounding only."""
    g, p, prim, met, blk = block(G, n, curved, recon)
    cons = G.prim2con(g, p, prim, met)
    dt = 0.25 * min(blk.dx)
    ub0, pb0 = seeds(G, g, 11)
    out = []
    for pp in (det(G, p), det(G, p), p):
        ub, pb = ub0.clone(), pb0.clone()
        gb = torch.zeros(1, dtype=torch.float64, device="cuda")
        G.rk_step_adjoint(g, pp, scheme, dt, cons, prim, ub, pb, gb, met)
        torch.cuda.synchronize()
        out.append((ub, pb, gb))
    for k in range(3):
        assert torch.equal(out[0][k], out[1][k])
    for k in range(2):
        assert close(out[0][k], out[2][k], 1e-13)
    assert abs(float(out[0][2]) - float(out[2][2])) <= 1e-13 * abs(float(out[2][2]))


@pytest.mark.parametrize("curved,recon", [(True, 1), (False, 1), (False, 0)])
def test_deterministic_rhs_adjoint_repeats_to_the_bit(G, curved, recon):
    """grmhd_rhs_adjoint (no workspace: the per-face pass) on ragged extents,
    one of them with fewer than six faces, so that some residue launches have
    no face."""
    g, p, prim, met, blk = block(G, (13, 4, 7), curved, recon)
    gen = torch.Generator(device="cuda").manual_seed(5)
    rb = torch.randn((8,) + g.shape, dtype=torch.float64, device="cuda", generator=gen)
    out = []
    for pp in (det(G, p), det(G, p), p):
        pb = torch.zeros_like(prim)
        gb = torch.zeros(1, dtype=torch.float64, device="cuda")
        G.rhs_adjoint(g, pp, prim, rb, pb, gb, met)
        torch.cuda.synchronize()
        out.append((pb, gb))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert close(out[0][0], out[2][0], 1e-13)
    assert abs(float(out[0][1]) - float(out[2][1])) <= 1e-13 * abs(float(out[2][1]))


def test_deterministic_checkpointed_gradient_repeats_to_the_bit(G, A):
    """evolve(..., deterministic=True): the gradient with respect to the
    initial primitives and Gamma after 4 SSP-RK3 steps (checkpoint every 2) is
    the same to the bit in two runs, and within rounding of the atomic one."""
    g, p, prim, met, blk = block(G, (10, 10, 10), True, 1, seed=8)
    dt = 0.25 * blk.dx[0]
    res = []
    for flag in (True, True, False):
        x = prim[:, 3:-3, 3:-3, 3:-3].clone().requires_grad_(True)
        gam = torch.tensor(p.gamma, dtype=torch.float64, requires_grad=True)
        out = A.evolve(x, gam, g, p, G.RK3, dt, 4, checkpoint_every=2, metric=met, deterministic=flag)
        A.density_l2(out, g, met).backward()
        res.append((x.grad.cpu().numpy(), float(gam.grad.item())))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
    assert np.abs(res[0][0] - res[2][0]).max() <= 1e-13 * np.abs(res[2][0]).max()
    assert abs(res[0][1] - res[2][1]) <= 1e-13 * abs(res[2][1])
