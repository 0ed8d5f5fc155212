"""Pins of the oracle's polytropic EOS (reading R20: P = K rho^Gamma as in
Sec. 2.3's EOS paragraph; recovery from D, S_i and B^i) against what the
mathematics fixes:

* recovery inverts prim -> cons (the covariant projections) to round-off on
  random magnetised states, flat and on Schwarzschild;
* tau is not read by the recovery, and the pressure entry of the input is
  not read by prim -> cons (the EOS sets it);
* the atmosphere is rho_atm, v = 0, P = K rho_atm^Gamma;
* with uniform density the polytrope's RHS equals the Gamma-law RHS of the
  same state (the face pressure then equals the cell pressure);
* a smooth sound wave evolved under the polytrope and under the Gamma-law
  (whose smooth flows are isentropic) converge to each other with resolution.
"""
import numpy as np

import oracle as O
from paper_2210_17509_gb300 import inputs as I

K, GAM = 100.0, 2.0          # the paper's TOV polytrope (Sec. 4.4)


def poly_params(recon=O.REC_WENO5, bc=O.BC_PERIODIC, K=K, gamma=GAM):
    return O.make_params(gamma=gamma, recon=recon, bc=bc, eos=O.EOS_POLYTROPE, poly_K=K)


def random_states(n, seed, metric=False, K=K, gamma=GAM):
    blk = I.Block((n, n, n), 3, (8.0 / n,) * 3, (4.0,) * 3) if metric else I.Block((n, n, n), 3, (1.0 / n,) * 3,
                                                                                     (0.0,) * 3)
    m = I.schwarzschild_metric(blk) if metric else None
    return blk, m, I.polytrope_prims(blk, seed, K, gamma, m)


def test_recovery_inverts_prim2con():
    for metric in (False, True):
        blk, m, prim = random_states(8, 3, metric)
        g = O.Grid(blk.n, 3, blk.dx)
        p = poly_params()
        cons = O.prim2con(g, GAM, prim, m, params=p)
        out, st, nf = O.con2prim(g, p, cons, m)
        assert nf == 0
        inner = (slice(None),) + (slice(3, -3),) * 3
        for q in range(8):
            a, b = out[q][inner[1:]], prim[q][inner[1:]]
            assert np.abs(a - b).max() <= 1e-11 * max(np.abs(b).max(), 1e-300), (metric, q)


def test_recovery_ignores_tau_and_prim2con_ignores_pressure():
    blk, m, prim = random_states(6, 5, True)
    g = O.Grid(blk.n, 3, blk.dx)
    p = poly_params()
    cons = O.prim2con(g, GAM, prim, m, params=p)
    junk = prim.copy()
    junk[4] *= np.random.default_rng(1).uniform(0.1, 10.0, junk[4].shape)
    assert np.array_equal(O.prim2con(g, GAM, junk, m, params=p), cons)
    a, _, _ = O.con2prim(g, p, cons, m)
    c2 = cons.copy()
    c2[4] *= 1.7
    b, _, _ = O.con2prim(g, p, c2, m)
    assert np.array_equal(a, b)


def test_atmosphere():
    p = poly_params()
    U = np.array([-1e-3, 0.1, 0.0, 0.0, 1.0, 0.2, 0.0, 0.0])
    out, st = O.con2prim_point(U, p)
    assert st != 0
    assert out[0] == p.rho_atm and np.all(out[1:4] == 0.0)
    assert out[4] == K * p.rho_atm ** GAM
    assert np.array_equal(out[5:], U[5:])


def test_uniform_density_rhs_equals_gamma_law():
    for metric in (False, True):
        blk, m, prim = random_states(10, 7, metric)
        prim[0] = 10 ** -3.0
        prim[4] = K * prim[0] ** GAM
        prim[5:] *= 0.3
        g = O.Grid(blk.n, 3, blk.dx)
        bc = O.BC_COPY if metric else O.BC_PERIODIC
        prim = O.fill_ghosts(g, bc, prim)
        for recon in (O.REC_MINMOD, O.REC_WENO5):
            rp = O.rhs(g, poly_params(recon, bc), prim, m)
            ri = O.rhs(g, O.make_params(gamma=GAM, recon=recon, bc=bc), prim, m)
            scale = np.abs(ri).max(axis=(1, 2, 3))
            err = np.abs(rp - ri).max(axis=(1, 2, 3)) / np.maximum(scale, 1e-300)
            assert np.all(err <= 1e-12), (metric, recon, err)


def sound_wave(n, t_end, eos):
    blk = I.Block((n, 1, 1), 3, (1.0 / n, 1.0 / n, 1.0 / n), (0.0, 0.0, 0.0))
    g = O.Grid(blk.n, 3, blk.dx)
    x, _, _ = blk.centres()
    Kw = 0.1
    prim = np.zeros((8,) + blk.shape)
    prim[0] = 1.0 + 0.05 * np.sin(2 * np.pi * x)
    prim[1] = 0.05 * np.sin(2 * np.pi * x)
    prim[4] = Kw * prim[0] ** GAM
    prim[5] = 0.1
    prim[6] = 0.05 * np.cos(2 * np.pi * x)
    prim = O.fill_ghosts(g, O.BC_PERIODIC, prim)
    if eos == O.EOS_POLYTROPE:
        p = poly_params(O.REC_WENO5, O.BC_PERIODIC, K=Kw)
    else:
        p = O.make_params(gamma=GAM, recon=O.REC_WENO5, bc=O.BC_PERIODIC)
    cons = O.prim2con(g, GAM, prim, None, params=p)
    nsteps = int(round(t_end / (0.4 / n)))
    dt = t_end / nsteps
    for _ in range(nsteps):
        cons, prim, nf = O.rk_step(g, p, O.RK3, dt, cons, prim)
        assert nf == 0
    return prim[:, 3, 3, 3:-3]


def test_isentropic_sound_wave_converges_to_the_gamma_law():
    diffs = []
    for n in (32, 64, 128):
        a = sound_wave(n, 0.3, O.EOS_POLYTROPE)
        b = sound_wave(n, 0.3, O.EOS_IDEAL)
        diffs.append(np.abs(a[0] - b[0]).mean())
    assert diffs[0] > 0.0
    assert diffs[1] < diffs[0] / 3.0 and diffs[2] < diffs[1] / 3.0, diffs
