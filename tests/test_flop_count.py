"""The algorithmic operation count behind the benchmark's roofline.

``oracle/flop_count.py`` restates one cell's right-hand side in the paper's
3+1 form (Eqs. 6-9, 12, 13 and the readings of the oracle header) with a
counting scalar.  These tests check (1) that the restatement computes the
method -- its cell RHS equals the oracle's on a curved block with shift and
extrinsic curvature -- so that what is counted is the right arithmetic, and
(2) that the stored count the benchmark reads is the generator's output.
"""
import json
import os

import numpy as np

import oracle as O
from oracle import flop_count as FC
from paper_2210_17509_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _curved_block():
    n = (7, 6, 5)
    h = 0.3
    blk = I.Block(n, 3, (h, h, h), (3.0, 2.5, 4.0))
    met = I.schwarzschild_metric(blk)
    x, y, z = blk.centres()
    met[1] = 0.05 * np.sin(x)              # a smooth shift and off-diagonal metric
    met[2] = -0.03 * np.cos(y)
    met[3] = 0.02 * np.sin(z)
    met[5] = 0.02 * np.sin(x + y)
    met[8] = -0.01 * np.cos(z)
    kij = np.zeros((6,) + blk.shape)
    for c in range(6):
        kij[c] = 0.01 * (c + 1) * np.cos(x + 0.3 * c * y)
    prim = I.smooth_prims(blk, 21, rho_range=(0.3, 1.0), metric=met, vmax=0.4)
    return blk, prim, met, kij


def _restated_rhs(blk, prim, met, kij, cell, gamma, eps):
    i, j, k = cell
    idx = [1.0 / h for h in blk.dx]

    def at(q, ii, jj, kk, arr):
        return arr[q, kk, jj, ii]

    faces = {}
    for d in range(3):
        for side in (0, 1):
            c = [i, j, k]
            c[d] += side                       # face between c - e_d and c
            st = []
            for q in range(8):
                row = []
                for s in range(6):
                    p = list(c)
                    p[d] += s - 3
                    row.append(at(q, *p, prim))
                st.append(row)
            cm = list(c)
            cm[d] -= 1
            mm = [at(q, *cm, met) for q in range(10)]
            mp = [at(q, *c, met) for q in range(10)]
            faces[(d, side)] = FC.face_flux(st, mm, mp, d, gamma, eps)
    dmet = []
    for e in range(3):
        row = []
        for q in range(10):
            f = []
            for s in (-2, -1, 1, 2):
                p = [i, j, k]
                p[e] += s
                f.append(at(q, *p, met))
            row.append(FC.fd4(f, 1.0 / (12.0 * blk.dx[e])))
        dmet.append(row)
    pc = [prim[q, k, j, i] for q in range(8)]
    mc = [met[q, k, j, i] for q in range(10)]
    kc = [kij[q, k, j, i] for q in range(6)]
    src = FC.source(pc, mc, dmet, kc, gamma)
    return FC.cell_rhs([faces[(d, 0)] for d in range(3)], [faces[(d, 1)] for d in range(3)], src, idx)


def test_restated_rhs_equals_the_oracle():
    blk, prim, met, kij = _curved_block()
    gamma, eps = I.GAMMA, 1e-6
    og = O.Grid(blk.n, blk.ng, blk.dx)
    par = O.make_params(gamma=gamma, recon=O.REC_WENO5, weno_eps=eps)
    cells = np.array([(3, 3, 3), (5, 4, 6), (9, 8, 7), (4, 7, 5)])
    ref = O.rhs_cells(og, par, prim, cells, met, kij)
    scale = np.abs(ref).max(axis=0) + 1e-300
    for s, cell in enumerate(cells):
        got = np.array([FC._v(x) for x in _restated_rhs(blk, prim, met, kij, cell, gamma, eps)])
        err = np.abs(got - ref[s]) / scale
        assert np.all(err < 1e-12), (cell, err)


def test_stored_count_is_the_generators():
    with open(os.path.join(ROOT, "paper_2210_17509_gb300", "flop_counts.json")) as f:
        stored = json.load(f)
    c = FC.count()
    assert stored["rhs_curved_weno5_per_cell"] == c["cell_total"]
    assert stored["parts"] == json.loads(json.dumps(c))


def test_executed_counts_are_the_committed_profiles():
    """The executed FP64 counts the roofline quotes are the ones in the
    committed ncu summary of the three RHS kernels."""
    from paper_2210_17509_gb300 import roofline as R
    path = os.path.join(ROOT, "profiles", "rhs_three_pass_fp64_cached_weno5_curved_96cube.md")
    row = next(ln for ln in open(path) if ln.startswith("| of them DADD / DMUL / DFMA"))
    cells = [c.strip() for c in row.strip().strip("|").split("|")[1:4]]  # the three RHS kernels
    got = [tuple(int(x) for x in c.split("/")) for c in cells]
    assert got == [R.EXECUTED_FP64_PER_CELL[k] for k in ("rhs_states_kernel", "rhs_face_kernel", "rhs_div_kernel")]
