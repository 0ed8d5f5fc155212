"""Host checks of the seeded input builders (no GPU)."""
import json
import os

import numpy as np

from paper_2210_17509_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_balsara_table_matches_golden_copy():
    """The shock-tube states in inputs.BALSARA are the paper's table (golden copy with citation)."""
    gold = json.load(open(os.path.join(GOLDEN, "balsara_table.json")))["tests"]
    for k, t in I.BALSARA.items():
        gt = gold[f"balsara{k}"]
        assert t["Bx"] == gt["Bx"] and abs(t["gamma"] - gt["gamma"]) < 1e-15 and t["t_ref"] == gt["t_ref"]
        for side in ("left", "right"):
            rho, eps, v, byz = t[side]
            gs = gt[side]
            assert (rho, eps) == (gs["rho"], gs["eps"])
            assert list(v) == gs["v"] and list(byz) == gs["ByBz"]


def test_shocktube_orientations_are_relabellings():
    for test in (1, 5):
        bx, px, g, _ = I.shocktube(test, 32, 0, 2)
        for axis in (1, 2):
            b, p, _, _ = I.shocktube(test, 32, axis, 2)
            assert b.n[axis] == 32 and b.dx == bx.dx
            # tube profile along the axis, components relabelled to the x frame
            prof = []
            for q in range(8):
                a = p[q]
                idx = [2, 2, 2]  # (z, y, x) transverse index inside the interior
                idx[2 - axis] = slice(None)
                prof.append(a[tuple(idx)])
            prof = np.array(prof)
            comp = [0, 1 + axis, 1 + (axis + 1) % 3, 1 + (axis + 2) % 3, 4,
                    5 + axis, 5 + (axis + 1) % 3, 5 + (axis + 2) % 3]
            ref = px[:, 2, 2, :]
            assert np.array_equal(prof[comp], ref)
