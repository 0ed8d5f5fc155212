"""Algorithmic FP64 operation count of the method-of-lines RHS, per cell.

TEST AND MEASUREMENT INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the
product path never imports it.  ``python -m oracle.flop_count`` writes
``paper_2210_17509_gb300/flop_counts.json``, the per-cell count the
benchmark's roofline divides by the kernel time; ``tests/test_flop_count.py``
checks that file against this generator and checks this restatement's
arithmetic against the oracle.

What is counted: one evaluation of the right-hand side dU/dt = -d_i F^i + S
(Eq. 11) of one interior cell, with the stage combination of the RK update,
written plainly in the 3+1 form the paper prints:
  - WENO5 reconstruction (Jiang-Shu indicators, reading R3) of the 8
    primitives to both sides of a face, each face value on its own;
  - the face metric as the mean of the two cells (reading R7), its
    determinant, sqrt(gamma) and the inverse entries the flux needs;
  - per side: W, b^mu (reading R6), h, rho h*, P*, the conserved vector
    (Eqs. 6-9), the flux (Eq. 12) and the fast-magnetosonic signal speeds in
    closed form (reading R5);
  - the HLLE combination of the 8 components (Sec. 2.3 step 3);
  - the flux divergence (every face counted once: a cell owns 3 of its 6);
  - the source terms (Eq. 13) in the standard 3+1 form, with 4th-order
    centred metric derivatives (reading R7) and K_ij;
  - the stage combination U = c0 U0 + c1 (U + dt L).
Each +, -, *, / and sqrt counts one, as do min and max; a fused multiply-add
counts two.  Nothing is shared between the two faces of a cell or between the
two sides of a face beyond what the formulas themselves share, so the count
is that of a straightforward evaluation, not of any particular kernel.
"""
from __future__ import annotations

import json
import math
import os

COUNTS = {"add": 0, "mul": 0, "div": 0, "sqrt": 0, "minmax": 0}


def _v(x):
    return x.v if isinstance(x, Num) else float(x)


class Num:
    """A float that counts the arithmetic done on it."""
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = _v(v)

    def __add__(self, o):
        COUNTS["add"] += 1
        return Num(self.v + _v(o))

    __radd__ = __add__

    def __sub__(self, o):
        COUNTS["add"] += 1
        return Num(self.v - _v(o))

    def __rsub__(self, o):
        COUNTS["add"] += 1
        return Num(_v(o) - self.v)

    def __mul__(self, o):
        COUNTS["mul"] += 1
        return Num(self.v * _v(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        COUNTS["div"] += 1
        return Num(self.v / _v(o))

    def __rtruediv__(self, o):
        COUNTS["div"] += 1
        return Num(_v(o) / self.v)

    def __neg__(self):
        return Num(-self.v)

    def __lt__(self, o):
        return self.v < _v(o)

    def __gt__(self, o):
        return self.v > _v(o)


def sqrt(x):
    COUNTS["sqrt"] += 1
    return Num(math.sqrt(_v(x)))


def fmin(a, b):
    COUNTS["minmax"] += 1
    return Num(min(_v(a), _v(b)))


def fmax(a, b):
    COUNTS["minmax"] += 1
    return Num(max(_v(a), _v(b)))


def reset():
    for k in COUNTS:
        COUNTS[k] = 0


def total():
    return sum(COUNTS.values())


# ------------------------------------------------------------- the method --
SYM = ((4, 5, 6), (5, 7, 8), (6, 8, 9))   # gamma_ij in the 10-component metric


def weno5(um2, um1, u0, up1, up2, eps):
    """Value at the right face of cell 0 from cells -2 .. 2 (Jiang-Shu)."""
    q0 = (2.0 * um2 - 7.0 * um1 + 11.0 * u0) / 6.0
    q1 = (-1.0 * um1 + 5.0 * u0 + 2.0 * up1) / 6.0
    q2 = (2.0 * u0 + 5.0 * up1 - up2) / 6.0
    d0 = um2 - 2.0 * um1 + u0
    e0 = um2 - 4.0 * um1 + 3.0 * u0
    d1 = um1 - 2.0 * u0 + up1
    e1 = um1 - up1
    d2 = u0 - 2.0 * up1 + up2
    e2 = 3.0 * u0 - 4.0 * up1 + up2
    b0 = (13.0 / 12.0) * (d0 * d0) + 0.25 * (e0 * e0)
    b1 = (13.0 / 12.0) * (d1 * d1) + 0.25 * (e1 * e1)
    b2 = (13.0 / 12.0) * (d2 * d2) + 0.25 * (e2 * e2)
    s0 = eps + b0
    s1 = eps + b1
    s2 = eps + b2
    a0 = 0.1 / (s0 * s0)
    a1 = 0.6 / (s1 * s1)
    a2 = 0.3 / (s2 * s2)
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def inverse_sym(g):
    """det and inverse of a symmetric 3x3 [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]
    by cofactors; returns (det, gu) with gu as nested lists."""
    xx, xy, xz = g[0][0], g[0][1], g[0][2]
    yy, yz, zz = g[1][1], g[1][2], g[2][2]
    cxx = yy * zz - yz * yz
    cxy = xz * yz - xy * zz
    cxz = xy * yz - xz * yy
    cyy = xx * zz - xz * xz
    cyz = xy * xz - xx * yz
    czz = xx * yy - xy * xy
    det = xx * cxx + xy * cxy + xz * cxz
    idet = 1.0 / det
    gu = [[cxx * idet, cxy * idet, cxz * idet],
          [cxy * idet, cyy * idet, cyz * idet],
          [cxz * idet, cyz * idet, czz * idet]]
    return det, gu


def lower(g, a):
    return [g[i][0] * a[0] + g[i][1] * a[1] + g[i][2] * a[2] for i in range(3)]


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def side(prim, alpha, beta, g, sg, guu_d, d, gamma):
    """Conserved vector (Eqs. 6-9), flux along d (Eq. 12) and signal speeds
    (reading R5) of one primitive state at one face."""
    rho, v, P, B = prim[0], prim[1:4], prim[4], prim[5:8]
    vl = lower(g, v)
    v2 = dot(v, vl)
    W = 1.0 / sqrt(1.0 - v2)
    Bl = lower(g, B)
    BB = dot(B, Bl)
    Bv = dot(B, vl)
    ab0 = W * Bv                                     # alpha b^0
    bl = [Bl[i] / W + ab0 * vl[i] for i in range(3)]  # b_i
    b2 = (BB + ab0 * ab0) / (W * W)
    h = 1.0 + gamma / (gamma - 1.0) * P / rho
    rhoh = rho * h
    hs = rhoh + b2                                   # rho h*
    Ps = P + 0.5 * b2                                # P*
    hsW2 = hs * W * W
    D = sg * rho * W
    S = [sg * (hsW2 * vl[i] - ab0 * bl[i]) for i in range(3)]
    tau = sg * (hsW2 - Ps - ab0 * ab0) - D
    Bc = [sg * B[i] for i in range(3)]
    U = [D, S[0], S[1], S[2], tau, Bc[0], Bc[1], Bc[2]]
    vt = v[d] - beta[d] / alpha                      # v^d - beta^d / alpha
    F = [alpha * (D * vt)]
    for j in range(3):
        f = S[j] * vt - bl[j] * Bc[d] / W
        if j == d:
            f = f + sg * Ps
        F.append(alpha * f)
    F.append(alpha * (tau * vt + sg * Ps * v[d] - ab0 * Bc[d] / W))
    for k in range(3):
        F.append(alpha * (Bc[k] * vt - Bc[d] * (v[k] - beta[k] / alpha)))
    cs2 = gamma * P / rhoh
    va2 = b2 / hs
    a2 = cs2 + va2 - cs2 * va2
    den = 1.0 - v2 * a2
    root = sqrt(a2 * (1.0 - v2) * (guu_d * den - v[d] * v[d] * (1.0 - a2)))
    base = v[d] * (1.0 - a2)
    lam_m = alpha * (base - root) / den - beta[d]
    lam_p = alpha * (base + root) / den - beta[d]
    return U, F, lam_m, lam_p


def face_flux(stencil, met_m, met_p, d, gamma, eps):
    """HLLE flux through the face between cells c-1 and c along d from the
    8 primitives on cells c-3 .. c+2 (stencil[q][0..5]) and the metric of
    the two cells beside the face."""
    pL, pR = [], []
    for q in range(8):
        u = stencil[q]
        pL.append(weno5(u[0], u[1], u[2], u[3], u[4], eps))
        pR.append(weno5(u[5], u[4], u[3], u[2], u[1], eps))
    m = [0.5 * (met_m[c] + met_p[c]) for c in range(10)]
    alpha, beta = m[0], m[1:4]
    g = [[m[SYM[i][j]] for j in range(3)] for i in range(3)]
    det, gu = inverse_sym(g)
    sg = sqrt(det)
    UL, FL, lmL, lpL = side(pL, alpha, beta, g, sg, gu[d][d], d, gamma)
    UR, FR, lmR, lpR = side(pR, alpha, beta, g, sg, gu[d][d], d, gamma)
    xm = fmin(0.0, fmin(lmL, lmR))
    xp = fmax(0.0, fmax(lpL, lpR))
    xpm = xp * xm
    idn = 1.0 / (xp - xm)
    return [(xp * FL[c] - xm * FR[c] + xpm * (UR[c] - UL[c])) * idn for c in range(8)]


def fd4(f, idx12):
    """4th-order centred derivative from f(-2), f(-1), f(1), f(2); idx12 = 1 / (12 dx)."""
    return (f[0] - f[3] + 8.0 * (f[2] - f[1])) * idx12


def source(prim, met, dmet, kij, gamma):
    """Eq. 13 in the standard 3+1 form for a static lapse and shift:
      S_{S_i} = alpha sqrt(gamma) [T^00 (beta^j beta^k d_i g_jk / 2 - alpha d_i alpha)
                + T^0j beta^k d_i g_jk + T^0_j d_i beta^j + T^jk d_i g_jk / 2],
      S_tau   = alpha sqrt(gamma) [T^00 (beta^i beta^j K_ij - beta^i d_i alpha)
                + T^0i (2 beta^j K_ij - d_i alpha) + T^ij K_ij];
    dmet[i][c] = d_i of metric component c.  Returns [S_x, S_y, S_z, S_tau]."""
    alpha, beta = met[0], met[1:4]
    g = [[met[SYM[i][j]] for j in range(3)] for i in range(3)]
    det, gu = inverse_sym(g)
    sg = sqrt(det)
    rho, v, P, B = prim[0], prim[1:4], prim[4], prim[5:8]
    vl = lower(g, v)
    W = 1.0 / sqrt(1.0 - dot(v, vl))
    Bl = lower(g, B)
    ab0 = W * dot(B, vl)
    b0 = ab0 / alpha
    vt = [v[i] - beta[i] / alpha for i in range(3)]
    bu = [B[i] / W + ab0 * vt[i] for i in range(3)]   # b^i
    b2 = (dot(B, Bl) + ab0 * ab0) / (W * W)
    hs = rho + gamma / (gamma - 1.0) * P + b2
    Ps = P + 0.5 * b2
    ia2 = 1.0 / (alpha * alpha)
    u0 = W / alpha
    ui = [W * vt[i] for i in range(3)]
    T00 = hs * u0 * u0 - Ps * ia2 - b0 * b0
    T0 = [hs * u0 * ui[i] + Ps * beta[i] * ia2 - b0 * bu[i] for i in range(3)]
    T = [[hs * ui[i] * ui[j] + Ps * (gu[i][j] - beta[i] * beta[j] * ia2) - bu[i] * bu[j] for j in range(3)]
         for i in range(3)]
    betal = lower(g, beta)
    T0l = [betal[j] * T00 + g[j][0] * T0[0] + g[j][1] * T0[1] + g[j][2] * T0[2] for j in range(3)]
    asg = alpha * sg
    out = []
    for i in range(3):
        dg = [[dmet[i][SYM[a][b]] for b in range(3)] for a in range(3)]
        dgb = [dg[j][0] * beta[0] + dg[j][1] * beta[1] + dg[j][2] * beta[2] for j in range(3)]  # d_i g_jk beta^k
        s = T00 * (0.5 * dot(beta, dgb) - alpha * dmet[i][0]) + dot(T0, dgb)
        s = s + T0l[0] * dmet[i][1] + T0l[1] * dmet[i][2] + T0l[2] * dmet[i][3]
        half = T[0][0] * dg[0][0] + T[1][1] * dg[1][1] + T[2][2] * dg[2][2] \
            + 2.0 * (T[0][1] * dg[0][1] + T[0][2] * dg[0][2] + T[1][2] * dg[1][2])
        out.append(asg * (s + 0.5 * half))
    K = [[kij[(0, 1, 2, 1, 3, 4, 2, 4, 5)[3 * a + b]] for b in range(3)] for a in range(3)]
    Kb = [K[j][0] * beta[0] + K[j][1] * beta[1] + K[j][2] * beta[2] for j in range(3)]
    da = [dmet[i][0] for i in range(3)]
    st = T00 * (dot(beta, Kb) - dot(beta, da))
    st = st + dot(T0, [2.0 * Kb[i] - da[i] for i in range(3)])
    st = st + T[0][0] * K[0][0] + T[1][1] * K[1][1] + T[2][2] * K[2][2] \
        + 2.0 * (T[0][1] * K[0][1] + T[0][2] * K[0][2] + T[1][2] * K[1][2])
    out.append(asg * st)
    return out


def cell_rhs(faces_lo, faces_hi, src, idx):
    """-sum_d (F_hi - F_lo) / dx_d plus the source (D and B~ have none)."""
    out = []
    for c in range(8):
        r = (faces_hi[0][c] - faces_lo[0][c]) * idx[0]
        r = r + (faces_hi[1][c] - faces_lo[1][c]) * idx[1]
        r = r + (faces_hi[2][c] - faces_lo[2][c]) * idx[2]
        r = -r
        if 1 <= c <= 4:
            r = r + src[c - 1]
        out.append(r)
    return out


def stage(u0, u, L, c0, c1, dt):
    return [c0 * u0[c] + c1 * (u[c] + dt * L[c]) for c in range(8)]


# ------------------------------------------------------------- the count --
def _state(seed=0):
    """A representative smooth magnetised state with shift (values only
    steer which branch min/max take; the count does not depend on them)."""
    import random
    r = random.Random(seed)
    prim = [[Num(x) for x in row] for row in
            [[1.0 + 0.05 * r.uniform(-1, 1) for _ in range(6)],
             [0.2 + 0.02 * r.uniform(-1, 1) for _ in range(6)],
             [-0.1 + 0.02 * r.uniform(-1, 1) for _ in range(6)],
             [0.05 + 0.02 * r.uniform(-1, 1) for _ in range(6)],
             [0.5 + 0.05 * r.uniform(-1, 1) for _ in range(6)],
             [0.3 + 0.02 * r.uniform(-1, 1) for _ in range(6)],
             [0.1 + 0.02 * r.uniform(-1, 1) for _ in range(6)],
             [-0.2 + 0.02 * r.uniform(-1, 1) for _ in range(6)]]]
    met = [Num(x) for x in (0.8, 0.05, -0.02, 0.01, 1.3, 0.02, 0.01, 1.25, -0.03, 1.35)]
    return prim, met


def count():
    """Operation counts of one cell's RHS and stage update (curved metric,
    WENO5): returns a dict with the per-part and total counts."""
    prim, met = _state()
    gamma, eps = 5.0 / 3.0, 1e-6
    out = {}
    reset()
    F = face_flux(prim, met, met, 0, gamma, eps)
    out["face"] = dict(COUNTS, total=total())
    reset()
    for q in range(8):
        weno5(*prim[q][:5], eps)
    out["weno5_one_value"] = total() // 8
    reset()
    dmet = [[fd4([met[c], met[c], met[c], met[c]], Num(1.0)) for c in range(10)] for _ in range(3)]
    out["fd4_metric_derivatives"] = total()
    reset()
    src = source([p[2] for p in prim], met, dmet, [Num(0.01)] * 6, gamma)
    out["source"] = total()
    reset()
    L = cell_rhs([F, F, F], [F, F, F], src, [Num(1.0)] * 3)
    out["divergence"] = total()
    reset()
    stage([Num(1.0)] * 8, [Num(1.0)] * 8, L, 0.75, 0.25, Num(0.1))
    out["stage_update"] = total()
    out["cell_total"] = (3 * out["face"]["total"] + out["fd4_metric_derivatives"] + out["source"]
                         + out["divergence"] + out["stage_update"])
    return out


def main(path=None):
    here = os.path.dirname(os.path.abspath(__file__))
    path = path or os.path.join(os.path.dirname(here), "paper_2210_17509_gb300", "flop_counts.json")
    c = count()
    doc = {
        "what": "FP64 operations per interior cell of one RHS evaluation with the RK stage update, curved "
                "metric, WENO5 + HLLE, each face counted once (3 per cell); +, -, *, /, sqrt, min, max = 1",
        "generator": "python -m oracle.flop_count",
        "rhs_curved_weno5_per_cell": c["cell_total"],
        "parts": c,
    }
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    return doc


if __name__ == "__main__":
    print(json.dumps(main()["parts"], indent=1))
