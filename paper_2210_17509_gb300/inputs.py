"""Seeded synthetic inputs for the GRMHD hot path.

This module holds no arithmetic of the method itself: it only draws random
smooth fields, samples the closed-form Schwarzschild metric in isotropic
coordinates and lays the results out in the library's array format.  Both
the CUDA path and the CPU oracle are fed from here.

Layout: SoA ``[var][z][y][x]`` float64, x fastest, ``N = n + 2*ng``.
Primitives ``[rho, v^x, v^y, v^z, P, B^x, B^y, B^z]`` (Valencia 3-velocity
v^i, Eulerian field B^i); metric ``[alpha, beta^x, beta^y, beta^z, g_xx,
g_xy, g_xz, g_yy, g_yz, g_zz]`` at cell centres, ghosts included.

Workloads (shapes follow the paper's test and benchmark setups, Secs. 4-5):
  * ``smooth_flat``: periodic block, Minkowski; rho = 1 + 0.2 * (sum of 4
    random Fourier modes normalised to max 1); P = 0.1 rho^Gamma; v^i from
    3 random-mode fields scaled to |v| <= 0.5; B = curl A, A random modes of
    amplitude 0.1 (analytic curl, divergence free).
  * ``smooth_schwarzschild``: same generator on a block spanning [4, 12]^3 M
    around a Schwarzschild mass M = 1, rho mapped into [1e-3, 1], |v| <= 0.5
    measured with the spatial metric.
  * ``riemann_schwarzschild``: planar jump along x at the block centre,
    left (rho, P) = (1, 1), right (0.125, 0.1), B^x = 0.5, B^y = +1 | -1,
    1% seeded multiplicative perturbation of rho and P.
  * ``amr_boxes``: 512 boxes, edges from {8, 16, 24, 32, 48, 64} per axis,
    refinement level 0/1/2 round-robin (dx = 1, 1/2, 1/4), smooth_flat data.
  * ``shocktube``: the 1D MHD shock tubes of Sec. 4.1 (Balsara tests 1-5,
    the paper's table of left / right states) along x, y or z, Minkowski,
    with a few transverse cells; the table gives eps, laid out here as the
    primitive pressure P = (Gamma - 1) rho eps of the Gamma-law EOS.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NG = 3
GAMMA = 5.0 / 3.0


@dataclass
class Block:
    n: tuple          # interior cells (nx, ny, nz)
    ng: int
    dx: tuple         # (dx, dy, dz)
    origin: tuple     # coordinate of the lower interior face (x0, y0, z0)

    @property
    def shape(self):
        nx, ny, nz = (v + 2 * self.ng for v in self.n)
        return (nz, ny, nx)

    def centres(self):
        """Cell-centre coordinates of every point (ghosts included) as 3 arrays [z][y][x]."""
        ax = []
        for d in range(3):
            i = np.arange(self.n[d] + 2 * self.ng, dtype=np.float64)
            ax.append(self.origin[d] + (i - self.ng + 0.5) * self.dx[d])
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z

    def interior(self):
        g = self.ng
        nx, ny, nz = self.n
        return (slice(g, g + nz), slice(g, g + ny), slice(g, g + nx))

    @property
    def ncells(self):
        return self.n[0] * self.n[1] * self.n[2]


def _modes(rng, nmodes, kmax=4):
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(k != 0):
            ks.append(k.astype(np.float64))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
    amp = rng.uniform(0.5, 1.0, size=nmodes)
    return ks, ph, amp


def _mode_field(blk, x, y, z, ks, ph, amp):
    L = [blk.n[d] * blk.dx[d] for d in range(3)]
    f = np.zeros_like(x)
    for k, p, a in zip(ks, ph, amp):
        arg = 2 * math.pi * (k[0] * (x - blk.origin[0]) / L[0] + k[1] * (y - blk.origin[1]) / L[1]
                             + k[2] * (z - blk.origin[2]) / L[2]) + p
        f += a * np.sin(arg)
    return f


def _curl_of_modes(blk, x, y, z, rng, amp_total, nmodes=4):
    """Analytic curl of a random-mode vector potential A (div B = 0 exactly)."""
    L = [blk.n[d] * blk.dx[d] for d in range(3)]
    B = [np.zeros_like(x) for _ in range(3)]
    for _ in range(nmodes):
        k = np.zeros(3)
        while not np.any(k != 0):
            k = rng.integers(-4, 5, size=3).astype(np.float64)
        a = rng.normal(size=3)
        a *= amp_total / np.linalg.norm(a)
        p = rng.uniform(0, 2 * math.pi)
        kk = np.array([2 * math.pi * k[d] / L[d] for d in range(3)])
        arg = kk[0] * (x - blk.origin[0]) + kk[1] * (y - blk.origin[1]) + kk[2] * (z - blk.origin[2]) + p
        c = np.cos(arg)
        # A = a sin(arg): curl A = (k x a) cos(arg)
        kxa = np.cross(kk, a)
        for d in range(3):
            B[d] += kxa[d] * c
    # scale so that max |A| ~ amp_total corresponds to |B| of order amp_total * |k|
    return B


def flat_metric():
    """Minkowski space is passed to the library as a NULL metric."""
    return None


def schwarzschild_metric(blk: Block, M: float = 1.0):
    """alpha, beta = 0, gamma_ij = psi^4 delta_ij, psi = 1 + M / (2 r) (isotropic)."""
    x, y, z = blk.centres()
    r = np.sqrt(x * x + y * y + z * z)
    psi = 1.0 + M / (2.0 * r)
    alpha = (1.0 - M / (2.0 * r)) / (1.0 + M / (2.0 * r))
    m = np.zeros((10,) + blk.shape)
    m[0] = alpha
    p4 = psi ** 4
    m[4] = p4
    m[7] = p4
    m[9] = p4
    return m


def _conformal_factor(metric):
    if metric is None:
        return None
    return metric[4] ** 0.25  # psi for a conformally flat gamma_ij


def smooth_prims(blk: Block, seed: int, gamma: float = GAMMA, rho_range=None, metric=None,
                 vmax=0.5, b_amp=0.1):
    rng = np.random.Generator(np.random.Philox(seed))
    x, y, z = blk.centres()
    inner = blk.interior()
    ks, ph, amp = _modes(rng, 4)
    f = _mode_field(blk, x, y, z, ks, ph, amp)
    if rho_range is None:
        f = f / np.max(np.abs(f[inner]))
        rho = 1.0 + 0.2 * f
    else:
        lo, hi = rho_range
        fi = f[inner]
        rho = lo + (hi - lo) * (f - fi.min()) / (fi.max() - fi.min())
        rho = np.maximum(rho, 0.5 * lo)
    P = 0.1 * rho ** gamma
    v = []
    for _ in range(3):
        ks, ph, amp = _modes(rng, 3)
        v.append(_mode_field(blk, x, y, z, ks, ph, amp))
    vmag = np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    scale = vmax / np.max(vmag[inner])
    v = [c * scale for c in v]
    psi = _conformal_factor(metric)
    if psi is not None:
        v = [c / psi ** 2 for c in v]
    B = _curl_of_modes(blk, x, y, z, rng, b_amp)
    bmag = np.sqrt(B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    bscale = b_amp / np.max(bmag[inner])
    B = [c * bscale for c in B]
    prim = np.stack([rho, v[0], v[1], v[2], P, B[0], B[1], B[2]])
    return np.ascontiguousarray(prim)


def riemann_prims(blk: Block, seed: int, perturb: float = 0.01):
    rng = np.random.Generator(np.random.Philox(seed))
    x, _, _ = blk.centres()
    xm = blk.origin[0] + 0.5 * blk.n[0] * blk.dx[0]
    left = x < xm
    rho = np.where(left, 1.0, 0.125)
    P = np.where(left, 1.0, 0.1)
    rho = rho * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=rho.shape))
    P = P * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=P.shape))
    zero = np.zeros_like(rho)
    Bx = np.full_like(rho, 0.5)
    By = np.where(left, 1.0, -1.0)
    prim = np.stack([rho, zero, zero, zero, P, Bx, By, zero.copy()])
    return np.ascontiguousarray(prim)


# ------------------------------------------------------------- workloads --
def smooth_flat(n=32, seed=0, gamma=GAMMA, ng=NG):
    blk = Block((n, n, n), ng, (1.0 / n,) * 3, (0.0, 0.0, 0.0))
    return blk, smooth_prims(blk, seed, gamma), flat_metric()


def smooth_schwarzschild(n=128, seed=1, gamma=GAMMA, ng=NG):
    h = 8.0 / n
    blk = Block((n, n, n), ng, (h, h, h), (4.0, 4.0, 4.0))
    metric = schwarzschild_metric(blk)
    return blk, smooth_prims(blk, seed, gamma, rho_range=(1e-3, 1.0), metric=metric), metric


def riemann_schwarzschild(n=256, seed=4, ng=NG):
    h = 8.0 / n
    blk = Block((n, n, n), ng, (h, h, h), (4.0, 4.0, 4.0))
    metric = schwarzschild_metric(blk)
    return blk, riemann_prims(blk, seed), metric


def window(blk: Block, arr, lo, m):
    """The m^3 sub-block of blk whose interior starts at interior cell lo
    (x, y, z), with ng ghost layers taken from arr's neighbouring points: its
    Block (same spacing, shifted origin) and a copy of arr's values there."""
    g = blk.ng
    for d in range(3):
        if not (0 <= lo[d] and lo[d] + m <= blk.n[d]):
            raise ValueError("window outside the block interior")
    wblk = Block((m, m, m), g, blk.dx, tuple(blk.origin[d] + lo[d] * blk.dx[d] for d in range(3)))
    sl = (slice(None),) + tuple(slice(lo[d], lo[d] + m + 2 * g) for d in (2, 1, 0))
    return wblk, np.ascontiguousarray(arr[sl])


EDGES = (8, 16, 24, 32, 48, 64)


def amr_box_shapes(nbox=512, seed=2):
    rng = np.random.Generator(np.random.Philox(seed))
    shapes = rng.choice(np.array(EDGES), size=(nbox, 3))
    levels = np.arange(nbox) % 3
    return [(tuple(int(v) for v in s), int(l)) for s, l in zip(shapes, levels)]


def amr_boxes(nbox=512, seed=2, gamma=GAMMA, ng=NG, max_boxes=None):
    """List of (Block, prim) for the batched workload (flat metric)."""
    out = []
    for b, (shape, lev) in enumerate(amr_box_shapes(nbox, seed)):
        if max_boxes is not None and b >= max_boxes:
            break
        h = 1.0 / (2 ** lev)
        blk = Block(shape, ng, (h, h, h), (0.0, 0.0, 0.0))
        out.append((blk, smooth_prims(blk, 1000 + b, gamma)))
    return out


def cfl_dt(blk: Block, cfl: float) -> float:
    """dt = CFL * min dx (the paper's CFL definition, Sec. 4.1)."""
    return cfl * min(blk.dx)


# 1D shock tubes of Sec. 4.1 (the paper's table of Balsara tests 1-5): per
# test the normal field B^x, Gamma, the end time t_ref, and the left / right
# states (rho, eps, (v^x, v^y, v^z), (B^y, B^z)); left is x < 0 on [-0.5, 0.5].
BALSARA = {
    1: dict(Bx=0.5, gamma=2.0, t_ref=0.4,
            left=(1.0, 1.0, (0.0, 0.0, 0.0), (1.0, 0.0)),
            right=(0.125, 0.8, (0.0, 0.0, 0.0), (-1.0, 0.0))),
    2: dict(Bx=5.0, gamma=5.0 / 3.0, t_ref=0.4,
            left=(1.0, 45.0, (0.0, 0.0, 0.0), (6.0, 6.0)),
            right=(1.0, 1.5, (0.0, 0.0, 0.0), (0.7, 0.7))),
    3: dict(Bx=10.0, gamma=5.0 / 3.0, t_ref=0.4,
            left=(1.0, 1500.0, (0.0, 0.0, 0.0), (7.0, 7.0)),
            right=(1.0, 0.15, (0.0, 0.0, 0.0), (0.7, 0.7))),
    4: dict(Bx=10.0, gamma=5.0 / 3.0, t_ref=0.4,
            left=(1.0, 0.15, (0.999, 0.0, 0.0), (7.0, 7.0)),
            right=(1.0, 0.15, (-0.999, 0.0, 0.0), (-7.0, -7.0))),
    5: dict(Bx=2.0, gamma=5.0 / 3.0, t_ref=0.55,
            left=(1.08, 1.3194, (0.4, 0.3, 0.2), (0.3, 0.3)),
            right=(1.0, 1.5, (-0.45, -0.2, 0.2), (-0.7, 0.5))),
}


def shocktube(test: int, n: int = 1600, axis: int = 0, transverse: int = 8, ng: int = NG):
    """Balsara shock tube ``test`` along ``axis``: n cells of width 1/n on
    [-0.5, 0.5] along the axis, ``transverse`` cells of the same width across
    it, Minkowski.  The table's x components (v, B) lie along ``axis`` and
    its y, z components along the next two axes in cyclic order, so the
    three orientations are relabellings of one another.  Ghosts are filled
    by copying the nearest interior cell (the tests' boundary, Sec. 4.1).
    Returns (Block, prim, gamma, t_ref)."""
    t = BALSARA[test]
    nv = [transverse, transverse, transverse]
    nv[axis] = n
    origin = [0.0, 0.0, 0.0]
    origin[axis] = -0.5
    blk = Block(tuple(nv), ng, (1.0 / n,) * 3, tuple(origin))
    coords = blk.centres()
    left = coords[axis] < 0.0
    prim = np.zeros((8,) + blk.shape)
    for state, mask in ((t["left"], left), (t["right"], ~left)):
        rho, eps, v, byz = state
        comp_v = (v[0], v[1], v[2])
        comp_b = (t["Bx"], byz[0], byz[1])
        prim[0][mask] = rho
        prim[4][mask] = (t["gamma"] - 1.0) * rho * eps
        for k in range(3):
            d = (axis + k) % 3
            prim[1 + d][mask] = comp_v[k]
            prim[5 + d][mask] = comp_b[k]
    return blk, prim, t["gamma"], t["t_ref"]



def edge_potential(blk: Block, seed: int, shift=(0.0, 0.0, 0.0), nmodes=4):
    """Random-mode vector potential sampled on cell edges: component c at
    the c-edge through the corner of each cell that is lower in the other
    two axes, shape [3][z][y][x].  `shift` displaces the pattern (the
    potential at x is the pattern at x - shift), for advected references."""
    rng = np.random.default_rng(np.random.Philox(seed))
    modes = [_modes(rng, nmodes) for _ in range(3)]
    xc, yc, zc = blk.centres()
    A = np.zeros((3,) + blk.shape)
    for c in range(3):
        pos = [xc, yc, zc]
        for e in range(3):
            if e != c:
                pos[e] = pos[e] - 0.5 * blk.dx[e]
        ks, ph, amp = modes[c]
        A[c] = _mode_field(blk, pos[0] - shift[0], pos[1] - shift[1], pos[2] - shift[2], ks, ph, amp)
    return A


def face_curl(blk: Block, A):
    """Densitised face field as the discrete curl of an edge potential:
    component a on the lower a-face of each cell,
    B^a = (A_c[+e_b] - A_c) / dx_b - (A_b[+e_c] - A_b) / dx_c, (a, b, c)
    cyclic (entries whose stencil leaves the array are 0).  Its discrete
    divergence vanishes identically."""
    B = np.zeros_like(A)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        # array axes are (z, y, x): coordinate axis e is array axis 3 - e of A[.] (axis 2 - e of a field)
        Ac, Ab = A[c], A[b]
        dAc = np.zeros_like(Ac)
        dAb = np.zeros_like(Ab)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[2 - b] = slice(0, -1)
        sl_hi[2 - b] = slice(1, None)
        dAc[tuple(sl_lo)] = (Ac[tuple(sl_hi)] - Ac[tuple(sl_lo)]) / blk.dx[b]
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[2 - c] = slice(0, -1)
        sl_hi[2 - c] = slice(1, None)
        dAb[tuple(sl_lo)] = (Ab[tuple(sl_hi)] - Ab[tuple(sl_lo)]) / blk.dx[c]
        B[a] = dAc - dAb
    return B


def polytrope_prims(blk: Block, seed: int, K: float, gamma: float, metric=None, vmax=0.9, log_rho=(-4.0, -2.5),
                    b_scale=1.0):
    """Random magnetised states on the polytrope P = K rho^gamma: log10 rho
    uniform in log_rho, |v| uniform in [0, vmax) (lengths taken in the metric
    when given, for isotropic metrics), B normal with scale b_scale sqrt(rho)
    (so b^2/rho of order b_scale^2)."""
    rng = np.random.default_rng(np.random.Philox(seed))
    shp = blk.shape
    prim = np.zeros((8,) + shp)
    prim[0] = 10 ** rng.uniform(log_rho[0], log_rho[1], shp)
    v = rng.normal(size=(3,) + shp)
    vmag = rng.uniform(0, vmax, shp)
    psi4 = metric[4] if metric is not None else 1.0
    prim[1:4] = v / np.sqrt((v ** 2).sum(0)) * vmag / np.sqrt(psi4)
    prim[4] = K * prim[0] ** gamma
    prim[5:] = b_scale * rng.normal(size=(3,) + shp) * np.sqrt(prim[0])
    return prim
