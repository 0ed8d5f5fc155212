"""Plain FP64 CPU oracle for the GRMHD method-of-lines hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path (the CUDA library
and its binding) never imports, links or runs anything here.

The numerics live in ``grmhd_oracle.cpp`` (see its header for the paper
passages each routine follows).  This module only compiles it with the host
compiler and marshals numpy arrays through ``ctypes``.

Array layout (shared with the CUDA library only as a data format): SoA
``[var][z][y][x]`` float64, x fastest, ``N = n + 2*ng`` points per axis.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grmhd_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

REC_MINMOD, REC_WENO5 = 0, 1
BC_PERIODIC, BC_COPY = 0, 1
EOS_IDEAL, EOS_POLYTROPE = 0, 1
RK2, RK3, RK4 = 2, 3, 4


class OParams(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("recon", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("rho_atm", ctypes.c_double),
        ("p_atm", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("eos", ctypes.c_int32),
        ("poly_K", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (g++ -O2 -fopenmp)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        Dd = ctypes.c_double
        pp = ctypes.POINTER(OParams)
        lib.oracle_num_threads.restype = I
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_prim2con.argtypes = [P, I, P, Dd, P, P, P]
        lib.oracle_prim2con_eos.argtypes = [P, I, P, pp, P, P, P]
        lib.oracle_con2prim.argtypes = [P, I, P, pp, P, P, P, P]
        lib.oracle_con2prim.restype = I
        lib.oracle_fill_ghosts.argtypes = [P, I, I, I, P]
        lib.oracle_rhs.argtypes = [P, I, P, pp, P, P, P, P]
        lib.oracle_rhs_cells.argtypes = [P, I, P, pp, P, P, P, ctypes.c_long, P, P]
        lib.oracle_source_cells.argtypes = [P, I, P, pp, P, P, P, ctypes.c_long, P, P]
        lib.oracle_rk_step.argtypes = [P, I, P, pp, I, Dd, P, P, P, P, P]
        lib.oracle_rk_step.restype = I
        lib.oracle_point.argtypes = [P, P, Dd, P, P, P, P]
        lib.oracle_hlle.argtypes = [P, P, P, Dd, I, P, P]
        lib.oracle_reconstruct_1d.argtypes = [I, Dd, I, P, P, P]
        lib.oracle_con2prim_point.argtypes = [P, P, pp, P]
        lib.oracle_con2prim_point.restype = I
        lib.oracle_loss_jvp.argtypes = [P, I, P, pp, I, Dd, I, P, P, Dd, P, P, P, P]
        lib.oracle_loss_jvp.restype = I
        lib.oracle_con2prim_nh_point.argtypes = [P, pp, Dd, P]
        lib.oracle_con2prim_nh_point.restype = I
        lib.oracle_ct_rate.argtypes = [P, I, P, pp, P, P, P]
        lib.oracle_ct_divergence.argtypes = [P, I, P, P, P]
        lib.oracle_ct_rk_step.argtypes = [P, I, P, pp, I, Dd, P, P, P, P]
        lib.oracle_ct_rk_step.restype = I
        lib.oracle_restrict.argtypes = [P, I, P, P, P, I, P, P, P, I]
        lib.oracle_prolongate.argtypes = [P, I, P, P, P, I, P, P, P, I, I]
        lib.oracle_reflux.argtypes = [P, I, P, pp, P, P, P, I, P, P, P, P, Dd, P]
        lib.oracle_amr2_step.argtypes = [P, I, P, pp, I, Dd, P, P, P, I, P, P, P, P, P, P]
        lib.oracle_amr2_step.restype = I
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(gamma=5.0 / 3.0, recon=REC_WENO5, bc=BC_PERIODIC, rho_atm=1e-10, p_atm=None, weno_eps=1e-6,
                eos=None, poly_K=0.0):
    """eos: EOS_IDEAL (Gamma-law, default) or EOS_POLYTROPE with P = poly_K rho^gamma (reading R20)."""
    if p_atm is None:
        p_atm = 1e-2 * rho_atm ** gamma
    return OParams(gamma, recon, bc, rho_atm, p_atm, weno_eps, EOS_IDEAL if eos is None else eos, poly_K)


class Grid:
    """Interior extent n (x, y, z), ghost width ng, spacing dx (x, y, z)."""

    def __init__(self, n, ng, dx):
        self.n = tuple(int(v) for v in n)
        self.ng = int(ng)
        self.dx = tuple(float(v) for v in dx)
        self._n = (ctypes.c_int * 3)(*self.n)
        self._dx = (ctypes.c_double * 3)(*self.dx)

    @property
    def shape(self):
        nx, ny, nz = (v + 2 * self.ng for v in self.n)
        return (nz, ny, nx)

    def interior(self):
        g = self.ng
        nx, ny, nz = self.n
        return (slice(g, g + nz), slice(g, g + ny), slice(g, g + nx))


def threads() -> int:
    return _load().oracle_num_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def prim2con(grid: Grid, gamma: float, prim, metric=None, params: OParams = None):
    """prim -> cons; with params, under its EOS (the polytrope takes P = K rho^Gamma)."""
    prim = _f64(prim)
    metric = _f64(metric)
    cons = np.zeros_like(prim)
    if params is not None:
        _load().oracle_prim2con_eos(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(prim), _ptr(metric),
                                    _ptr(cons))
    else:
        _load().oracle_prim2con(grid._n, grid.ng, grid._dx, gamma, _ptr(prim), _ptr(metric), _ptr(cons))
    return cons


def con2prim(grid: Grid, params: OParams, cons, metric=None, prim_init=None):
    """Recover primitives on the interior; ghost entries copied from prim_init."""
    cons = _f64(cons)
    metric = _f64(metric)
    prim = np.zeros_like(cons) if prim_init is None else np.array(prim_init, dtype=np.float64, copy=True)
    status = np.zeros(grid.shape, dtype=np.int8)
    nfail = _load().oracle_con2prim(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(cons),
                                    _ptr(metric), _ptr(prim), _ptr(status))
    return prim, status, nfail


def fill_ghosts(grid: Grid, bc: int, arr):
    arr = np.array(arr, dtype=np.float64, copy=True, order="C")
    nvar = arr.shape[0]
    _load().oracle_fill_ghosts(grid._n, grid.ng, bc, nvar, _ptr(arr))
    return arr


def rhs(grid: Grid, params: OParams, prim, metric=None, kij=None):
    prim = _f64(prim)
    metric = _f64(metric)
    kij = _f64(kij)
    out = np.zeros_like(prim)
    _load().oracle_rhs(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(prim), _ptr(metric),
                       _ptr(kij), _ptr(out))
    return out


def rhs_cells(grid: Grid, params: OParams, prim, cells, metric=None, kij=None):
    """RHS at selected cells; ``cells`` is an (m, 3) int array of (i, j, k) full-array indices."""
    prim = _f64(prim)
    metric = _f64(metric)
    kij = _f64(kij)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros((cells.shape[0], 8), dtype=np.float64)
    _load().oracle_rhs_cells(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(prim), _ptr(metric),
                             _ptr(kij), cells.shape[0], _ptr(cells), _ptr(out))
    return out


def source_cells(grid: Grid, params: OParams, prim, cells, metric=None, kij=None):
    """Eq. 13 source vector at selected (i, j, k) cells, shape (m, 8)."""
    prim = _f64(prim)
    metric = _f64(metric)
    kij = _f64(kij)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros((cells.shape[0], 8), dtype=np.float64)
    _load().oracle_source_cells(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(prim), _ptr(metric),
                                _ptr(kij), cells.shape[0], _ptr(cells), _ptr(out))
    return out


def rk_step(grid: Grid, params: OParams, scheme: int, dt: float, cons, prim, metric=None, kij=None):
    cons = np.array(cons, dtype=np.float64, copy=True)
    prim = np.array(prim, dtype=np.float64, copy=True)
    metric = _f64(metric)
    kij = _f64(kij)
    status = np.zeros(grid.shape, dtype=np.int8)
    nfail = _load().oracle_rk_step(grid._n, grid.ng, grid._dx, ctypes.byref(params), scheme, dt, _ptr(cons),
                                   _ptr(prim), _ptr(metric), _ptr(kij), _ptr(status))
    return cons, prim, nfail


def point(prim8, gamma, adm10=None):
    """Conserved vector, fluxes F[d][8], speeds lam[d][(minus, plus)], extras (W, b^2, b.u, u.u)."""
    p = _f64(np.asarray(prim8).reshape(8))
    a = None if adm10 is None else _f64(np.asarray(adm10).reshape(10))
    U = np.zeros(8)
    F = np.zeros((3, 8))
    lam = np.zeros((3, 2))
    ex = np.zeros(4)
    _load().oracle_point(_ptr(p), _ptr(a), gamma, _ptr(U), _ptr(F), _ptr(lam), _ptr(ex))
    return U, F, lam, ex


def hlle(pL, pR, gamma, direction, adm10=None):
    pL = _f64(np.asarray(pL).reshape(8))
    pR = _f64(np.asarray(pR).reshape(8))
    a = None if adm10 is None else _f64(np.asarray(adm10).reshape(10))
    F = np.zeros(8)
    sp = np.zeros(4)
    _load().oracle_hlle(_ptr(pL), _ptr(pR), _ptr(a), gamma, int(direction), _ptr(F), _ptr(sp))
    return F, sp


def reconstruct_1d(recon: int, u, eps=1e-6):
    """Face states for faces between cells c-1 and c, c = 3 .. n-3 (NaN elsewhere)."""
    u = _f64(np.asarray(u).ravel())
    n = u.size
    uL = np.full(n, np.nan)
    uR = np.full(n, np.nan)
    _load().oracle_reconstruct_1d(recon, eps, n, _ptr(u), _ptr(uL), _ptr(uR))
    return uL, uR


def con2prim_point(U8, params: OParams, adm10=None):
    U = _f64(np.asarray(U8).reshape(8))
    a = None if adm10 is None else _f64(np.asarray(adm10).reshape(10))
    out = np.zeros(8)
    st = _load().oracle_con2prim_point(_ptr(U), _ptr(a), ctypes.byref(params), _ptr(out))
    return out, st


def con2prim_nh_point(U8, params: OParams, P0):
    """Newman-Hamlin recovery of one flat-space state (reading R18); (prim, status 0 ok / 1 failed)."""
    U = _f64(np.asarray(U8).reshape(8))
    out = np.zeros(8)
    st = _load().oracle_con2prim_nh_point(_ptr(U), ctypes.byref(params), float(P0), _ptr(out))
    return out, st


def loss_jvp(grid: Grid, params: OParams, scheme: int, dt: float, nsteps: int, prim0, dprim0=None, dgamma=0.0,
             metric=None, kij=None):
    """Value and directional derivative of L = sum rho^2 sqrt(gamma) dV after nsteps."""
    prim0 = _f64(prim0)
    dprim0 = _f64(dprim0)
    metric = _f64(metric)
    kij = _f64(kij)
    L = ctypes.c_double()
    dL = ctypes.c_double()
    nfail = _load().oracle_loss_jvp(grid._n, grid.ng, grid._dx, ctypes.byref(params), scheme, dt, nsteps,
                                    _ptr(prim0), _ptr(dprim0), float(dgamma), _ptr(metric), _ptr(kij),
                                    ctypes.byref(L), ctypes.byref(dL))
    return L.value, dL.value, nfail


# ------------------------------------------- two-level AMR transfer (R14-R17) --
def _lo(lo):
    return (ctypes.c_int * 3)(*[int(v) for v in lo])


def restrict(coarse_grid: Grid, coarse, fine_grid: Grid, fine, lo):
    """Covered coarse cells := mean of their 8 fine children (R14); returns a new coarse array."""
    coarse = np.array(coarse, dtype=np.float64, copy=True)
    fine = _f64(fine)
    _load().oracle_restrict(coarse_grid._n, coarse_grid.ng, coarse_grid._dx, _ptr(coarse), fine_grid._n,
                            fine_grid.ng, fine_grid._dx, _ptr(fine), _lo(lo), coarse.shape[0])
    return coarse


def prolongate(coarse_grid: Grid, coarse, fine_grid: Grid, fine, lo, ghosts_only=True):
    """Fine points (ghosts only, or all) from the coarse parents, limited-linear (R15)."""
    coarse = _f64(coarse)
    fine = np.array(fine, dtype=np.float64, copy=True)
    _load().oracle_prolongate(coarse_grid._n, coarse_grid.ng, coarse_grid._dx, _ptr(coarse), fine_grid._n,
                              fine_grid.ng, fine_grid._dx, _ptr(fine), _lo(lo), fine.shape[0], int(ghosts_only))
    return fine


def reflux(coarse_grid: Grid, params: OParams, coarse_prim, fine_grid: Grid, fine_prim, lo, scale=1.0, out=None,
           coarse_metric=None, fine_metric=None):
    """Adds scale * (coarse RHS change from flux restriction, R16) to out (zeros if None)."""
    cp = _f64(coarse_prim)
    fp = _f64(fine_prim)
    out = np.zeros_like(cp) if out is None else np.array(out, dtype=np.float64, copy=True)
    _load().oracle_reflux(coarse_grid._n, coarse_grid.ng, coarse_grid._dx, ctypes.byref(params), _ptr(cp),
                          _ptr(_f64(coarse_metric)), fine_grid._n, fine_grid.ng, fine_grid._dx, _ptr(fp),
                          _ptr(_f64(fine_metric)), _lo(lo), float(scale), _ptr(out))
    return out


def amr2_step(coarse_grid: Grid, params: OParams, scheme: int, dt: float, ccons, cprim, fine_grids, fcons, fprim,
              los, coarse_metric=None, fine_metrics=None):
    """One composite step (R17) of a coarse block and its fine blocks; returns
    (ccons, cprim, [fcons], [fprim], nfail)."""
    nf = len(fine_grids)
    ccons = np.array(ccons, dtype=np.float64, copy=True)
    cprim = np.array(cprim, dtype=np.float64, copy=True)
    fcons = [np.array(a, dtype=np.float64, copy=True) for a in fcons]
    fprim = [np.array(a, dtype=np.float64, copy=True) for a in fprim]
    fmet = [None] * nf if fine_metrics is None else [_f64(m) for m in fine_metrics]
    fn = (ctypes.c_int * (3 * nf))(*[v for g in fine_grids for v in g.n])
    fdx = (ctypes.c_double * (3 * nf))(*[v for g in fine_grids for v in g.dx])
    lo = (ctypes.c_int * (3 * nf))(*[int(v) for l in los for v in l])
    P = ctypes.c_void_p
    pc = (P * nf)(*[a.ctypes.data for a in fcons])
    pp_ = (P * nf)(*[a.ctypes.data for a in fprim])
    pm = (P * nf)(*[None if m is None else m.ctypes.data for m in fmet])
    for g in fine_grids:
        assert g.ng == coarse_grid.ng
    nfail = _load().oracle_amr2_step(coarse_grid._n, coarse_grid.ng, coarse_grid._dx, ctypes.byref(params),
                                     int(scheme), float(dt), _ptr(ccons), _ptr(cprim), _ptr(_f64(coarse_metric)),
                                     nf, fn, fdx, pc, pp_, pm, lo)
    return ccons, cprim, fcons, fprim, nfail


# ------------------------------------------ constrained transport (R19) --
def ct_rate(grid: Grid, params: OParams, prim, metric=None):
    """Rate of change of the face field (3 x ncell): minus the discrete curl of the edge field."""
    prim = _f64(prim)
    out = np.zeros((3,) + grid.shape)
    _load().oracle_ct_rate(grid._n, grid.ng, grid._dx, ctypes.byref(params), _ptr(prim), _ptr(_f64(metric)),
                           _ptr(out))
    return out


def ct_divergence(grid: Grid, bface):
    bface = _f64(bface)
    out = np.zeros(grid.shape)
    _load().oracle_ct_divergence(grid._n, grid.ng, grid._dx, _ptr(bface), _ptr(out))
    return out


def ct_rk_step(grid: Grid, params: OParams, scheme: int, dt: float, cons, prim, bface, metric=None):
    """One step with constrained transport (R19); returns (cons, prim, bface, nfail)."""
    cons = np.array(cons, dtype=np.float64, copy=True)
    prim = np.array(prim, dtype=np.float64, copy=True)
    bface = np.array(bface, dtype=np.float64, copy=True)
    nfail = _load().oracle_ct_rk_step(grid._n, grid.ng, grid._dx, ctypes.byref(params), int(scheme), float(dt),
                                      _ptr(cons), _ptr(prim), _ptr(bface), _ptr(_f64(metric)))
    return cons, prim, bface, nfail



def ct_cell_field(prim, bface, metric=None):
    """Primitives whose field is the cell mean of the face field divided by
    sqrt(gamma) of the cell (reading R19: the cell-centred densitised field is
    the mean of a cell's two faces), for every cell, ghosts included, that has
    both of its faces in the array; the other entries keep ``prim``."""
    prim = np.array(prim, dtype=np.float64, copy=True)
    sg = np.ones(prim.shape[1:])
    if metric is not None:
        g = metric
        det = (g[4] * (g[7] * g[9] - g[8] * g[8]) - g[5] * (g[5] * g[9] - g[8] * g[6])
               + g[6] * (g[5] * g[8] - g[7] * g[6]))
        sg = np.sqrt(det)
    for a in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[2 - a] = slice(0, -1)
        hi[2 - a] = slice(1, None)
        cell = 0.5 * (bface[a][tuple(lo)] + bface[a][tuple(hi)])
        prim[5 + a][tuple(lo)] = cell / sg[tuple(lo)]
    return prim
