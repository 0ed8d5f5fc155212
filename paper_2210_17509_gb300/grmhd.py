"""Thin Python binding of libgrmhd.so (the C ABI declared in include/grmhd.h).

Argument marshalling only: every function checks the tensors it is given
(CUDA, float64, contiguous, expected shape), passes raw device pointers and
the current torch stream to the C entry point of the same name, and raises
``GrmhdError`` on a non-zero return code.  All arithmetic runs in the CUDA
kernels of the library.  Importing this module fails loudly when the
library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgrmhd.so")

MINMOD, WENO5 = 0, 1
BC_PERIODIC, BC_COPY = 0, 1
FP64, MIXED = 0, 1
RK2, RK3, RK4 = 2, 3, 4
REUSE_GEOMETRY = 1
NEWMAN_HAMLIN = 2
SINGLE_PASS = 4
DETERMINISTIC = 8
EOS_IDEAL, EOS_POLYTROPE = 0, 1


class GrmhdError(RuntimeError):
    pass


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libgrmhd.so not found at {LIB_PATH}; build it with "
        "`python -m paper_2210_17509_gb300.build` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)


class CGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("ng", ctypes.c_int32), ("dx", ctypes.c_double * 3)]


class CParams(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("recon", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("nr_maxit", ctypes.c_int32),
        ("rho_atm", ctypes.c_double),
        ("p_atm", ctypes.c_double),
        ("nr_tol", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("tile", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("eos", ctypes.c_int32),
        ("poly_K", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_pg = ctypes.POINTER(CGrid)
_pp = ctypes.POINTER(CParams)

_lib.grmhd_prim2con.argtypes = [_pg, _pp, _P, _P, _P, _P]
_lib.grmhd_con2prim.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, _P]
_lib.grmhd_fill_ghosts.argtypes = [_pg, _I32, _I32, _P, _P]
_lib.grmhd_rhs.argtypes = [_pg, _pp, _P, _P, _P, _P, _P]
_lib.grmhd_rk_workspace_bytes.argtypes = [_pg, _I32]
_lib.grmhd_rk_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_rk_workspace_bytes_cached.argtypes = [_pg, _I32]
_lib.grmhd_rk_workspace_bytes_cached.restype = ctypes.c_size_t
_lib.grmhd_rk_step.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P]
_lib.grmhd_rk_step_static.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _P, _P, _P]
_lib.grmhd_rk_step_static.restype = _I
_lib.grmhd_error_string.argtypes = [_I]
_lib.grmhd_error_string.restype = ctypes.c_char_p
_lib.grmhd_version.restype = _I
for _name in ("grmhd_prim2con", "grmhd_con2prim", "grmhd_fill_ghosts", "grmhd_rhs", "grmhd_rk_step"):
    getattr(_lib, _name).restype = _I

C_SYMBOLS = ("grmhd_prim2con", "grmhd_con2prim", "grmhd_fill_ghosts", "grmhd_rhs", "grmhd_rk_workspace_bytes",
             "grmhd_rk_workspace_bytes_cached", "grmhd_rk_step", "grmhd_rk_step_static", "grmhd_error_string", "grmhd_version")
STATIC_SCRATCH_BYTES = 64 << 20


@dataclass
class Grid:
    """Interior cells n = (nx, ny, nz), ghost width ng, spacing dx = (dx, dy, dz)."""
    n: tuple
    ng: int
    dx: tuple

    def c(self) -> CGrid:
        return CGrid((ctypes.c_int32 * 3)(*[int(v) for v in self.n]), int(self.ng),
                     (ctypes.c_double * 3)(*[float(v) for v in self.dx]))

    @property
    def shape(self):
        nx, ny, nz = (v + 2 * self.ng for v in self.n)
        return (nz, ny, nx)

    @property
    def ncell(self):
        nz, ny, nx = self.shape
        return nx * ny * nz


@dataclass
class Params:
    gamma: float = 5.0 / 3.0
    recon: int = WENO5
    bc: int = BC_PERIODIC
    precision: int = FP64
    nr_maxit: int = 50
    rho_atm: float = 1e-10
    p_atm: float = 1e-20
    nr_tol: float = 1e-12
    weno_eps: float = 1e-6
    tile: int = 0
    flags: int = 0
    eos: int = 0         # EOS_IDEAL | EOS_POLYTROPE
    poly_K: float = 0.0  # K of P = K rho^gamma (EOS_POLYTROPE)

    def c(self) -> CParams:
        return CParams(self.gamma, self.recon, self.bc, self.precision, self.nr_maxit, self.rho_atm, self.p_atm,
                       self.nr_tol, self.weno_eps, self.tile, self.flags, self.eos, self.poly_K)


def version() -> int:
    return _lib.grmhd_version()


def _check(rc: int, what: str):
    if rc != 0:
        raise GrmhdError(f"{what}: {_lib.grmhd_error_string(rc).decode()} ({rc})")


def _field(t, grid: Grid, ncomp: int, name: str, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != (ncomp,) + grid.shape:
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {(ncomp,) + grid.shape}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def prim2con(grid: Grid, params: Params, prim, metric=None, cons=None, stream=None):
    if cons is None:
        cons = torch.empty_like(prim)
    rc = _lib.grmhd_prim2con(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                             _field(metric, grid, 10, "metric", True), _field(cons, grid, 8, "cons"),
                             _stream(stream))
    _check(rc, "grmhd_prim2con")
    return cons


def con2prim(grid: Grid, params: Params, cons, prim, metric=None, status=None, nfail=None, stream=None):
    """In place on prim (guess in, result out)."""
    st = None
    if status is not None:
        if status.dtype != torch.int8 or tuple(status.shape) != grid.shape or not status.is_cuda:
            raise ValueError("status must be a CUDA int8 tensor of the block shape")
        st = ctypes.c_void_p(status.data_ptr())
    nf = None
    if nfail is not None:
        if nfail.dtype != torch.int32 or nfail.numel() < 1 or not nfail.is_cuda:
            raise ValueError("nfail must be a CUDA int32 tensor")
        nf = ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_con2prim(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(cons, grid, 8, "cons"),
                             _field(metric, grid, 10, "metric", True), _field(prim, grid, 8, "prim"), st, nf,
                             _stream(stream))
    _check(rc, "grmhd_con2prim")
    return prim


def fill_ghosts(grid: Grid, bc: int, field, stream=None):
    nvar = field.shape[0]
    rc = _lib.grmhd_fill_ghosts(ctypes.byref(grid.c()), bc, nvar, _field(field, grid, nvar, "field"),
                                _stream(stream))
    _check(rc, "grmhd_fill_ghosts")
    return field


def rhs(grid: Grid, params: Params, prim, metric=None, kij=None, out=None, stream=None):
    if out is None:
        out = torch.zeros_like(prim)
    rc = _lib.grmhd_rhs(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                        _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                        _field(out, grid, 8, "rhs"), _stream(stream))
    _check(rc, "grmhd_rhs")
    return out


_lib.grmhd_rhs_workspace_bytes.argtypes = [_pg]
_lib.grmhd_rhs_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_rhs_cached.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]
_lib.grmhd_rhs_cached.restype = _I
C_SYMBOLS = C_SYMBOLS + ("grmhd_rhs_workspace_bytes", "grmhd_rhs_cached")


def rhs_workspace(grid: Grid, device=None):
    nbytes = int(_lib.grmhd_rhs_workspace_bytes(ctypes.byref(grid.c())))
    if nbytes == 0:
        raise GrmhdError("invalid grid for the RHS workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def rhs_cached(grid: Grid, params: Params, prim, metric=None, kij=None, out=None, ws=None, stream=None):
    """grmhd_rhs_cached: the RHS from geometry caches kept in ws."""
    if out is None:
        out = torch.zeros_like(prim)
    if ws is None:
        ws = rhs_workspace(grid, prim.device)
    rc = _lib.grmhd_rhs_cached(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                               _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                               _field(out, grid, 8, "rhs"), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                               _stream(stream))
    _check(rc, "grmhd_rhs_cached")
    return out


def rk_workspace_bytes(grid: Grid, scheme: int) -> int:
    return int(_lib.grmhd_rk_workspace_bytes(ctypes.byref(grid.c()), scheme))


def rk_workspace_bytes_cached(grid: Grid, scheme: int) -> int:
    return int(_lib.grmhd_rk_workspace_bytes_cached(ctypes.byref(grid.c()), scheme))


def workspace(grid: Grid, scheme: int, device=None, cached: bool = True):
    """Device workspace for rk_step; by default large enough for the cached
    paths (geometry caches, FP32 primitive copy)."""
    nbytes = rk_workspace_bytes_cached(grid, scheme) if cached else rk_workspace_bytes(grid, scheme)
    if nbytes == 0:
        raise GrmhdError("invalid grid or scheme for the workspace")
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def rk_step(grid: Grid, params: Params, scheme: int, dt: float, cons, prim, metric=None, kij=None, ws=None,
            nfail=None, stream=None):
    """One step in place on cons and prim."""
    if ws is None:
        ws = workspace(grid, scheme, cons.device)
    nf = None
    if nfail is not None:
        nf = ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_rk_step(ctypes.byref(grid.c()), ctypes.byref(params.c()), scheme, float(dt),
                            _field(cons, grid, 8, "cons"), _field(prim, grid, 8, "prim"),
                            _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), nf, _stream(stream))
    _check(rc, "grmhd_rk_step")
    return cons, prim


def rk_step_static(grid: Grid, params: Params, scheme: int, dt: float, cons, prim, metric=None, kij=None,
                   nfail=None, stream=None):
    """grmhd_rk_step_static: one step in place, with no workspace argument.

    For callers that cannot allocate device memory; the library supplies the
    scratch from a fixed 64 MiB device array (blocks whose workspace would
    exceed it raise GrmhdError).  Overlapping calls on the GPU race on that
    array; the first call on a device should precede any stream capture."""
    nf = None
    if nfail is not None:
        nf = ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_rk_step_static(ctypes.byref(grid.c()), ctypes.byref(params.c()), scheme, float(dt),
                                   _field(cons, grid, 8, "cons"), _field(prim, grid, 8, "prim"),
                                   _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                                   nf, _stream(stream))
    _check(rc, "grmhd_rk_step_static")
    return cons, prim


# ------------------------------------------------------------ batched boxes --
class CBox(ctypes.Structure):
    _fields_ = [("grid", CGrid), ("cons", _P), ("prim", _P), ("metric", _P), ("rhs", _P), ("tile", _I32),
                ("bc", _I32), ("faces", _P), ("states", _P)]


class CBatch(ctypes.Structure):
    _fields_ = [("ws", _P), ("ws_bytes", ctypes.c_size_t), ("nbox", _I32), ("curved", _I32), ("ntiles", ctypes.c_int64),
                ("nc2p_items", ctypes.c_int64), ("nghost_items", ctypes.c_int64), ("two_pass", _I32),
                ("three_pass", _I32)]


_lib.grmhd_batch_workspace_bytes.argtypes = [_I32]
_lib.grmhd_batch_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_batch_prepare.argtypes = [ctypes.POINTER(CBox), _I32, _pp, _P, ctypes.c_size_t, ctypes.POINTER(CBatch), _P]
_lib.grmhd_batch_prepare.restype = _I
_lib.grmhd_batch_rhs.argtypes = [ctypes.POINTER(CBatch), _pp, _P, _P]
_lib.grmhd_batch_rhs.restype = _I
_lib.grmhd_batch_rhs_fused.argtypes = [ctypes.POINTER(CBatch), _pp, _P, _P, _P]
_lib.grmhd_batch_rhs_fused.restype = _I
_lib.grmhd_batch_graph_create.argtypes = [ctypes.POINTER(CBatch), _pp, _P, ctypes.POINTER(_P)]
_lib.grmhd_batch_graph_create.restype = _I
_lib.grmhd_batch_graph_launch.argtypes = [_P, _P]
_lib.grmhd_batch_graph_launch.restype = _I
_lib.grmhd_batch_graph_destroy.argtypes = [_P]
_lib.grmhd_batch_graph_destroy.restype = _I
C_SYMBOLS = C_SYMBOLS + ("grmhd_batch_workspace_bytes", "grmhd_batch_prepare", "grmhd_batch_rhs",
                         "grmhd_batch_graph_create", "grmhd_batch_graph_launch", "grmhd_batch_graph_destroy",
                         "grmhd_batch_rhs_fused")


@dataclass
class Box:
    """One block of a batch: its grid, state tensors, tile shape and boundary."""
    grid: Grid
    cons: "torch.Tensor"
    prim: "torch.Tensor"
    rhs: "torch.Tensor"
    metric: "torch.Tensor" = None
    tile: int = 0
    bc: int = BC_PERIODIC
    faces: "torch.Tensor" = None  # [24][z][y][x] face buffer of the multi-pass FP64 RHS
    states: "torch.Tensor" = None  # [48][z][y][x] WENO5 state buffer of the three-pass FP64 RHS


class Batch:
    """A prepared box table (grmhd_batch_prepare); keeps the tensors alive.
    two_pass (default: FP64): give every box a face buffer (allocated here
    where a box has none), so that the FP64 RHS runs in several passes; for
    WENO5 also a state buffer, so that it runs in three (states, faces,
    cells)."""

    def __init__(self, boxes, params: Params, stream=None, two_pass=None):
        self.boxes = list(boxes)
        n = len(self.boxes)
        if two_pass is None:
            two_pass = params.precision == FP64
        three = bool(two_pass) and params.recon == WENO5
        if two_pass:
            for b in self.boxes:
                if b.faces is None:
                    b.faces = torch.empty((24,) + b.grid.shape, dtype=torch.float64, device=b.cons.device)
                if three and b.states is None:
                    b.states = torch.empty((48,) + b.grid.shape, dtype=torch.float64, device=b.cons.device)
        arr = (CBox * n)()
        for i, b in enumerate(self.boxes):
            arr[i] = CBox(b.grid.c(), _field(b.cons, b.grid, 8, "cons"), _field(b.prim, b.grid, 8, "prim"),
                          _field(b.metric, b.grid, 10, "metric", True), _field(b.rhs, b.grid, 8, "rhs"),
                          int(b.tile), int(b.bc),
                          _field(b.faces, b.grid, 24, "faces", True) if two_pass else None,
                          _field(b.states, b.grid, 48, "states", True) if three else None)
        nbytes = int(_lib.grmhd_batch_workspace_bytes(n))
        if nbytes == 0:
            raise GrmhdError("invalid number of boxes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.boxes[0].cons.device)
        self.c = CBatch()
        rc = _lib.grmhd_batch_prepare(arr, n, ctypes.byref(params.c()), ctypes.c_void_p(self.ws.data_ptr()), nbytes,
                                      ctypes.byref(self.c), _stream(stream))
        _check(rc, "grmhd_batch_prepare")

    @property
    def ncells(self):
        return sum(b.grid.n[0] * b.grid.n[1] * b.grid.n[2] for b in self.boxes)

    def rhs(self, params: Params, nfail=None, stream=None):
        nf = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
        rc = _lib.grmhd_batch_rhs(ctypes.byref(self.c), ctypes.byref(params.c()), nf, _stream(stream))
        _check(rc, "grmhd_batch_rhs")

    def rhs_fused(self, params: Params, nfail=None, status=None, stream=None):
        """grmhd_batch_rhs_fused: the whole evaluation in one persistent launch
        (status: optional device int32, set to GRMHD_ERR_TIMEOUT if a wait gave up)."""
        nf = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
        st = None if status is None else ctypes.c_void_p(status.data_ptr())
        rc = _lib.grmhd_batch_rhs_fused(ctypes.byref(self.c), ctypes.byref(params.c()), nf, st, _stream(stream))
        _check(rc, "grmhd_batch_rhs_fused")

    def graph(self, params: Params, nfail=None):
        """grmhd_batch_graph_create: the batch evaluation as a library-owned
        CUDA graph (BatchGraph), replayed with one launch per evaluation."""
        return BatchGraph(self, params, nfail)


class BatchGraph:
    """A library-owned graph of one batch evaluation; keeps the batch (and
    so its tensors) and nfail alive, and destroys the graph when collected
    or closed."""

    def __init__(self, batch: Batch, params: Params, nfail=None):
        self.batch = batch
        self.nfail = nfail
        self.h = _P()
        nf = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
        rc = _lib.grmhd_batch_graph_create(ctypes.byref(batch.c), ctypes.byref(params.c()), nf, ctypes.byref(self.h))
        _check(rc, "grmhd_batch_graph_create")

    def launch(self, stream=None):
        _check(_lib.grmhd_batch_graph_launch(self.h, _stream(stream)), "grmhd_batch_graph_launch")

    def close(self):
        if self.h:
            _lib.grmhd_batch_graph_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ adjoint --
_lib.grmhd_rhs_adjoint.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, _P, _P]
_lib.grmhd_con2prim_adjoint.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, _P, _P]
_lib.grmhd_prim2con_adjoint.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, _P]
_lib.grmhd_fill_ghosts_adjoint.argtypes = [_pg, _I32, _I32, _P, _P]
_lib.grmhd_density_l2.argtypes = [_pg, _P, _P, ctypes.c_double, _P, _P, _P]
_lib.grmhd_rk_adjoint_workspace_bytes.argtypes = [_pg, _I32]
_lib.grmhd_rk_adjoint_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_rk_step_adjoint.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                       ctypes.c_size_t, _P]
_lib.grmhd_rk_step_record.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P,
                                      _P]
_lib.grmhd_rk_step_record.restype = _I
for _name in ("grmhd_rhs_adjoint", "grmhd_con2prim_adjoint", "grmhd_prim2con_adjoint", "grmhd_fill_ghosts_adjoint",
              "grmhd_density_l2", "grmhd_rk_step_adjoint"):
    getattr(_lib, _name).restype = _I
C_SYMBOLS = C_SYMBOLS + ("grmhd_rhs_adjoint", "grmhd_con2prim_adjoint", "grmhd_prim2con_adjoint",
                         "grmhd_fill_ghosts_adjoint", "grmhd_density_l2", "grmhd_rk_adjoint_workspace_bytes",
                         "grmhd_rk_step_adjoint", "grmhd_rk_step_record")


def _scalar(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.numel() < 1:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def rhs_adjoint(grid: Grid, params: Params, prim, rhs_bar, prim_bar, gamma_bar, metric=None, kij=None, stream=None):
    rc = _lib.grmhd_rhs_adjoint(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                                _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                                _field(rhs_bar, grid, 8, "rhs_bar"), _field(prim_bar, grid, 8, "prim_bar"),
                                _scalar(gamma_bar, "gamma_bar"), _stream(stream))
    _check(rc, "grmhd_rhs_adjoint")


def con2prim_adjoint(grid: Grid, params: Params, prim, prim_bar, cons_bar, gamma_bar, metric=None, stream=None):
    rc = _lib.grmhd_con2prim_adjoint(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                                     _field(metric, grid, 10, "metric", True), _field(prim_bar, grid, 8, "prim_bar"),
                                     _field(cons_bar, grid, 8, "cons_bar"), _scalar(gamma_bar, "gamma_bar"), None,
                                     _stream(stream))
    _check(rc, "grmhd_con2prim_adjoint")


def prim2con_adjoint(grid: Grid, params: Params, prim, cons_bar, prim_bar, gamma_bar, metric=None, stream=None):
    rc = _lib.grmhd_prim2con_adjoint(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                                     _field(metric, grid, 10, "metric", True), _field(cons_bar, grid, 8, "cons_bar"),
                                     _field(prim_bar, grid, 8, "prim_bar"), _scalar(gamma_bar, "gamma_bar"),
                                     _stream(stream))
    _check(rc, "grmhd_prim2con_adjoint")


def fill_ghosts_adjoint(grid: Grid, bc: int, field_bar, stream=None):
    nvar = field_bar.shape[0]
    rc = _lib.grmhd_fill_ghosts_adjoint(ctypes.byref(grid.c()), bc, nvar, _field(field_bar, grid, nvar, "field_bar"),
                                        _stream(stream))
    _check(rc, "grmhd_fill_ghosts_adjoint")


def density_l2(grid: Grid, prim, metric=None, lbar=0.0, loss=None, prim_bar=None, stream=None):
    rc = _lib.grmhd_density_l2(ctypes.byref(grid.c()), _field(prim, grid, 8, "prim"),
                               _field(metric, grid, 10, "metric", True), float(lbar),
                               None if loss is None else _scalar(loss, "loss"),
                               None if prim_bar is None else _field(prim_bar, grid, 8, "prim_bar"), _stream(stream))
    _check(rc, "grmhd_density_l2")


def adjoint_workspace(grid: Grid, scheme: int, device=None):
    nbytes = int(_lib.grmhd_rk_adjoint_workspace_bytes(ctypes.byref(grid.c()), scheme))
    if nbytes == 0:
        raise GrmhdError("invalid grid or scheme for the adjoint workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def stage_count(scheme: int) -> int:
    return {RK2: 2, RK3: 3, RK4: 4}[scheme]


def rk_step_record(grid: Grid, params: Params, scheme: int, dt: float, cons, prim, stage_prims, metric=None,
                   kij=None, ws=None, nfail=None, stream=None):
    """rk_step that also stores the per-stage primitives in stage_prims [stages, 8, *shape]."""
    if ws is None:
        ws = workspace(grid, scheme, cons.device)
    ns = stage_count(scheme)
    if (stage_prims.dtype != torch.float64 or not stage_prims.is_cuda or not stage_prims.is_contiguous()
            or tuple(stage_prims.shape) != (ns, 8) + grid.shape):
        raise ValueError("stage_prims must be a contiguous CUDA float64 tensor [stages, 8, *shape]")
    nf = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_rk_step_record(ctypes.byref(grid.c()), ctypes.byref(params.c()), scheme, float(dt),
                                   _field(cons, grid, 8, "cons"), _field(prim, grid, 8, "prim"),
                                   _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(stage_prims.data_ptr()),
                                   nf, _stream(stream))
    _check(rc, "grmhd_rk_step_record")
    return cons, prim


def rk_step_adjoint(grid: Grid, params: Params, scheme: int, dt: float, cons, prim, cons_bar, prim_bar, gamma_bar,
                    metric=None, kij=None, ws=None, stream=None, stage_prims=None):
    if ws is None:
        ws = adjoint_workspace(grid, scheme, cons.device)
    sp = None
    if stage_prims is not None:
        if tuple(stage_prims.shape) != (stage_count(scheme), 8) + grid.shape or not stage_prims.is_contiguous():
            raise ValueError("stage_prims has the wrong shape")
        sp = ctypes.c_void_p(stage_prims.data_ptr())
    rc = _lib.grmhd_rk_step_adjoint(ctypes.byref(grid.c()), ctypes.byref(params.c()), scheme, float(dt),
                                    _field(cons, grid, 8, "cons"), _field(prim, grid, 8, "prim"),
                                    _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True), sp,
                                    _field(cons_bar, grid, 8, "cons_bar"), _field(prim_bar, grid, 8, "prim_bar"),
                                    _scalar(gamma_bar, "gamma_bar"), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                    _stream(stream))
    _check(rc, "grmhd_rk_step_adjoint")


# ----------------------------------------------- two-level AMR transfer --
_lib.grmhd_restrict.argtypes = [_pg, _P, _pg, _P, _P, _I32, _P]
_lib.grmhd_prolongate.argtypes = [_pg, _P, _pg, _P, _P, _I32, _I32, _P]
_lib.grmhd_reflux.argtypes = [_pg, _pp, _P, _P, _pg, _P, _P, _P, ctypes.c_double, _P, ctypes.c_double, _P, _P]
_lib.grmhd_amr2_workspace_bytes.argtypes = [_pg, _I32, _P, _I32]
_lib.grmhd_amr2_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_amr2_step.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P,
                                 ctypes.c_size_t, _P, _P]
for _name in ("grmhd_restrict", "grmhd_prolongate", "grmhd_reflux", "grmhd_amr2_step"):
    getattr(_lib, _name).restype = _I
C_SYMBOLS = C_SYMBOLS + ("grmhd_restrict", "grmhd_prolongate", "grmhd_reflux", "grmhd_amr2_workspace_bytes",
                         "grmhd_amr2_step")


def _lo3(lo):
    return (ctypes.c_int32 * 3)(*[int(v) for v in lo])


def restrict(coarse: Grid, coarse_field, fine: Grid, fine_field, lo, stream=None):
    """grmhd_restrict: covered coarse cells of coarse_field (in place) := mean of their 8 children."""
    nvar = coarse_field.shape[0]
    rc = _lib.grmhd_restrict(ctypes.byref(coarse.c()), _field(coarse_field, coarse, nvar, "coarse_field"),
                             ctypes.byref(fine.c()), _field(fine_field, fine, nvar, "fine_field"), _lo3(lo), nvar,
                             _stream(stream))
    _check(rc, "grmhd_restrict")
    return coarse_field


def prolongate(coarse: Grid, coarse_field, fine: Grid, fine_field, lo, ghosts_only=True, stream=None):
    """grmhd_prolongate: fine points (ghosts only, or all) of fine_field (in place) from the coarse parents."""
    nvar = fine_field.shape[0]
    rc = _lib.grmhd_prolongate(ctypes.byref(coarse.c()), _field(coarse_field, coarse, nvar, "coarse_field"),
                               ctypes.byref(fine.c()), _field(fine_field, fine, nvar, "fine_field"), _lo3(lo), nvar,
                               int(bool(ghosts_only)), _stream(stream))
    _check(rc, "grmhd_prolongate")
    return fine_field


def reflux(coarse: Grid, params: Params, coarse_prim, fine: Grid, fine_prim, lo, out, scale=1.0, coarse_metric=None,
           fine_metric=None, acc=None, acc_scale=0.0, stream=None):
    """grmhd_reflux: out += scale * (coarse RHS change from flux restriction at the interface)."""
    rc = _lib.grmhd_reflux(ctypes.byref(coarse.c()), ctypes.byref(params.c()), _field(coarse_prim, coarse, 8, "coarse_prim"),
                           _field(coarse_metric, coarse, 10, "coarse_metric", True), ctypes.byref(fine.c()),
                           _field(fine_prim, fine, 8, "fine_prim"), _field(fine_metric, fine, 10, "fine_metric", True),
                           _lo3(lo), float(scale), _field(out, coarse, 8, "out"), float(acc_scale),
                           _field(acc, coarse, 8, "acc", True), _stream(stream))
    _check(rc, "grmhd_reflux")
    return out


def _grid_array(grids):
    arr = (CGrid * max(1, len(grids)))()
    for i, g in enumerate(grids):
        arr[i] = g.c()
    return arr


def amr2_workspace(coarse: Grid, fine, scheme: int, device=None):
    ga = _grid_array(fine)
    nbytes = int(_lib.grmhd_amr2_workspace_bytes(ctypes.byref(coarse.c()), len(fine), ctypes.cast(ga, _P), scheme))
    if nbytes == 0:
        raise GrmhdError("invalid grids for the AMR workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def amr2_step(coarse: Grid, params: Params, scheme: int, dt: float, coarse_cons, coarse_prim, fine, fine_cons,
              fine_prim, los, coarse_metric=None, fine_metrics=None, ws=None, nfail=None, stream=None):
    """grmhd_amr2_step: one composite step of a coarse block and its fine blocks (in place)."""
    nf = len(fine)
    if ws is None:
        ws = amr2_workspace(coarse, fine, scheme, coarse_cons.device)
    ga = _grid_array(fine)
    pc = (_P * max(1, nf))(*[_field(fine_cons[i], fine[i], 8, "fine_cons").value for i in range(nf)])
    pp_ = (_P * max(1, nf))(*[_field(fine_prim[i], fine[i], 8, "fine_prim").value for i in range(nf)])
    pm = None
    if fine_metrics is not None:
        pm = (_P * max(1, nf))(*[_field(fine_metrics[i], fine[i], 10, "fine_metric").value for i in range(nf)])
    lo = (ctypes.c_int32 * max(3, 3 * nf))(*[int(v) for l in los for v in l])
    nf_ptr = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_amr2_step(ctypes.byref(coarse.c()), ctypes.byref(params.c()), scheme, float(dt),
                              _field(coarse_cons, coarse, 8, "coarse_cons"), _field(coarse_prim, coarse, 8, "coarse_prim"),
                              _field(coarse_metric, coarse, 10, "coarse_metric", True), nf, ctypes.cast(ga, _P),
                              ctypes.cast(pc, _P), ctypes.cast(pp_, _P), None if pm is None else ctypes.cast(pm, _P),
                              ctypes.cast(lo, _P), ctypes.c_void_p(ws.data_ptr()), ws.numel(), nf_ptr, _stream(stream))
    _check(rc, "grmhd_amr2_step")


# ------------------------------------------------ constrained transport --
_lib.grmhd_ct_flux_bytes.argtypes = [_pg]
_lib.grmhd_ct_flux_bytes.restype = ctypes.c_size_t
_lib.grmhd_ct_workspace_bytes.argtypes = [_pg, _I32]
_lib.grmhd_ct_workspace_bytes.restype = ctypes.c_size_t
_lib.grmhd_ct_workspace_bytes_cached.argtypes = [_pg, _I32]
_lib.grmhd_ct_workspace_bytes_cached.restype = ctypes.c_size_t
_lib.grmhd_ct_rate.argtypes = [_pg, _pp, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]
_lib.grmhd_ct_rk_step.argtypes = [_pg, _pp, _I32, ctypes.c_double, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P]
_lib.grmhd_ct_divergence.argtypes = [_pg, _P, _P, _P, _P]
_lib.grmhd_ct_cell_field.argtypes = [_pg, _P, _P, _P, _P]
C_SYMBOLS = C_SYMBOLS + ("grmhd_ct_flux_bytes", "grmhd_ct_workspace_bytes", "grmhd_ct_workspace_bytes_cached",
                         "grmhd_ct_rate", "grmhd_ct_rk_step", "grmhd_ct_divergence", "grmhd_ct_cell_field")


def ct_workspace(grid: Grid, scheme: int, device=None, cached: bool = True):
    """Device workspace for ct_rk_step (by default large enough for the cached paths)."""
    fn = _lib.grmhd_ct_workspace_bytes_cached if cached else _lib.grmhd_ct_workspace_bytes
    nbytes = int(fn(ctypes.byref(grid.c()), scheme))
    if nbytes == 0:
        raise GrmhdError("invalid grid or scheme for the workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def ct_rate(grid: Grid, params: Params, prim, metric=None, kij=None, out=None, ws=None, stream=None):
    """grmhd_ct_rate: d(face field)/dt of the interior faces, [3][z][y][x]."""
    if out is None:
        out = torch.empty((3,) + grid.shape, dtype=torch.float64, device=prim.device)
    if ws is None:
        nbytes = int(_lib.grmhd_ct_flux_bytes(ctypes.byref(grid.c())))
        if nbytes == 0:
            raise GrmhdError("invalid grid for the workspace")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=prim.device)
    rc = _lib.grmhd_ct_rate(ctypes.byref(grid.c()), ctypes.byref(params.c()), _field(prim, grid, 8, "prim"),
                            _field(metric, grid, 10, "metric", True), _field(kij, grid, 6, "kij", True),
                            _field(out, grid, 3, "rate"), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _check(rc, "grmhd_ct_rate")
    return out


def ct_rk_step(grid: Grid, params: Params, scheme: int, dt: float, cons, prim, bface, metric=None, kij=None,
               ws=None, nfail=None, stream=None):
    """grmhd_ct_rk_step: one step with constrained transport, in place on cons, prim and bface."""
    if ws is None:
        ws = ct_workspace(grid, scheme, cons.device)
    nf = None if nfail is None else ctypes.c_void_p(nfail.data_ptr())
    rc = _lib.grmhd_ct_rk_step(ctypes.byref(grid.c()), ctypes.byref(params.c()), scheme, float(dt),
                               _field(cons, grid, 8, "cons"), _field(prim, grid, 8, "prim"),
                               _field(bface, grid, 3, "bface"), _field(metric, grid, 10, "metric", True),
                               _field(kij, grid, 6, "kij", True), ctypes.c_void_p(ws.data_ptr()), ws.numel(), nf,
                               _stream(stream))
    _check(rc, "grmhd_ct_rk_step")
    return cons, prim, bface


def ct_divergence(grid: Grid, bface, div=None, maxabs=None, stream=None):
    """grmhd_ct_divergence: the discrete divergence [z][y][x] (interior; 0 elsewhere) and/or
    its largest magnitude (a one-element device tensor).  Returns (div, maxabs)."""
    if div is None and maxabs is None:
        div = torch.empty(grid.shape, dtype=torch.float64, device=bface.device)
    if div is not None and (div.dtype != torch.float64 or not div.is_cuda or not div.is_contiguous()
                            or tuple(div.shape) != grid.shape):
        raise ValueError("div must be a contiguous CUDA float64 tensor of the grid's shape")
    if maxabs is not None and (maxabs.dtype != torch.float64 or not maxabs.is_cuda or maxabs.numel() < 1):
        raise ValueError("maxabs must be a CUDA float64 tensor")
    rc = _lib.grmhd_ct_divergence(ctypes.byref(grid.c()), _field(bface, grid, 3, "bface"),
                                  None if div is None else ctypes.c_void_p(div.data_ptr()),
                                  None if maxabs is None else ctypes.c_void_p(maxabs.data_ptr()), _stream(stream))
    _check(rc, "grmhd_ct_divergence")
    return div, maxabs


def ct_cell_field(grid: Grid, bface, prim, metric=None, stream=None):
    """grmhd_ct_cell_field: the primitive field of every interior cell from
    the face field (face mean over sqrt(gamma)), in place on prim."""
    rc = _lib.grmhd_ct_cell_field(ctypes.byref(grid.c()), _field(bface, grid, 3, "bface"),
                                  _field(metric, grid, 10, "metric", True), _field(prim, grid, 8, "prim"),
                                  _stream(stream))
    _check(rc, "grmhd_ct_cell_field")
    return prim
