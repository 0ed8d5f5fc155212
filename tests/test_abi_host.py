"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/grmhd.h declares, and rejects bad arguments before
touching any device pointer."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grmhd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2210_17509_gb300 import build
    build.build()
    from paper_2210_17509_gb300 import grmhd
    return grmhd


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("grmhd_rhs", "grmhd_con2prim", "grmhd_rk_step", "grmhd_prim2con", "grmhd_fill_ghosts"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(so, n), n


def _grid(lib, n=(8, 8, 8), ng=3, dx=0.1):
    return lib.Grid(n, ng, (dx, dx, dx))


FAKE = ctypes.c_void_p(0x1000)    # never dereferenced: every case fails validation first


def test_rejects_insufficient_ghosts(lib):
    g = _grid(lib, ng=2).c()
    p = lib.Params(recon=lib.WENO5).c()
    rc = lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None)
    assert rc == -1


def test_rejects_bad_params(lib):
    g = _grid(lib).c()
    for kw in ({"gamma": 1.0}, {"recon": 7}, {"bc": 3}, {"precision": 5}, {"nr_maxit": 0}, {"nr_tol": 0.0},
               {"weno_eps": -1.0}, {"rho_atm": 0.0}, {"tile": 7}):
        p = lib.Params(**kw).c()
        rc = lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None)
        assert rc == -1, kw


def test_rejects_null_and_misaligned(lib):
    g = _grid(lib).c()
    p = lib.Params().c()
    assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), None, None, None, FAKE, None) == -1
    assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(0x1003), None, None, FAKE,
                              None) == -1
    # K_ij without a metric is meaningless
    assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, FAKE, FAKE, None) == -1
    assert lib._lib.grmhd_fill_ghosts(ctypes.byref(g), 9, 8, FAKE, None) == -1


def test_workspace_size_and_rk_validation(lib):
    g = _grid(lib, n=(10, 12, 14))
    N = (16 * 18 * 20)
    for scheme, nfield in ((lib.RK2, 1), (lib.RK3, 1), (lib.RK4, 2)):
        b = lib.rk_workspace_bytes(g, scheme)
        assert b >= nfield * 8 * N * 8 and b % 256 == 0
    assert lib.rk_workspace_bytes(g, 5) == 0
    gc = g.c()
    p = lib.Params().c()
    ws = ctypes.c_void_p(0x100000)
    small = lib.rk_workspace_bytes(g, lib.RK3) - 8
    rc = lib._lib.grmhd_rk_step(ctypes.byref(gc), ctypes.byref(p), lib.RK3, 0.01, FAKE, FAKE, None, None, ws,
                                small, None, None)
    assert rc == -4
    rc = lib._lib.grmhd_rk_step(ctypes.byref(gc), ctypes.byref(p), lib.RK3, -0.01, FAKE, FAKE, None, None, ws,
                                10 ** 9, None, None)
    assert rc == -1
    rc = lib._lib.grmhd_rk_step(ctypes.byref(gc), ctypes.byref(p), lib.RK3, 0.01, FAKE, FAKE, None, None,
                                ctypes.c_void_p(0x100008), 10 ** 9, None, None)
    assert rc == -1          # workspace must be 256-byte aligned


def test_recovery_flag_validation(lib):
    """Unknown flag bits are rejected; every call here fails validation before any launch."""
    g = _grid(lib).c()
    ws = ctypes.c_void_p(0x100000)
    known = lib.REUSE_GEOMETRY | lib.NEWMAN_HAMLIN | lib.SINGLE_PASS | lib.DETERMINISTIC
    for flags in (16, lib.NEWMAN_HAMLIN | 32, 1 << 20):
        assert flags & ~known
        p = lib.Params(flags=flags).c()
        assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None) == -1
    # the known flags pass the parameter check and stop at the workspace size
    for flags in (lib.NEWMAN_HAMLIN, lib.NEWMAN_HAMLIN | lib.REUSE_GEOMETRY, lib.SINGLE_PASS, lib.DETERMINISTIC):
        p = lib.Params(flags=flags).c()
        rc = lib._lib.grmhd_rk_step(ctypes.byref(g), ctypes.byref(p), lib.RK3, 0.01, FAKE, FAKE, None, None, ws, 8,
                                    None, None)
        assert rc == -4
    # the reverse calls check the same bits before any launch
    for flags in (16, lib.DETERMINISTIC | 32, 1 << 20):
        p = lib.Params(flags=flags).c()
        assert lib._lib.grmhd_rhs_adjoint(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, FAKE, FAKE,
                                          None) == -1


def test_error_strings(lib):
    assert lib._lib.grmhd_error_string(0) == b"ok"
    assert lib._lib.grmhd_error_string(-4) == b"workspace too small"
    assert lib.version() >= 100


def test_batch_prepare_validation(lib):
    import ctypes as C
    G = lib
    p = G.Params().c()
    assert G._lib.grmhd_batch_workspace_bytes(0) == 0
    nb = G._lib.grmhd_batch_workspace_bytes(4)
    assert nb > 0 and nb % 256 == 0
    boxes = (G.CBox * 1)()
    g = G.Grid((8, 8, 8), 2, (0.1, 0.1, 0.1))       # too few ghosts for WENO5
    boxes[0] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 0, 0)
    out = G.CBatch()
    rc = G._lib.grmhd_batch_prepare(boxes, 1, C.byref(p), C.c_void_p(0x100000), nb, C.byref(out), None)
    assert rc == -1
    g = G.Grid((8, 8, 8), 3, (0.1, 0.1, 0.1))
    boxes[0] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 9, 0)  # bad tile shape
    rc = G._lib.grmhd_batch_prepare(boxes, 1, C.byref(p), C.c_void_p(0x100000), nb, C.byref(out), None)
    assert rc == -1
    boxes[0] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 0, 0)
    rc = G._lib.grmhd_batch_prepare(boxes, 1, C.byref(p), C.c_void_p(0x100000), 16, C.byref(out), None)
    assert rc == -4


def test_batch_prepare_rejects_inconsistent_state_buffers(lib):
    """A state buffer needs a face buffer, and three passes take every box or
    none: both are rejected while validating, before the box table is copied
    anywhere (the pointers here are never dereferenced)."""
    import ctypes as C
    G = lib
    p = G.Params().c()
    nb = G._lib.grmhd_batch_workspace_bytes(2)
    g = G.Grid((8, 8, 8), 3, (0.1, 0.1, 0.1))
    out = G.CBatch()
    boxes = (G.CBox * 1)()
    boxes[0] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 0, 0, None, FAKE)  # states without faces
    assert G._lib.grmhd_batch_prepare(boxes, 1, C.byref(p), C.c_void_p(0x100000), nb, C.byref(out), None) == -1
    boxes = (G.CBox * 2)()
    boxes[0] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 0, 0, FAKE, FAKE)
    boxes[1] = G.CBox(g.c(), FAKE, FAKE, None, FAKE, 0, 0, FAKE, None)  # faces only
    assert G._lib.grmhd_batch_prepare(boxes, 2, C.byref(p), C.c_void_p(0x100000), nb, C.byref(out), None) == -1


def test_autotuner_choice_logic_on_cpu():
    from paper_2210_17509_gb300 import autotune
    costs = {0: 1.0, 1: 1.0, 2: 1.0, 3: 1.0}
    assert autotune.n_tiles(0, (8, 8, 4)) == 1
    assert autotune.n_tiles(2, (8, 8, 8)) == 8        # 32-wide tiles waste 3/4 on an 8-wide box
    assert autotune.choose((8, 8, 8), costs) in (0, 3)
    assert autotune.choose((64, 8, 8), {0: 1.0, 1: 1.0, 2: 0.5, 3: 1.0}) == 2


def test_amr_placement_validation(lib):
    """Fine grids must halve the spacing, have even extents and lie inside the coarse interior."""
    c = lib.Grid((16, 16, 16), 3, (0.1, 0.1, 0.1))
    ok = lib.Grid((8, 8, 8), 3, (0.05, 0.05, 0.05))
    lo = (ctypes.c_int32 * 3)(4, 4, 4)
    cases = [
        (lib.Grid((7, 8, 8), 3, (0.05, 0.05, 0.05)), lo),                 # odd extent
        (lib.Grid((8, 8, 8), 3, (0.1, 0.05, 0.05)), lo),                  # not half the spacing
        (lib.Grid((8, 8, 8), 2, (0.05, 0.05, 0.05)), lo),                 # ghost widths differ
        (ok, (ctypes.c_int32 * 3)(13, 4, 4)),                             # sticks out of the coarse interior
        (ok, (ctypes.c_int32 * 3)(-1, 4, 4)),
    ]
    for fine, l in cases:
        rc = lib._lib.grmhd_restrict(ctypes.byref(c.c()), FAKE, ctypes.byref(fine.c()), FAKE, l, 8, None)
        assert rc == -1
        rc = lib._lib.grmhd_prolongate(ctypes.byref(c.c()), FAKE, ctypes.byref(fine.c()), FAKE, l, 8, 1, None)
        assert rc == -1
    # a valid placement still needs real pointers
    assert lib._lib.grmhd_restrict(ctypes.byref(c.c()), None, ctypes.byref(ok.c()), FAKE, lo, 8, None) == -1


def test_amr2_step_validation_and_workspace(lib):
    c = lib.Grid((16, 16, 16), 3, (0.1, 0.1, 0.1))
    f = [lib.Grid((8, 8, 8), 3, (0.05, 0.05, 0.05)), lib.Grid((6, 6, 6), 3, (0.05, 0.05, 0.05))]
    ga = (lib.CGrid * 2)(f[0].c(), f[1].c())
    b = lib._lib.grmhd_amr2_workspace_bytes(ctypes.byref(c.c()), 2, ctypes.cast(ga, ctypes.c_void_p), lib.RK3)
    assert b == sum(((8 * n.ncell * 8 + 255) // 256) * 256 for n in [c] + f)
    b4 = lib._lib.grmhd_amr2_workspace_bytes(ctypes.byref(c.c()), 2, ctypes.cast(ga, ctypes.c_void_p), lib.RK4)
    assert b4 == 2 * b
    p = lib.Params().c()
    ptrs = (ctypes.c_void_p * 2)(0x1000, 0x2000)
    ws = ctypes.c_void_p(0x100000)

    def step(lo, ws_bytes=10 ** 10, params=p):
        loa = (ctypes.c_int32 * 6)(*lo)
        return lib._lib.grmhd_amr2_step(ctypes.byref(c.c()), ctypes.byref(params), lib.RK3, 0.01, FAKE, FAKE, None, 2,
                                        ctypes.cast(ga, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                                        ctypes.cast(ptrs, ctypes.c_void_p), None, ctypes.cast(loa, ctypes.c_void_p),
                                        ws, ws_bytes, None, None)

    assert step((0, 4, 4, 10, 10, 10)) == -1          # no gap to the coarse boundary
    assert step((2, 2, 2, 6, 6, 6)) == -1             # fine grids touch: [2, 6) and [6, 9)
    assert step((2, 2, 2, 9, 9, 9), ws_bytes=b - 8) == -4
    mixed = lib.Params(precision=lib.MIXED).c()
    assert step((2, 2, 2, 9, 9, 9), params=mixed) == -1   # the composite step is FP64 only


def test_rejects_empty_and_oversized_grids(lib):
    """Empty, negative, too-large and too-many-ghost grids fail validation before any launch."""
    p = lib.Params(recon=lib.MINMOD).c()
    for n, ng in (((0, 8, 8), 3), ((8, -1, 8), 3), ((8, 8, (1 << 20) + 1), 3), ((1 << 14, 1 << 14, 1 << 14), 3),
                  ((8, 8, 8), 17)):
        g = lib.Grid(n, ng, (0.1, 0.1, 0.1)).c()
        assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None) == -1, n
        assert lib._lib.grmhd_fill_ghosts(ctypes.byref(g), 0, 8, FAKE, None) == -1, n
        assert lib._lib.grmhd_rk_workspace_bytes(ctypes.byref(g), lib.RK3) == 0, n
    g = lib.Grid((8, 8, 8), 3, (0.1, 0.0, 0.1)).c()     # zero spacing
    assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None) == -1


def test_ct_workspace_and_validation(lib):
    """Constrained transport: workspace sizes, and short workspaces or bad
    arguments rejected before any launch."""
    g = _grid(lib, n=(10, 12, 14))
    gc = g.c()
    N = 16 * 18 * 20
    r256 = lambda b: (b + 255) // 256 * 256
    assert lib._lib.grmhd_ct_flux_bytes(ctypes.byref(gc)) == r256(9 * N * 8) + r256(3 * N * 8)
    for scheme in (lib.RK2, lib.RK3, lib.RK4):
        part = r256(9 * N * 8) + r256(3 * N * 8) * (3 if scheme == lib.RK4 else 2)
        assert lib._lib.grmhd_ct_workspace_bytes(ctypes.byref(gc), scheme) == part + lib.rk_workspace_bytes(g, scheme)
        assert (lib._lib.grmhd_ct_workspace_bytes_cached(ctypes.byref(gc), scheme)
                == part + lib.rk_workspace_bytes_cached(g, scheme))
    assert lib._lib.grmhd_ct_workspace_bytes(ctypes.byref(gc), 7) == 0
    p = lib.Params().c()
    ws = ctypes.c_void_p(0x100000)
    need = lib._lib.grmhd_ct_workspace_bytes(ctypes.byref(gc), lib.RK3)

    def step(ws_bytes=10 ** 9, dt=0.01, bface=FAKE, wsp=ws, params=p):
        return lib._lib.grmhd_ct_rk_step(ctypes.byref(gc), ctypes.byref(params), lib.RK3, dt, FAKE, FAKE, bface,
                                         None, None, wsp, ws_bytes, None, None)

    assert step(ws_bytes=need - 8) == -4
    assert step(dt=0.0) == -1
    assert step(bface=None) == -1
    assert step(bface=ctypes.c_void_p(0x1004)) == -1
    assert step(wsp=ctypes.c_void_p(0x100008)) == -1
    rc = lib._lib.grmhd_ct_rate(ctypes.byref(gc), ctypes.byref(p), FAKE, None, None, FAKE, ws,
                                lib._lib.grmhd_ct_flux_bytes(ctypes.byref(gc)) - 8, None)
    assert rc == -4
    assert lib._lib.grmhd_ct_divergence(ctypes.byref(gc), FAKE, None, None, None) == -1
    thin = lib.Grid((8, 8, 8), 2, (0.1, 0.1, 0.1)).c()     # WENO5 needs three ghost layers
    rc = lib._lib.grmhd_ct_rk_step(ctypes.byref(thin), ctypes.byref(p), lib.RK3, 0.01, FAKE, FAKE, FAKE, None, None,
                                   ws, 10 ** 9, None, None)
    assert rc == -1


def test_eos_validation(lib):
    """An unknown EOS, a polytrope without a positive K, and the adjoint under the polytrope are refused
    before any launch."""
    g = _grid(lib).c()
    for eos, K in ((2, 1.0), (lib.EOS_POLYTROPE, 0.0), (lib.EOS_POLYTROPE, float("nan"))):
        p = lib.Params(eos=eos, poly_K=K).c()
        assert lib._lib.grmhd_rhs(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, None) == -1
        assert lib._lib.grmhd_con2prim(ctypes.byref(g), ctypes.byref(p), FAKE, None, FAKE, None, None, None) == -1
    p = lib.Params(eos=lib.EOS_POLYTROPE, poly_K=100.0).c()
    assert lib._lib.grmhd_rhs_adjoint(ctypes.byref(g), ctypes.byref(p), FAKE, None, None, FAKE, FAKE, FAKE,
                                      None) == -1


def test_batch_rejects_the_polytrope(lib):
    import ctypes as C
    p = lib.Params(eos=lib.EOS_POLYTROPE, poly_K=100.0).c()
    boxes = (lib.CBox * 1)()
    out = lib.CBatch()
    nb = lib._lib.grmhd_batch_workspace_bytes(1)
    assert lib._lib.grmhd_batch_prepare(boxes, 1, C.byref(p), C.c_void_p(0x100000), nb, C.byref(out), None) == -1


def test_one_launch_graph_and_cell_field_validation(lib):
    """The one-launch batch, the library graph and the cell-field set-up
    reject bad arguments before any CUDA call; the batch workspace holds the
    completion counters of the one-launch form ahead of the box table."""
    import ctypes as C
    G = lib
    p = G.Params().c()
    b = G.CBatch()                                    # ws NULL, nbox 0
    assert G._lib.grmhd_batch_rhs_fused(C.byref(b), C.byref(p), None, None, None) == -1
    assert G._lib.grmhd_batch_rhs_fused(None, C.byref(p), None, None, None) == -1
    b.ws, b.nbox = C.c_void_p(0x100000), 4
    bad = G.Params(recon=7).c()
    assert G._lib.grmhd_batch_rhs_fused(C.byref(b), C.byref(bad), None, None, None) == -1
    poly = G.Params(eos=G.EOS_POLYTROPE, poly_K=1.0).c()
    assert G._lib.grmhd_batch_rhs_fused(C.byref(b), C.byref(poly), None, None, None) == -1
    assert G._lib.grmhd_batch_rhs_fused(C.byref(b), C.byref(p), None, C.c_void_p(0x1002), None) == -1  # misaligned
    h = C.c_void_p()
    assert G._lib.grmhd_batch_graph_create(None, C.byref(p), None, C.byref(h)) == -1 and not h.value
    assert G._lib.grmhd_batch_graph_create(C.byref(b), C.byref(p), None, None) == -1
    assert G._lib.grmhd_batch_graph_launch(None, None) == -1
    assert G._lib.grmhd_batch_graph_destroy(None) == 0
    # 4 boxes: header 256 B, 2 x 4 counters rounded to 256 B, then the table
    nb = G._lib.grmhd_batch_workspace_bytes(4)
    assert nb >= 512 + 4 * C.sizeof(G.CBox) and nb % 256 == 0
    g = _grid(lib)
    G._lib.grmhd_ct_cell_field.restype = C.c_int
    assert G._lib.grmhd_ct_cell_field(C.byref(g.c()), None, None, FAKE, None) == -1
    assert G._lib.grmhd_ct_cell_field(C.byref(g.c()), FAKE, None, None, None) == -1
    assert G._lib.grmhd_ct_cell_field(C.byref(g.c()), C.c_void_p(0x1001), None, FAKE, None) == -1
