/*
 * grmhd.h -- C ABI of the GB300 GRMHD method-of-lines library (libgrmhd.so).
 *
 * The library evaluates the Valencia-formulation GRMHD right-hand side of
 * GRaM-X (arXiv 2210.17509), Sec. 2.2-2.3, on one 3D Cartesian block with
 * ghost zones, plus the pieces a method-of-lines step needs around it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array pointers are DEVICE pointers (cudaMalloc / torch CUDA memory)
 *    unless the argument says "host".  The caller owns every buffer; the
 *    library never allocates, frees or retains device memory (the one thing
 *    it holds is the graph handle of grmhd_batch_graph_create, until the
 *    caller destroys it).
 *  - Layout: structure of arrays, double precision, [var][z][y][x] with x
 *    fastest.  Every field spans the full block including ghosts:
 *    N_d = n_d + 2 ng points per axis, ncell = N_x N_y N_z, component q of a
 *    field starts at element q * ncell.
 *      prim   8 comps  [rho, v^x, v^y, v^z, P, B^x, B^y, B^z]
 *             v^i is the Valencia 3-velocity (Eq. 10), B^i the Eulerian field
 *             (undensitised).  Pressure replaces the paper's eps as the
 *             thermal variable: eps = P / ((Gamma - 1) rho) (Gamma-law EOS).
 *      cons   8 comps  [D, S_x, S_y, S_z, tau, B~^x, B~^y, B~^z]  (Eqs. 6-9)
 *      metric 10 comps [alpha, beta^x, beta^y, beta^z,
 *                       g_xx, g_xy, g_xz, g_yy, g_yz, g_zz] at cell centres,
 *             ghosts included.  NULL means Minkowski (alpha = 1, beta = 0,
 *             gamma_ij = delta_ij); the kernels then take a flat fast path.
 *      kij    6 comps  [K_xx, K_xy, K_xz, K_yy, K_yz, K_zz]; NULL means 0.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  No call synchronises the device.
 *  - Return value: GRMHD_OK, or a negative error code.  Argument errors are
 *    detected on the host before anything is launched.  Per-cell physics
 *    failures of the primitive recovery are NOT return codes: they go to the
 *    optional `status` array and `nfail` counter.
 *  - Buffers passed to one call must not overlap unless stated otherwise.
 */
#ifndef GRMHD_H
#define GRMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRMHD_OK 0
#define GRMHD_ERR_ARG (-1)     /* invalid argument (NULL, extent, ghost width, alignment, size) */
#define GRMHD_ERR_CUDA (-2)    /* a CUDA runtime call or launch failed */
#define GRMHD_ERR_TIMEOUT (-3) /* a bounded device-side wait gave up */
#define GRMHD_ERR_SIZE (-4)    /* workspace too small */

/* reconstruction (Sec. 2.3: TVD with minmod limiter, or WENO5 after Shu 1998) */
#define GRMHD_MINMOD 0
#define GRMHD_WENO5 1
/* boundary condition applied to primitive ghost zones: periodic, or a copy of
 * the nearest interior cell (the "von Neumann" condition of Sec. 4.1) */
#define GRMHD_BC_PERIODIC 0
#define GRMHD_BC_COPY 1
/* arithmetic of the RHS: all FP64, or FP32 reconstruction / Riemann flux /
 * divergence with FP64 primitive recovery, sqrt(gamma) and metric inverse */
#define GRMHD_FP64 0
#define GRMHD_MIXED 1
/* method-of-lines integrators: SSP Heun, SSP Shu-Osher RK3, classical RK4 */
#define GRMHD_RK2 2
#define GRMHD_RK3 3
#define GRMHD_RK4 4

/* Block geometry.  n = interior cells per axis (x, y, z); ng = ghost width
 * (>= 3 for WENO5 and for a curved metric, >= 2 for minmod on a flat
 * metric); dx = cell size per axis. */
typedef struct {
  int32_t n[3];
  int32_t ng;
  double dx[3];
} grmhd_grid;

/* Method parameters. */
typedef struct {
  double gamma;      /* Gamma-law index, P = (Gamma - 1) rho eps (Sec. 2.3); 1 < gamma <= 3 */
  int32_t recon;     /* GRMHD_MINMOD | GRMHD_WENO5 */
  int32_t bc;        /* GRMHD_BC_PERIODIC | GRMHD_BC_COPY */
  int32_t precision; /* GRMHD_FP64 | GRMHD_MIXED */
  int32_t nr_maxit;  /* Newton iteration cap of the primitive recovery (e.g. 50) */
  double rho_atm;    /* atmosphere density (Sec. 4.4 uses an artificial atmosphere) */
  double p_atm;      /* atmosphere pressure */
  double nr_tol;     /* Newton stop: |dz|/z and |dW|/W below nr_tol (e.g. 1e-12) */
  double weno_eps;   /* WENO5 epsilon in alpha_k = d_k / (eps + beta_k)^2 (e.g. 1e-6) */
  int32_t tile;      /* RHS tile shape GRMHD_TILE_* (0 = 8x8x4); performance only */
  int32_t flags;     /* 0, or GRMHD_REUSE_GEOMETRY | GRMHD_NEWMAN_HAMLIN | GRMHD_SINGLE_PASS |
                        GRMHD_DETERMINISTIC */
  int32_t eos;       /* GRMHD_EOS_IDEAL (Gamma-law, P = (Gamma - 1) rho eps) | GRMHD_EOS_POLYTROPE */
  double poly_K;     /* polytropic constant K of P = K rho^gamma (GRMHD_EOS_POLYTROPE; > 0) */
} grmhd_params;

/* Equations of state (Sec. 2.3, EOS paragraph).  Under GRMHD_EOS_POLYTROPE
 * the pressure is K rho^gamma wherever it is used: the face states take it
 * from the reconstructed density, prim -> cons ignores the pressure entry
 * of its input, the recovery solves for W from D, S_i and B^i only (tau is
 * evolved but not read) and writes P = K rho^gamma, and the atmosphere
 * pressure is K rho_atm^gamma (p_atm is not used).  Cell primitives passed
 * to the RHS must carry P = K rho^gamma, as the recovery writes them.
 * eps = P / ((gamma - 1) rho) under both.  The polytrope's RHS runs on
 * the default tile shape whatever params.tile says.  The adjoint and the
 * batched-box entry points accept GRMHD_EOS_IDEAL only. */
#define GRMHD_EOS_IDEAL 0
#define GRMHD_EOS_POLYTROPE 1

/* flags: the metric, the grid and the precision are unchanged since the
 * previous grmhd_rk_step with this same workspace, so the geometry caches
 * (built from the metric, see grmhd_rk_workspace_bytes_cached) are reused
 * instead of rebuilt.  A static spacetime sets it after its first step.
 * Ignored by every other call. */
#define GRMHD_REUSE_GEOMETRY 1
/* flags: the primitive recovery starts with the Newman-Hamlin iteration
 * instead of the Newton iteration (see grmhd_con2prim). */
#define GRMHD_NEWMAN_HAMLIN 2
/* flags: the FP64 RHS of the cached paths runs in one pass (each tile
 * computing the faces on its boundaries as well) instead of several (for
 * WENO5 the face states of every cell into the workspace's state buffer,
 * every face flux once into its face buffer, then a per-cell pass; for
 * minmod tiled faces, then the per-cell pass).  The results are the same; a
 * switch for comparison. */
#define GRMHD_SINGLE_PASS 4
/* flags: the reverse-mode calls (grmhd_rhs_adjoint, grmhd_con2prim_adjoint,
 * grmhd_prim2con_adjoint, grmhd_rk_step_adjoint) add in a fixed order, so
 * their results are the same to the bit from run to run.  Each direction's
 * face adjoint runs in six launches, the faces by their index mod 6 (faces
 * six apart have disjoint stencils, so no cell receives two adds in one
 * launch), and the Gamma sums go to per-warp slots that the last block of
 * each launch adds in slot order.  The slots belong to the library: calls
 * with this flag must not run concurrently on different streams.  Without
 * it the adds are atomic, their order varies and so do the last bits.
 * grmhd_density_l2's loss sum stays atomic; the forward calls ignore it. */
#define GRMHD_DETERMINISTIC 8

/* RHS tile shapes (cells per CTA along x, y, z; 256 threads per CTA).  The
 * shape changes only how the work is cut, never the result.  8x8x8 (two
 * cells per thread, fewer recomputed tile-boundary faces) is for single
 * blocks; batched boxes use 0..3. */
#define GRMHD_TILE_8x8x4 0
#define GRMHD_TILE_16x4x4 1
#define GRMHD_TILE_32x4x2 2
#define GRMHD_TILE_4x8x8 3
#define GRMHD_TILE_8x8x8 4

/* Primitive -> conserved variables, Eqs. 6-9 (Sec. 2.2), on every cell of
 * the block (ghosts included), with the metric of that cell.
 *   prim   in   8 x ncell
 *   metric in   10 x ncell or NULL
 *   cons   out  8 x ncell */
int grmhd_prim2con(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                   const double* metric, double* cons, void* stream);

/* Conserved -> primitive recovery (Sec. 2.3, "Find the primitive variable
 * vector"): per interior cell, a 2D Newton-Raphson in (z = rho h W^2, W)
 * (the paper's 3D Newton with the temperature eliminated by the Gamma-law);
 * if it does not converge or converges to an unphysical root, the
 * Newman-Hamlin iteration over P (an Aitken-accelerated fixed point, each
 * step a closed-form cubic root in eps = B^2 + z), as in the paper; if that
 * fails too, bracketed bisection in z.  With GRMHD_NEWMAN_HAMLIN in
 * params.flags the Newman-Hamlin iteration comes first.  Cells that still
 * fail or come out unphysical (no root, NaN, rho < rho_atm, v >= 1) get the
 * atmosphere (rho_atm, v = 0, p_atm, B kept); a valid root with P <= 0 keeps
 * rho and v and gets the pressure floor P = p_atm (Sec. 2.3 lists these
 * failure modes).  The initial pressure of the Newman-Hamlin iteration is
 * the incoming primitive pressure.
 *   cons   in      8 x ncell (interior read)
 *   metric in      10 x ncell or NULL
 *   prim   in/out  8 x ncell: interior holds the initial guess on entry and
 *                  the result on exit; ghost entries are not touched
 *   status out     int8 x ncell or NULL: 0 Newton or Newman-Hamlin,
 *                  1 bisection fallback, 2 atmosphere, 3 pressure floor
 *                  (interior entries only)
 *   nfail  in/out  one device int32 or NULL: atomically incremented by the
 *                  number of atmosphere and pressure-floor cells (caller
 *                  zeroes it) */
int grmhd_con2prim(const grmhd_grid* grid, const grmhd_params* params, const double* cons,
                   const double* metric, double* prim, int8_t* status, int32_t* nfail,
                   void* stream);

/* Ghost-zone fill of an nvar-component field from its interior: periodic
 * wrap or copy of the nearest interior cell (Sec. 4.1 boundary; Sec. 5 runs
 * are periodic).  Edges and corners are filled consistently. */
int grmhd_fill_ghosts(const grmhd_grid* grid, int32_t bc, int32_t nvar, double* field, void* stream);

/* Method-of-lines right-hand side dU/dt = -d_i F^i + S (Eq. 11): reconstruct
 * the primitives to faces (minmod or WENO5), metric at faces as the mean of
 * the two adjacent cells (a face state with rho <= 0, P <= 0 or v >= 1 is
 * replaced by its cell's state), HLLE fluxes (Eq. 12), flux divergence, source
 * terms (Eq. 13, 3+1 form, metric derivatives by 4th-order centred
 * differences).  Each face flux is computed once per launch tile.
 *   prim   in   8 x ncell, ghosts filled
 *   metric in   10 x ncell or NULL
 *   kij    in   6 x ncell or NULL
 *   rhs    out  8 x ncell; interior written, ghost entries not touched */
int grmhd_rhs(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
              const double* metric, const double* kij, double* rhs, void* stream);

/* grmhd_rhs computed from the geometry caches of grmhd_rk_workspace_bytes_cached
 * (and, for GRMHD_MIXED, an FP32 copy of prim; for FP64 with a metric, the
 * multi-pass state and face buffers) held in ws: the same RHS,
 * with the per-face and per-cell metric algebra done once per static metric.
 * ws >= grmhd_rhs_workspace_bytes(grid), 256-byte aligned; the caches are
 * rebuilt unless params->flags has GRMHD_REUSE_GEOMETRY (same grid, metric and
 * precision as the previous call with this ws). */
size_t grmhd_rhs_workspace_bytes(const grmhd_grid* grid);
int grmhd_rhs_cached(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                     const double* metric, const double* kij, double* rhs, void* ws, size_t ws_bytes,
                     void* stream);

/* Bytes of device workspace grmhd_rk_step needs for `scheme`. */
size_t grmhd_rk_workspace_bytes(const grmhd_grid* grid, int32_t scheme);

/* Bytes of workspace with which grmhd_rk_step runs from caches: a geometry
 * cache of the metric (face and cell sqrt(gamma), inverse metric and 4th-order
 * metric derivatives, computed in FP64 once per step -- or once per static
 * spacetime with GRMHD_REUSE_GEOMETRY -- stored as FP64 for the FP64 path and
 * as FP32 for the mixed path), an FP64 inverse-metric cache for the recovery,
 * for the mixed path an FP32 copy of the primitives, and for the FP64 path a
 * face buffer of 24 and a state buffer of 48 doubles per point (the
 * multi-pass RHS: every cell's face states and every face flux computed
 * once, see GRMHD_SINGLE_PASS).  With less (but at least
 * grmhd_rk_workspace_bytes) the kernels read the FP64 inputs directly;
 * results agree to round-off. */
size_t grmhd_rk_workspace_bytes_cached(const grmhd_grid* grid, int32_t scheme);

/* One method-of-lines step of size dt (Sec. 2.3; integrators RK2/RK4 as in
 * Secs. 4-5, and SSP RK3).  Every stage evaluates the RHS from the current
 * primitives and folds the stage combination into the RHS epilogue, then
 * recovers primitives (con2prim) and fills their ghosts.
 *   cons   in/out  8 x ncell: U^n on entry (interior), U^{n+1} on exit
 *   prim   in/out  8 x ncell: on entry consistent with cons, ghosts filled;
 *                  on exit the primitives of U^{n+1}, ghosts filled
 *   metric, kij    as for grmhd_rhs
 *   ws             device workspace of ws_bytes >= grmhd_rk_workspace_bytes()
 *                  (256-byte aligned), contents scratch
 *   nfail          as for grmhd_con2prim (summed over the stages) or NULL */
int grmhd_rk_step(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                  double* cons, double* prim, const double* metric, const double* kij, void* ws,
                  size_t ws_bytes, int32_t* nfail, void* stream);

/* ----------------------------------------------------------------------
 * Batched boxes: many independent, unevenly sized blocks (the AMR block
 * structure of Sec. 3.1, here as independent boxes with their own ghost
 * zones) swept by persistent kernels -- one launch per phase over the whole
 * box table, with a dynamic work counter.  Each box carries its own tile
 * shape (chosen by the project's autotuner); the result does not depend on it.
 * ---------------------------------------------------------------------- */
typedef struct {
  grmhd_grid grid;
  double* cons;          /* 8 x ncell: conserved variables, interior read */
  double* prim;          /* 8 x ncell: Newton guess in; primitives out, ghosts filled */
  const double* metric;  /* 10 x ncell or NULL; a batch is all flat or all curved */
  double* rhs;           /* 8 x ncell: interior RHS out, ghost entries untouched */
  int32_t tile;          /* GRMHD_TILE_* for this box */
  int32_t bc;            /* GRMHD_BC_* for this box's primitive ghosts */
  double* faces;         /* nullable: 24 x ncell doubles of face buffer; when every box has one, the
                            FP64 RHS runs in several passes (every face flux once), else in one */
  double* states;        /* nullable (needs faces): 48 x ncell doubles of WENO5 face states; when every
                            box has one, the FP64 WENO5 RHS runs in three passes (every cell's face
                            states once, then every face flux once, then the per-cell pass) */
} grmhd_box;

/* Prepared batch (filled by grmhd_batch_prepare; plain data, caller-owned). */
typedef struct {
  void* ws;              /* device workspace holding the box table */
  size_t ws_bytes;
  int32_t nbox;
  int32_t curved;        /* 1 if the boxes carry a metric */
  int64_t ntiles;        /* RHS work items */
  int64_t nc2p_items;    /* recovery work items (256 interior cells each) */
  int64_t nghost_items;  /* ghost-fill work items (256 points each) */
  int32_t two_pass;      /* 1 if every box carries a face buffer */
  int32_t three_pass;    /* 1 if every box also carries a state buffer */
} grmhd_batch;

/* Device workspace (bytes) for a batch of nbox boxes; 0 if nbox is invalid. */
size_t grmhd_batch_workspace_bytes(int32_t nbox);

/* Validate the host array `boxes`, order them largest first, lay the box
 * table and work offsets into the device workspace `ws` (256-byte aligned,
 * >= grmhd_batch_workspace_bytes) and fill `batch`.  Synchronises `stream`
 * once (host-to-device copy of the table); call it outside stream capture.
 * The box buffers must stay valid for every later grmhd_batch_rhs. */
int grmhd_batch_prepare(const grmhd_box* boxes, int32_t nbox, const grmhd_params* params, void* ws,
                        size_t ws_bytes, grmhd_batch* batch, void* stream);

/* For every box: primitive recovery from cons (as grmhd_con2prim), ghost fill
 * (as grmhd_fill_ghosts with the box's bc), then the RHS (as grmhd_rhs with
 * the box's tile shape; the same bits in several passes when batch->two_pass
 * and params->precision is GRMHD_FP64: two, or three for WENO5 with
 * batch->three_pass).  Three persistent launches on `stream` (four with two
 * passes, five with three; plus one memset of the work counters), no host
 * synchronisation: the sequence can be captured into a CUDA graph.  nfail as
 * for grmhd_con2prim.  Boxes' face and state buffers must not overlap. */
int grmhd_batch_rhs(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail, void* stream);

/* grmhd_batch_rhs in ONE persistent launch (plus one memset of the work and
 * completion counters): recovery, ghost fill and the one-pass RHS of every
 * box in a single kernel.  One work counter hands out the items of the three
 * phases in phase order; an item that needs an earlier phase of its own box
 * (the ghost fill needs the box's recovery, its RHS tiles its ghost fill)
 * waits, with a bounded spin, until that phase's completion counter for the
 * box is full.  Every item waited on was handed out earlier to a running CTA,
 * so the waits end without any co-residency requirement.  Results: the bits
 * of grmhd_batch_rhs without face buffers (the one-pass RHS, whatever
 * batch->two_pass says; in FP64 WENO5 the tiles then stage their face
 * states in 211 KB of shared memory, one CTA per SM).
 *   status (device int32, nullable): set to GRMHD_ERR_TIMEOUT if a wait gave
 *   up (the results are then not valid); the caller zeroes it.
 *   nfail as for grmhd_batch_rhs.  Overlapping calls on one batch race. */
int grmhd_batch_rhs_fused(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail, int32_t* status,
                          void* stream);

/* A CUDA graph of one grmhd_batch_rhs, owned by the library: an opaque
 * handle. */
typedef struct grmhd_batch_graph_t* grmhd_batch_graph;

/* Capture grmhd_batch_rhs(batch, params, nfail) -- the memset of the work
 * counters and the persistent launches -- into a CUDA graph and instantiate
 * it.  The capture runs on a private stream that the call creates and
 * destroys; nothing runs on the GPU.  The batch's workspace and box buffers,
 * *params' values and nfail are fixed into the graph: they must stay valid,
 * and the graph computes with the captured params, until the handle is
 * destroyed.  The handle (host memory and the instantiated graph's driver
 * resources; no device memory of the caller) is the one thing the library
 * holds on the caller's behalf.  *graph = NULL on failure; argument errors
 * of grmhd_batch_rhs are returned as it returns them. */
int grmhd_batch_graph_create(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail,
                             grmhd_batch_graph* graph);

/* One evaluation of the captured batch on `stream`: one graph launch,
 * results as grmhd_batch_rhs.  Launches of one handle on different streams
 * must not overlap (they share the work counters). */
int grmhd_batch_graph_launch(grmhd_batch_graph graph, void* stream);

/* Release the handle (NULL is a no-op).  No launch of it may be pending. */
int grmhd_batch_graph_destroy(grmhd_batch_graph graph);

/* ----------------------------------------------------------------------
 * Reverse mode (adjoint) of the FP64 method, hand-written.  The paper has no
 * adjoint; these are the transposes of the forward entry points above, so
 * that gradients of a functional of the evolved state with respect to the
 * initial primitives and Gamma can be accumulated backwards through a
 * checkpointed sequence of grmhd_rk_step calls.  All require
 * params->precision == GRMHD_FP64.  "Accumulated" outputs are added to.
 * ---------------------------------------------------------------------- */

/* prim_bar += (d rhs / d prim)^T rhs_bar, gamma_bar += (d rhs / d Gamma)^T rhs_bar.
 *   prim      in   8 x ncell, ghosts filled (the RHS input)
 *   rhs_bar   in   8 x ncell, interior read
 *   prim_bar  acc  8 x ncell, ghost entries included (they receive the
 *                  adjoint of the stencil reads; see grmhd_fill_ghosts_adjoint)
 *   gamma_bar acc  one device double
 * Contributions are added with atomics, in an order that varies, unless
 * params->flags has GRMHD_DETERMINISTIC. */
int grmhd_rhs_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                      const double* metric, const double* kij, const double* rhs_bar, double* prim_bar,
                      double* gamma_bar, void* stream);

/* Adjoint of the primitive recovery at its solution prim (interior): the
 * recovery inverts prim -> cons (Eqs. 6-9), so cons_bar += (dU/dP)^{-T}
 * prim_bar and gamma_bar -= cons_bar_added . dU/dGamma (implicit function
 * theorem).  nsingular (device int32, nullable) counts cells whose Jacobian
 * could not be inverted (their contribution is skipped). */
int grmhd_con2prim_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                           const double* metric, const double* prim_bar, double* cons_bar,
                           double* gamma_bar, int32_t* nsingular, void* stream);

/* Adjoint of grmhd_prim2con on the interior: prim_bar += (dU/dP)^T cons_bar,
 * gamma_bar += cons_bar . dU/dGamma. */
int grmhd_prim2con_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                           const double* metric, const double* cons_bar, double* prim_bar,
                           double* gamma_bar, void* stream);

/* Transpose of grmhd_fill_ghosts: every ghost entry of field_bar is added to
 * the interior entry it was copied from, then set to zero. */
int grmhd_fill_ghosts_adjoint(const grmhd_grid* grid, int32_t bc, int32_t nvar, double* field_bar,
                              void* stream);

/* Functional L = sum over interior cells of rho^2 sqrt(gamma) dx dy dz:
 * loss (device double, nullable) += L; prim_bar (nullable) += lbar dL/dprim. */
int grmhd_density_l2(const grmhd_grid* grid, const double* prim, const double* metric, double lbar,
                     double* loss, double* prim_bar, void* stream);

/* Bytes of workspace for grmhd_rk_step_adjoint (RK2 / RK3; 0 otherwise):
 * the stage and adjoint arrays (5 + stages fields of 8 x ncell doubles) and
 * the cell-state buffer of the WENO5 face adjoint (96 x ncell doubles: both
 * WENO5 states of every cell of one direction with their derivatives). */
size_t grmhd_rk_adjoint_workspace_bytes(const grmhd_grid* grid, int32_t scheme);

/* grmhd_rk_step that also records the primitives after each stage (ghosts
 * filled) into stage_prims: stages x 8 x ncell doubles, stage k at offset
 * k * 8 * ncell; the last one equals the step's output primitives.  Feeds
 * grmhd_rk_step_adjoint without a second recomputation. */
int grmhd_rk_step_record(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                         double* cons, double* prim, const double* metric, const double* kij, void* ws,
                         size_t ws_bytes, double* stage_prims, int32_t* nfail, void* stream);

/* Reverse of one grmhd_rk_step (SSP RK2 or RK3) taken from (cons, prim):
 * recomputes the stages (or takes them from stage_prims, as recorded by
 * grmhd_rk_step_record for this step), then sweeps them backwards.
 *   cons, prim  in      the step's inputs (prim ghosts filled), unchanged
 *   stage_prims in      NULL, or the recorded stage primitives of the step
 *   cons_bar    in/out  adjoint of the step's output U (interior) on entry,
 *                       adjoint of the input U on exit
 *   prim_bar    in/out  adjoint of the step's output primitives (8 x ncell,
 *                       ghost entries included) on entry; adjoint of the
 *                       input primitives (ghost entries included) on exit
 *   gamma_bar   acc     one device double
 *   ws          >= grmhd_rk_adjoint_workspace_bytes, 256-byte aligned */
int grmhd_rk_step_adjoint(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                          const double* cons, const double* prim, const double* metric, const double* kij,
                          const double* stage_prims, double* cons_bar, double* prim_bar, double* gamma_bar,
                          void* ws, size_t ws_bytes, void* stream);

/* Size of the library-owned scratch of grmhd_rk_step_static: 64 MiB. */
#define GRMHD_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

/* grmhd_rk_step without a caller workspace.  The paper has no counterpart:
 * this is a convenience for callers that cannot call cudaMalloc or any other
 * allocating routine (a host code whose device memory belongs to another
 * allocator or pool, a callback context where allocation is forbidden, a
 * binding without a device allocator).  Same arguments and results as
 * grmhd_rk_step minus ws/ws_bytes, with that step's workspace laid over a
 * file-scope device array of GRMHD_STATIC_SCRATCH_BYTES.  The array is held
 * on every GPU where this library's device code is loaded (under CUDA's
 * default lazy module loading, from the library's first use there), until
 * the process exits.
 *   Limit: grmhd_rk_workspace_bytes(grid, scheme) <= GRMHD_STATIC_SCRATCH_BYTES,
 *   i.e. ncell <= 1,048,576 for RK2/RK3 and about half that for RK4 (e.g. a
 *   94^3 interior with 3 ghosts); larger blocks return GRMHD_ERR_SIZE.
 *   Paths: blocks whose grmhd_rk_workspace_bytes_cached fits in the array
 *   (ncell up to about 42,100 for RK2/RK3 and 40,500 for RK4, e.g. a 28^3
 *   interior with 3 ghosts) run the cached paths, larger ones the uncached paths; the
 *   results are those of grmhd_rk_step given a workspace of that size.
 *   GRMHD_REUSE_GEOMETRY is ignored: the geometry caches are rebuilt on
 *   every call, since the array may hold another block's caches.
 *   The first call on a device (that device current) looks up the array's
 *   device address once; make that first call before any stream capture,
 *   and do not use this function across a cudaDeviceReset.
 *   Every call shares the one array: calls that overlap on the GPU race.
 *   Allocates nothing: no cudaMalloc, no cudaFree, no allocating library call. */
int grmhd_rk_step_static(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                         double* cons, double* prim, const double* metric, const double* kij,
                         int32_t* nfail, void* stream);

/* ----------------------------------------------------------------------
 * Two-level block AMR without subcycling (Sec. 3: each refined grid halves
 * the spacing of the next coarser one and is properly nested in it; ghost
 * zones of a refined grid are filled by prolongation from the coarser level;
 * coarse cells overlaid by a refined grid are reset by restriction; fine
 * fluxes are restricted onto the coarse grid; one global time step, so no
 * refluxing in time).
 *
 * Placement: a fine grid at lo[3] (coarse interior cell indices) has
 * fine.n even per axis, fine.ng == coarse.ng >= 2 and fine.dx = coarse.dx/2
 * (relative 1e-12); its interior cell i lies in the coarse interior cell
 * lo + floor(i/2) per axis, and it covers coarse cells lo .. lo + fine.n/2 - 1,
 * which must lie inside the coarse interior (lo >= 0, lo + fine.n/2 <= coarse.n).
 * All fields are SoA [var][z][y][x] with ghosts, as everywhere else.
 * ---------------------------------------------------------------------- */

/* Restriction of conserved variables: every covered coarse interior cell of
 * coarse_field := mean of its 8 fine children in fine_field (the volume
 * mean, which conserves the integral).  nvar fields; nothing else changes. */
int grmhd_restrict(const grmhd_grid* coarse, double* coarse_field, const grmhd_grid* fine,
                   const double* fine_field, const int32_t lo[3], int32_t nvar, void* stream);

/* Prolongation of primitives: every fine point (ghosts_only != 0: the ghost
 * points only) := its coarse parent's value plus, per axis, the parent's
 * minmod-limited slope times the child's offset (-1/4 or +1/4 coarse cell);
 * the 8 children of a parent average to the parent.  coarse_field must have
 * its ghosts filled (the stencil of a fine ghost reaches coarse ghosts). */
int grmhd_prolongate(const grmhd_grid* coarse, const double* coarse_field, const grmhd_grid* fine,
                     double* fine_field, const int32_t lo[3], int32_t nvar, int32_t ghosts_only,
                     void* stream);

/* Flux restriction at the coarse-fine interface: for every coarse face on
 * the fine grid's boundary, the uncovered coarse cell beside it should see
 * the mean of the 4 fine face fluxes instead of the coarse face flux.  Adds
 * scale * (that change of its RHS) to coarse_out (8 fields), and, if acc is
 * not NULL, acc_scale * (the same change) to acc.  Face fluxes are those of
 * grmhd_rhs (params.recon, HLLE), computed from coarse_prim / fine_prim
 * (ghosts filled) and the metrics (NULL: Minkowski; both or neither). */
int grmhd_reflux(const grmhd_grid* coarse, const grmhd_params* params, const double* coarse_prim,
                 const double* coarse_metric, const grmhd_grid* fine, const double* fine_prim,
                 const double* fine_metric, const int32_t lo[3], double scale, double* coarse_out,
                 double acc_scale, double* acc, void* stream);

/* Device workspace (bytes) of grmhd_amr2_step; 0 if a grid is invalid. */
size_t grmhd_amr2_workspace_bytes(const grmhd_grid* coarse, int32_t nfine, const grmhd_grid* fine,
                                  int32_t scheme);

/* One composite step (FP64) of a coarse block and nfine fine blocks at the
 * next level: per RK stage, the fused RHS and stage update of every block,
 * flux restriction onto the coarse update, restriction of each fine U onto
 * its covered coarse cells, recovery on every block, then the coarse ghosts
 * by params.bc and every fine block's ghosts by prolongation.
 *   fine[nfine], fine_cons/fine_prim/fine_metric[nfine] (host arrays of
 *   device pointers; fine_metric entries NULL when coarse_metric is NULL),
 *   lo[3 * nfine] placements.  Fine grids must lie inside the coarse
 *   interior with a gap of at least one coarse cell to its boundary and to
 *   each other (the fine ghosts then come from the coarse level only).
 *   On entry the primitives of every block are consistent with its U and
 *   their ghosts filled (fine ghosts by grmhd_prolongate).
 *   ws: ws_bytes >= grmhd_amr2_workspace_bytes, 256-byte aligned; nfail as
 *   for grmhd_rk_step. */
int grmhd_amr2_step(const grmhd_grid* coarse, const grmhd_params* params, int32_t scheme, double dt,
                    double* coarse_cons, double* coarse_prim, const double* coarse_metric, int32_t nfine,
                    const grmhd_grid* fine, double* const* fine_cons, double* const* fine_prim,
                    const double* const* fine_metric, const int32_t* lo, void* ws, size_t ws_bytes,
                    int32_t* nfail, void* stream);

/* ----------------------------------------------------------------------
 * Constrained transport (Sec. 3: the magnetic field is evolved on staggered
 * grids so that its divergence stays zero).
 *
 * Face field bface [3][z][y][x] (ghosts included): component a holds the
 * densitised field sqrt(gamma) B^a on the lower a-face of each cell.  The
 * interior a-faces have a-index ng .. ng + n_a and interior transverse
 * indices; the step advances exactly those and reads no other entry.
 * Edge field: E_c at the c-edge through the corner of a cell that is lower
 * in a and b ((c, a, b) cyclic) is the mean of the four field fluxes of the
 * faces meeting there, E_c = (-F_a(B^b)[-e_b] - F_a(B^b) + F_b(B^a)[-e_a]
 * + F_b(B^a)) / 4, where F_d(B^a) is the B^a component of the HLLE flux of
 * grmhd_rhs on a lower d-face.  Face rate: dB^a/dt = -(E_c[+e_b] - E_c)/dx_b
 * + (E_b[+e_c] - E_b)/dx_c, (a, b, c) cyclic, which leaves the discrete
 * divergence sum_a (B^a[+e_a] - B^a)/dx_a of every cell unchanged.
 * The cell-centred field (conserved variables 5..7) is the mean of a cell's
 * two faces.
 * ---------------------------------------------------------------------- */

/* Bytes of the field-flux register and the edge fields (9 + 3 ncell
 * doubles, each part rounded up to 256 bytes); 0 if the grid is invalid. */
size_t grmhd_ct_flux_bytes(const grmhd_grid* grid);

/* Device workspace (bytes) of grmhd_ct_rk_step: the field-flux register and
 * edge fields (grmhd_ct_flux_bytes), the step-start face field, (RK4) a face-rate accumulator, then the
 * grmhd_rk_step workspace; the _cached size adds the geometry and primitive
 * caches that grmhd_rk_workspace_bytes_cached adds.  0 if invalid. */
size_t grmhd_ct_workspace_bytes(const grmhd_grid* grid, int32_t scheme);
size_t grmhd_ct_workspace_bytes_cached(const grmhd_grid* grid, int32_t scheme);

/* Face rate dB^a/dt of every interior face (the formula above) into rate
 * [3][ncell]; every other entry is set to 0.  prim has its ghosts filled;
 * metric/kij as for grmhd_rhs.  ws: device scratch of at least
 * grmhd_ct_flux_bytes, 256-byte aligned. */
int grmhd_ct_rate(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
                  const double* kij, double* rate, void* ws, size_t ws_bytes, void* stream);

/* One RK step (params precision) with constrained transport: the fluid
 * variables exactly as grmhd_rk_step, the interior faces of bface by the
 * same stage formulas with the face rate, and the field of cons (5..7) of
 * every interior cell replaced by the mean of its faces before each
 * recovery.  On entry prim is consistent with cons and has its ghosts
 * filled (its field normally the face mean).  ws >= grmhd_ct_workspace_bytes
 * (256-byte aligned; >= the _cached size takes the cached RHS paths as
 * grmhd_rk_step does).  Returns GRMHD_ERR_SIZE for a short workspace and
 * GRMHD_ERR_ARG for invalid arguments, before any launch. */
int grmhd_ct_rk_step(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt, double* cons,
                     double* prim, double* bface, const double* metric, const double* kij, void* ws,
                     size_t ws_bytes, int32_t* nfail, void* stream);

/* Cell-centred primitive field from the face field (the cell-centred
 * densitised field is the mean of a cell's two faces, as above): on every
 * interior cell prim[5 + a] := (bface[a] of the cell + bface[a] of the cell
 * above along a) / 2 / sqrt(gamma), sqrt(gamma) from the cell's metric (NULL:
 * 1).  Nothing else of prim is touched (fill the ghosts afterwards).  For
 * setting up a state whose cell field matches a given face field. */
int grmhd_ct_cell_field(const grmhd_grid* grid, const double* bface, const double* metric, double* prim,
                        void* stream);

/* Discrete divergence of the face field: div [ncell] (nullable) gets
 * sum_a (B^a[+e_a] - B^a)/dx_a on the interior cells and 0 elsewhere;
 * maxabs (nullable, one device double) the largest |div| (a NaN shows as
 * NaN).  At least one of div, maxabs. */
int grmhd_ct_divergence(const grmhd_grid* grid, const double* bface, double* div, double* maxabs, void* stream);

/* Human-readable name of a return code (static storage). */
const char* grmhd_error_string(int code);

/* Library version as 10000*major + 100*minor + patch. */
int grmhd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GRMHD_H */
