// Internal host/device declarations of libgrmhd (not part of the C ABI).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "grmhd.h"

namespace grmhd {

// Block geometry with the derived strides the kernels use.
struct DevGrid {
  int n[3];        // interior cells
  int ng;          // ghost width
  int N[3];        // points per axis incl. ghosts
  long long sy;    // stride of y (= N[0])
  long long sz;    // stride of z (= N[0] * N[1])
  long long ncell; // N[0] * N[1] * N[2]
  double dx[3];
  double idx[3];   // 1 / dx
  float idxf[3];   // 1 / dx rounded to FP32 (the FP32 kernels' copy)
};

// Method parameters with constants folded on the host.
struct DevParams {
  double gamma;
  double gfac;     // Gamma / (Gamma - 1): rho h = rho + gfac P
  double gm1g;     // (Gamma - 1) / Gamma
  double rho_atm, p_atm;
  double nr_tol;
  double weno_eps;
  int nr_maxit;
  int recon, bc, precision;
  int tile;        // RHS tile shape index (0..3)
  int flags;       // GRMHD_REUSE_GEOMETRY, ...
  int eos;         // GRMHD_EOS_IDEAL | GRMHD_EOS_POLYTROPE
  double poly_K;   // K of P = K rho^gamma (polytrope)
  int poly_g2;     // polytrope with gamma == 2: K rho^(gamma - 1) = K rho, no pow
  // FP32 copies for the FP32 kernels, rounded once on the host (the same
  // bits as a conversion in the kernel, without its FP64-pipe instruction)
  float gammaf, gfacf, weno_epsf, eps13f, gm1gf, rho_atmf, p_atmf;
};

// A parameter in the kernel's arithmetic type: the FP32 copy for float.
template <class T>
__host__ __device__ __forceinline__ T par_t(double d, float f) {
  if constexpr (sizeof(T) == 4) return f; else return (T)d;
}

// What the RHS kernel does with the RHS value r of each interior cell:
//   rhs     != NULL: rhs[cell] = r
//   u       != NULL: u[cell] = c0 * u0[cell] + c1 * u[cell] + cr * r
//                              (+ ca * acc_in[cell] if acc_in != NULL)
//   acc_out != NULL: acc_out[cell] = wr * r (+ wa * acc_in[cell] if acc_in != NULL)
//   fb      != NULL: fb[(3 d + a) * ncell + cell] = the flux of the field
//                    component B^a (a != d) through the lower d-face of the cell, for
//                    the d-faces 0 .. n_d with transverse indices -1 .. n
//                    (the tiles, then a ring kernel; constrained transport)
//   faces   != NULL: (FP64 with the geometry cache) device scratch of
//                    24 ncell doubles; the RHS then runs in several passes,
//                    every face flux computed once into it (rhs.cuh)
//   states  != NULL: (with faces, WENO5) 48 ncell doubles for the face states
//                    of every cell, computed once per cell and direction
// u0 must be valid whenever u is set.
struct StageEpilogue {
  double* rhs;
  double* fb;
  double* faces;
  double* states;
  double* u;
  const double* u0;
  const double* acc_in;
  double* acc_out;
  double c0, c1, cr, ca, wa, wr;
};

DevGrid make_grid(const grmhd_grid& g);
DevParams make_params(const grmhd_params& p);

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_rhs_fp64(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                            const double* kij, const StageEpilogue& ep, cudaStream_t s);
cudaError_t launch_rhs_mixed(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                             const double* kij, const StageEpilogue& ep, cudaStream_t s);
cudaError_t launch_con2prim(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                            double* prim, int8_t* status, int32_t* nfail, cudaStream_t s);
cudaError_t launch_prim2con(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                            double* cons, cudaStream_t s);
cudaError_t launch_fill_ghosts(const DevGrid& g, int bc, int nvar, double* field, cudaStream_t s);
// Fast mixed path: FP32 primitive copy and the FP64-computed geometry cache
// (geom32 nullable); result64 = false writes the FP32 primitives only.
cudaError_t launch_con2prim_mixed(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                                  double* prim, float* prim32, const double* mcache, const float* geom32,
                                  bool result64, int32_t* nfail, cudaStream_t s);
// Ghost fill of the FP32 primitive pairs (nvar variables, nvar even, in the
// [q/2][ncell] float2 layout of launch_prim_to_f32_pairs).
cudaError_t launch_fill_ghosts_f32(const DevGrid& g, int bc, int nvar, float* field, cudaStream_t s);
// FP32 copy of the primitives [8][ncell] in pairs: [q/2][ncell] float2.
cudaError_t launch_prim_to_f32_pairs(long long ncell, const double* prim, float* prim32, cudaStream_t s);
cudaError_t launch_geom_cache(const DevGrid& g, const double* metric, void* geom, bool fp64, double* mcache,
                              cudaStream_t s);
cudaError_t launch_con2prim_cached(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                                   const double* mcache, double* prim, int32_t* nfail, cudaStream_t s);
cudaError_t launch_rhs_fp64_cached(const DevGrid& g, const DevParams& p, const double* prim, const double* geom64,
                                   const double* kij, const StageEpilogue& ep, cudaStream_t s);
cudaError_t launch_rhs_mixed_cached(const DevGrid& g, const DevParams& p, const float* prim32, const float* geom,
                                    const double* kij, bool curved, const StageEpilogue& ep, cudaStream_t s);
constexpr int kGeomCacheComps = 108; // geometry cache components (layout in rhs.cuh)
constexpr int kGeomCacheFace = 53;   // FP64 cache: first of the 3 x 10 face-metric components
constexpr int kGeomCacheFaceIa = 83; // FP64 cache: first of the 3 face 1/alpha components
constexpr int kGeomCacheHalf32 = 53; // FP32 cache: first of the ten half-metric components
constexpr int kGeomCacheStat = 86;   // FP64 cache: first of the 22 metric factors of the sources
constexpr int kMetricCacheComps = 7;

// ---------------------------------------------------------- host helpers
inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

inline int check_grid(const grmhd_grid* g, int min_ng) {
  if (!g) return GRMHD_ERR_ARG;
  if (g->ng < min_ng || g->ng > 16) return GRMHD_ERR_ARG;
  long long cells = 1;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 1 || g->n[d] > (1 << 20)) return GRMHD_ERR_ARG;
    if (!(g->dx[d] > 0.0) || !std::isfinite(g->dx[d])) return GRMHD_ERR_ARG;
    cells *= (long long)(g->n[d] + 2 * g->ng);
    if (cells > (1LL << 40)) return GRMHD_ERR_ARG;
  }
  return GRMHD_OK;
}

inline int check_params(const grmhd_params* p) {
  if (!p) return GRMHD_ERR_ARG;
  if (!(p->gamma > 1.0 && p->gamma <= 3.0)) return GRMHD_ERR_ARG;
  if (p->recon != GRMHD_MINMOD && p->recon != GRMHD_WENO5) return GRMHD_ERR_ARG;
  if (p->bc != GRMHD_BC_PERIODIC && p->bc != GRMHD_BC_COPY) return GRMHD_ERR_ARG;
  if (p->precision != GRMHD_FP64 && p->precision != GRMHD_MIXED) return GRMHD_ERR_ARG;
  if (p->nr_maxit < 1 || p->nr_maxit > 1000) return GRMHD_ERR_ARG;
  if (!(p->nr_tol > 0.0 && p->nr_tol < 1.0)) return GRMHD_ERR_ARG;
  if (!(p->weno_eps > 0.0) || !std::isfinite(p->weno_eps)) return GRMHD_ERR_ARG;
  if (!(p->rho_atm > 0.0) || !(p->p_atm > 0.0)) return GRMHD_ERR_ARG;
  if (p->tile < 0 || p->tile > 4) return GRMHD_ERR_ARG;
  if ((p->flags & ~(GRMHD_REUSE_GEOMETRY | GRMHD_NEWMAN_HAMLIN | GRMHD_SINGLE_PASS | GRMHD_DETERMINISTIC)) != 0)
    return GRMHD_ERR_ARG;
  if (p->eos != GRMHD_EOS_IDEAL && p->eos != GRMHD_EOS_POLYTROPE) return GRMHD_ERR_ARG;
  if (p->eos == GRMHD_EOS_POLYTROPE && !(p->poly_K > 0.0 && std::isfinite(p->poly_K))) return GRMHD_ERR_ARG;
  return GRMHD_OK;
}

// Ghost width the stencils need: WENO5 reads 3 cells, minmod 2, the metric
// derivatives 2.
inline int min_ghosts(const grmhd_params* p, const double* metric) {
  int m = (p->recon == GRMHD_WENO5) ? 3 : 2;
  if (metric && m < 2) m = 2;
  return m;
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA; }

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

inline StageEpilogue no_epilogue() {
  StageEpilogue e;
  e.rhs = nullptr;
  e.fb = nullptr;
  e.faces = nullptr;
  e.states = nullptr;
  e.u = nullptr;
  e.u0 = nullptr;
  e.acc_in = nullptr;
  e.acc_out = nullptr;
  e.c0 = e.c1 = e.cr = e.ca = e.wa = e.wr = 0.0;
  return e;
}

// Stage coefficients of the integrators (reading R10): stage k sets
// u <- c0 u0 + c1 u + cr L (+ ca acc) and acc <- wa acc + wr L; RK2 = SSP
// Heun, RK3 = SSP Shu-Osher, RK4 = classical.  Returns the stage count.
struct RkStage {
  double c0, c1, cr, ca, wa, wr;
  bool acc_in, acc_out;
};

inline int rk_stages(int scheme, double dt, RkStage st[4]) {
  if (scheme == GRMHD_RK2) {
    st[0] = {1.0, 0.0, dt, 0, 0, 0, false, false};
    st[1] = {0.5, 0.5, 0.5 * dt, 0, 0, 0, false, false};
    return 2;
  }
  if (scheme == GRMHD_RK3) {
    st[0] = {1.0, 0.0, dt, 0, 0, 0, false, false};
    st[1] = {0.75, 0.25, 0.25 * dt, 0, 0, 0, false, false};
    st[2] = {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt, 0, 0, 0, false, false};
    return 3;
  }
  st[0] = {1.0, 0.0, 0.5 * dt, 0, 0, 1.0, false, true};
  st[1] = {1.0, 0.0, 0.5 * dt, 0, 1.0, 2.0, true, true};
  st[2] = {1.0, 0.0, dt, 0, 1.0, 2.0, true, true};
  st[3] = {1.0, 0.0, dt / 6.0, dt / 6.0, 0, 0, true, false};
  return 4;
}

// Constrained transport (ct.cu); layouts of the face field b [3][ncell] and
// of the field face fluxes fb [9][ncell] as in grmhd.h.
struct CtStep {
  double* fb;        // field face fluxes (filled by the RHS launch)
  double* E;         // edge fields [3][ncell]
  double* b;         // face field, advanced in place
  const double* b0;  // face field at the start of the step
  double* acc;       // RK4 accumulator of the face rates (NULL otherwise)
};
// Edge fields from fb into E [3][ncell], then the face rates / stage update.
cudaError_t launch_ct_faces(const DevGrid& g, const double* fb, double* E, double* rate, double* b, const double* b0,
                            const double* acc_in, double* acc_out, double c0, double c1, double cr, double ca,
                            double wa, double wr, cudaStream_t s);
cudaError_t launch_ct_face_to_cell(const DevGrid& g, const double* b, double* cons, cudaStream_t s);
cudaError_t launch_ct_divergence(const DevGrid& g, const double* b, double* div, double* maxabs, cudaStream_t s);
cudaError_t launch_ct_cell_field(const DevGrid& g, const double* b, const double* metric, double* prim,
                                 cudaStream_t s);

// Two-level AMR transfer (amr.cu).
cudaError_t launch_restrict(const DevGrid& c, double* coarse, const DevGrid& f, const double* fine, const int lo[3],
                            int nvar, cudaStream_t s);
cudaError_t launch_prolongate(const DevGrid& c, const double* coarse, const DevGrid& f, double* fine,
                              const int lo[3], int nvar, bool ghosts_only, cudaStream_t s);
cudaError_t launch_reflux(const DevGrid& c, const DevParams& p, const double* cprim, const double* cmetric,
                          const DevGrid& f, const double* fprim, const double* fmetric, const int lo[3],
                          double scale, double* out, double acc_scale, double* acc, cudaStream_t s);

}  // namespace grmhd
