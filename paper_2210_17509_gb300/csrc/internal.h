// Internal host/device declarations of libgrmhd (not part of the C ABI).
#pragma once

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
};

// What the RHS kernel does with the RHS value r of each interior cell:
//   rhs     != NULL: rhs[cell] = r
//   u       != NULL: u[cell] = c0 * u0[cell] + c1 * u[cell] + cr * r
//                              (+ ca * acc_in[cell] if acc_in != NULL)
//   acc_out != NULL: acc_out[cell] = wr * r (+ wa * acc_in[cell] if acc_in != NULL)
// u0 must be valid whenever u is set.
struct StageEpilogue {
  double* rhs;
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
cudaError_t launch_fill_ghosts_f32(const DevGrid& g, int bc, int nvar, float* field, cudaStream_t s);
cudaError_t launch_to_f32(long long n, const double* a, float* b, cudaStream_t s);
cudaError_t launch_geom_cache(const DevGrid& g, const double* metric, void* geom, bool fp64, double* mcache,
                              cudaStream_t s);
cudaError_t launch_con2prim_cached(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                                   const double* mcache, double* prim, int32_t* nfail, cudaStream_t s);
cudaError_t launch_rhs_fp64_cached(const DevGrid& g, const DevParams& p, const double* prim, const double* geom64,
                                   const double* kij, const StageEpilogue& ep, cudaStream_t s);
cudaError_t launch_rhs_mixed_cached(const DevGrid& g, const DevParams& p, const float* prim32, const float* geom,
                                    const double* kij, bool curved, const StageEpilogue& ep, cudaStream_t s);
constexpr int kGeomCacheComps = 53;
constexpr int kMetricCacheComps = 7;

}  // namespace grmhd
