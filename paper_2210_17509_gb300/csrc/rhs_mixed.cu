// Mixed-precision instantiation of the fused RHS kernel: reconstruction,
// Riemann fluxes, divergence and source contraction in FP32; the face and
// cell sqrt(gamma) and metric inverse in FP64 (see face_geom/source_terms);
// the stage epilogue accumulates in FP64.
#include "rhs.cuh"

namespace grmhd {

cudaError_t launch_rhs_mixed(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                             const double* kij, const StageEpilogue& ep, cudaStream_t s) {
  return launch_rhs_t<float>(g, p, prim, metric, kij, ep, s);
}

cudaError_t launch_rhs_mixed_cached(const DevGrid& g, const DevParams& p, const float* prim32, const float* geom,
                                    const double* kij, bool curved, const StageEpilogue& ep, cudaStream_t s) {
  SrcCache src;
  src.prim = prim32;
  src.geom = geom;
  src.kij = kij;
  return launch_rhs_src<float, SrcCache>(g, p, src, curved, ep, s);
}

}  // namespace grmhd
