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

}  // namespace grmhd
