// FP64 instantiation of the fused RHS kernel (the plain method).
#include "rhs.cuh"

namespace grmhd {

cudaError_t launch_rhs_fp64(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                            const double* kij, const StageEpilogue& ep, cudaStream_t s) {
  return launch_rhs_t<double>(g, p, prim, metric, kij, ep, s);
}

cudaError_t launch_rhs_fp64_cached(const DevGrid& g, const DevParams& p, const double* prim, const double* geom64,
                                   const double* kij, const StageEpilogue& ep, cudaStream_t s) {
  SrcCache64 src;
  src.prim = prim;
  src.geom = geom64;
  src.kij = kij;
  return launch_rhs_src<double, SrcCache64>(g, p, src, true, ep, s);
}

}  // namespace grmhd
