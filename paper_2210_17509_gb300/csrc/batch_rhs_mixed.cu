// Mixed-precision instantiations of the persistent batched RHS kernel and of the one-launch batch.
#include "batch.cuh"

namespace grmhd {
cudaError_t launch_batch_rhs_mixed(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                   cudaStream_t s) {
  return launch_batch_rhs_t<float>(head, boxes, p, curved, nsm, s);
}
cudaError_t launch_batch_fused_mixed(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                     int32_t* nfail, int32_t* status, cudaStream_t s) {
  return launch_batch_fused_t<float>(head, boxes, p, curved, nsm, nfail, status, s);
}
}  // namespace grmhd
