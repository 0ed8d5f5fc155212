// Mixed-precision instantiation of the persistent batched RHS kernel.
#include "batch.cuh"

namespace grmhd {
cudaError_t launch_batch_rhs_mixed(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                   cudaStream_t s) {
  return launch_batch_rhs_t<float>(head, boxes, p, curved, nsm, s);
}
}  // namespace grmhd
