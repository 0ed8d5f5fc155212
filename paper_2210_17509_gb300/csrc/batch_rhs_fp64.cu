// FP64 instantiations of the persistent batched RHS kernels.
#include "batch.cuh"

namespace grmhd {
cudaError_t launch_batch_rhs_fp64(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                  cudaStream_t s) {
  return launch_batch_rhs_t<double>(head, boxes, p, curved, nsm, s);
}

// Two passes: every face flux once into the boxes' face buffers, then the
// per-cell pass (work counters 0 and 3).
cudaError_t launch_batch_rhs_two_pass(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                      cudaStream_t s) {
  void (*k)(BatchHead*, const BoxDev*, DevParams) = nullptr;
  if (p.recon == GRMHD_WENO5)
    k = curved ? batch_faces_kernel<GRMHD_WENO5, true> : batch_faces_kernel<GRMHD_WENO5, false>;
  else
    k = curved ? batch_faces_kernel<GRMHD_MINMOD, true> : batch_faces_kernel<GRMHD_MINMOD, false>;
  const size_t smem = (size_t)16 *
                      (p.recon == GRMHD_WENO5 ? batch_stage_entries<double, GRMHD_WENO5>()
                                              : batch_stage_entries<double, GRMHD_MINMOD>()) *
                      sizeof(double);
  cudaError_t e = cudaSuccess;
  if (smem) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k<<<nsm * per_sm, kTileThreads, smem, s>>>(head, boxes, p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  void (*kd)(BatchHead*, const BoxDev*, DevParams) = curved ? batch_div_kernel<true> : batch_div_kernel<false>;
  per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kd, kBatchItem, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  kd<<<nsm * per_sm, kBatchItem, 0, s>>>(head, boxes, p);
  return cudaGetLastError();
}
}  // namespace grmhd
