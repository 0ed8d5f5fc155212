// FP64 instantiations of the persistent batched RHS kernels.
#include "batch.cuh"

namespace grmhd {
cudaError_t launch_batch_rhs_fp64(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                  cudaStream_t s) {
  return launch_batch_rhs_t<double>(head, boxes, p, curved, nsm, s);
}
cudaError_t launch_batch_fused_fp64(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                    int32_t* nfail, int32_t* status, cudaStream_t s) {
  return launch_batch_fused_t<double>(head, boxes, p, curved, nsm, nfail, status, s);
}

// Multi-pass FP64 RHS over the table, then the per-cell pass (work counter
// 3).  With `three` (WENO5, every box with a state buffer): the state and face
// passes (counters 4 and 5); otherwise every face flux once into the boxes'
// face buffers by tiles in each box's shape (counter 0).
template <class K>
static cudaError_t launch_persistent(K k, BatchHead* head, const BoxDev* boxes, const DevParams& p, int threads,
                                     size_t smem, int nsm, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (smem) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k<<<nsm * per_sm, threads, smem, s>>>(head, boxes, p);
  return cudaGetLastError();
}

cudaError_t launch_batch_rhs_two_pass(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved,
                                      bool three, int nsm, cudaStream_t s) {
  cudaError_t e;
  if (three && p.recon == GRMHD_WENO5) {
    e = launch_persistent(batch_states_kernel<GRMHD_WENO5>, head, boxes, p, kBatchItem, 0, nsm, s);
    if (e != cudaSuccess) return e;
    e = launch_persistent(curved ? batch_face_kernel<true> : batch_face_kernel<false>, head, boxes, p, kBatchFaces, 0,
                          nsm, s);
    if (e != cudaSuccess) return e;
  } else {
    void (*k)(BatchHead*, const BoxDev*, DevParams) = nullptr;
    if (p.recon == GRMHD_WENO5)
      k = curved ? batch_faces_kernel<GRMHD_WENO5, true> : batch_faces_kernel<GRMHD_WENO5, false>;
    else
      k = curved ? batch_faces_kernel<GRMHD_MINMOD, true> : batch_faces_kernel<GRMHD_MINMOD, false>;
    const size_t smem = (size_t)16 *
                        (p.recon == GRMHD_WENO5 ? batch_stage_entries<double, GRMHD_WENO5>()
                                                : batch_stage_entries<double, GRMHD_MINMOD>()) *
                        sizeof(double);
    e = launch_persistent(k, head, boxes, p, kTileThreads, smem, nsm, s);
    if (e != cudaSuccess) return e;
  }
  return launch_persistent(curved ? batch_div_kernel<true> : batch_div_kernel<false>, head, boxes, p, kBatchItem, 0,
                           nsm, s);
}
}  // namespace grmhd
