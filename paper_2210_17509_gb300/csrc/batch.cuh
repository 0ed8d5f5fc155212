// Persistent kernels that sweep a table of independent boxes (many uneven
// AMR-like blocks) in one launch per phase: a work counter hands out items
// (chunks of cells, or RHS tiles with the box's own tile shape) to resident
// CTAs until the table is exhausted.  No CTA ever waits for another.  The
// one-launch form (batch_fused_kernel, at the end) runs the three phases in
// one kernel, ordered per box by completion counters.
#pragma once

#include "recovery.cuh"
#include "rhs.cuh"

namespace grmhd {

// Device copy of one box (built by grmhd_batch_prepare).
struct BoxDev {
  DevGrid g;
  double* cons;
  double* prim;
  const double* metric;
  double* rhs;
  double* faces;       // multi-pass face buffer (24 ncell doubles) or NULL
  double* states;      // WENO5 state buffer (48 ncell doubles) or NULL
  int tile, bc;
  int nt[3];           // tiles per axis for the box's tile shape
  long long tile_begin;  // first RHS work item of the box
  long long c2p_begin;   // first recovery item (256 interior cells each)
  long long gh_begin;    // first ghost-fill item (256 points each)
  long long st_begin;    // first state item (kBatchItem state items each)
  long long fc_begin;    // first face item (kBatchFaces faces each)
};

struct BatchHead {
  int nbox;
  int pad;
  long long ntiles, nc2p, ngh, nst, nfc;
  // work counters, zeroed before every run: tiles, recovery, ghosts, cells, states, faces
  unsigned long long counter[6];
};

constexpr int kBatchItem = 256;
constexpr int kBatchFaces = kFaceThreads;

// Workspace layout: the header (256 bytes, its work counters last), then the
// per-box completion counters of the one-launch form (kDonePhases x nbox,
// zeroed with the work counters by one memset), then the box table.
constexpr size_t kBatchHeadBytes = 256;
constexpr int kDonePhases = 2;
__host__ __device__ __forceinline__ size_t batch_done_bytes(long long nbox) {
  return ((size_t)kDonePhases * nbox * sizeof(unsigned) + 255) & ~(size_t)255;
}

// Bounded wait of the one-launch form: polls of a completion counter before
// it gives up (about 2 s at the back-off below).
constexpr long long kBatchWaitPolls = 1LL << 23;

// Box holding work item `it` (boxes sorted by ascending begin offsets).
template <int WHICH>
__device__ __forceinline__ int find_box(const BoxDev* __restrict__ boxes, int nbox, long long it) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const BoxDev& x = boxes[mid];
    const long long b = WHICH == 0   ? x.tile_begin
                        : WHICH == 1 ? x.c2p_begin
                        : WHICH == 2 ? x.gh_begin
                        : WHICH == 3 ? x.st_begin
                                     : x.fc_begin;
    if (b <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ long long next_item(unsigned long long* counter) {
  __shared__ long long s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
  __syncthreads();
  return s_item;
}

template <class T, int RECON, bool CURVED>
__global__ void __launch_bounds__(kTileThreads) batch_rhs_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                                 DevParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sR = sF + 8 * kMaxTileFaces;
  const int nbox = head->nbox;
  const long long total = head->ntiles;
  for (;;) {
    const long long it = next_item(&head->counter[0]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<0>(boxes, nbox, it)];
    const long long t = it - b.tile_begin;
    const int tx = (int)(t % b.nt[0]);
    const int ty = (int)((t / b.nt[0]) % b.nt[1]);
    const int tz = (int)(t / ((long long)b.nt[0] * b.nt[1]));
    StageEpilogue ep;
    ep.fb = nullptr;
    ep.faces = nullptr;
    ep.states = nullptr;
    ep.rhs = b.rhs;
    ep.u = nullptr;
    ep.u0 = nullptr;
    ep.acc_in = nullptr;
    ep.acc_out = nullptr;
    ep.c0 = ep.c1 = ep.cr = ep.ca = ep.wa = ep.wr = 0.0;
    const DevGrid g = b.g;
    SrcF64 src;
    src.prim = b.prim;
    src.metric = b.metric;
    src.kij = nullptr;
    switch (b.tile) {
      case 1:
        rhs_tile<T, RECON, CURVED, 16, 4, 4, SrcF64>(g, p, src, ep, tx * 16, ty * 4, tz * 4, sF, sR);
        break;
      case 2:
        rhs_tile<T, RECON, CURVED, 32, 4, 2, SrcF64>(g, p, src, ep, tx * 32, ty * 4, tz * 2, sF, sR);
        break;
      case 3:
        rhs_tile<T, RECON, CURVED, 4, 8, 8, SrcF64>(g, p, src, ep, tx * 4, ty * 8, tz * 8, sF, sR);
        break;
      default:
        rhs_tile<T, RECON, CURVED, 8, 8, 4, SrcF64>(g, p, src, ep, tx * 8, ty * 8, tz * 4, sF, sR);
        break;
    }
  }
}

// Two-pass FP64 RHS over the table.  Pass 1: every face flux of every box
// once, into the box's face buffer, tiles in the box's own shape.
template <int RECON, bool CURVED>
__global__ void __launch_bounds__(kTileThreads) batch_faces_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                                   DevParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sR = reinterpret_cast<double*>(smem_raw);  // the stage only
  const int nbox = head->nbox;
  const long long total = head->ntiles;
  for (;;) {
    const long long it = next_item(&head->counter[0]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<0>(boxes, nbox, it)];
    const long long t = it - b.tile_begin;
    const int tx = (int)(t % b.nt[0]);
    const int ty = (int)((t / b.nt[0]) % b.nt[1]);
    const int tz = (int)(t / ((long long)b.nt[0] * b.nt[1]));
    const DevGrid g = b.g;
    SrcF64 src;
    src.prim = b.prim;
    src.metric = b.metric;
    src.kij = nullptr;
    switch (b.tile) {
      case 1:
        faces_tile<double, RECON, CURVED, 16, 4, 4, SrcF64, false>(g, p, src, tx * 16, ty * 4, tz * 4, b.faces, nullptr,
                                                                   sR);
        break;
      case 2:
        faces_tile<double, RECON, CURVED, 32, 4, 2, SrcF64, false>(g, p, src, tx * 32, ty * 4, tz * 2, b.faces, nullptr,
                                                                   sR);
        break;
      case 3:
        faces_tile<double, RECON, CURVED, 4, 8, 8, SrcF64, false>(g, p, src, tx * 4, ty * 8, tz * 8, b.faces, nullptr,
                                                                  sR);
        break;
      default:
        faces_tile<double, RECON, CURVED, 8, 8, 4, SrcF64, false>(g, p, src, tx * 8, ty * 8, tz * 4, b.faces, nullptr,
                                                                  sR);
        break;
    }
    __syncthreads();  // the stage is reused by the next item
  }
}

// Three-pass FP64 WENO5 RHS over the table (every box with a state buffer):
// the state and face items of rhs.cuh, handed out in chunks per box.
template <int RECON>
__global__ void __launch_bounds__(kBatchItem) batch_states_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                                  DevParams p) {
  static_assert(RECON == GRMHD_WENO5, "the state pass is WENO5's");
  const int nbox = head->nbox;
  const long long total = head->nst;
  for (;;) {
    const long long it = next_item(&head->counter[4]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<3>(boxes, nbox, it)];
    const long long t = (it - b.st_begin) * kBatchItem + threadIdx.x;
    if (t < state_items(b.g)) {
      SrcF64 src;
      src.prim = b.prim;
      src.metric = b.metric;
      src.kij = nullptr;
      rhs_state_item<SrcF64>(b.g, p, src, b.states, t);
    }
  }
}

template <bool CURVED>
__global__ void __launch_bounds__(kBatchFaces) batch_face_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                                 DevParams p) {
  const int nbox = head->nbox;
  const long long total = head->nfc;
  for (;;) {
    const long long it = next_item(&head->counter[5]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<4>(boxes, nbox, it)];
    const long long t = (it - b.fc_begin) * kBatchFaces + threadIdx.x;
    if (t < face_items(b.g)) {
      SrcF64 src;
      src.prim = b.prim;
      src.metric = b.metric;
      src.kij = nullptr;
      rhs_face_item<CURVED, SrcF64, false>(b.g, p, src, b.states, b.faces, nullptr, t);
    }
  }
}

// Pass 2: the per-cell pass of every box into its rhs, in the recovery's
// items of kBatchItem interior cells.
template <bool CURVED>
__global__ void __launch_bounds__(kBatchItem) batch_div_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                               DevParams p) {
  const int nbox = head->nbox;
  const long long total = head->nc2p;
  for (;;) {
    const long long it = next_item(&head->counter[3]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<1>(boxes, nbox, it)];
    const long long nint = (long long)b.g.n[0] * b.g.n[1] * b.g.n[2];
    const long long t = (it - b.c2p_begin) * kBatchItem + threadIdx.x;
    if (t < nint) {
      StageEpilogue ep;
      ep.fb = nullptr;
      ep.faces = nullptr;
    ep.states = nullptr;
      ep.rhs = b.rhs;
      ep.u = nullptr;
      ep.u0 = nullptr;
      ep.acc_in = nullptr;
      ep.acc_out = nullptr;
      ep.c0 = ep.c1 = ep.cr = ep.ca = ep.wa = ep.wr = 0.0;
      SrcF64 src;
      src.prim = b.prim;
      src.metric = b.metric;
      src.kij = nullptr;
      div_cell<double, CURVED, SrcF64>(b.g, p, src, b.faces, interior_cell(b.g, t), ep);
    }
  }
}

template <class T>
cudaError_t launch_batch_rhs_t(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                               cudaStream_t s) {
  void (*k)(BatchHead*, const BoxDev*, DevParams) = nullptr;
  if (p.recon == GRMHD_WENO5)
    k = curved ? batch_rhs_kernel<T, GRMHD_WENO5, true> : batch_rhs_kernel<T, GRMHD_WENO5, false>;
  else
    k = curved ? batch_rhs_kernel<T, GRMHD_MINMOD, true> : batch_rhs_kernel<T, GRMHD_MINMOD, false>;
  const size_t smem = p.recon == GRMHD_WENO5 ? batch_smem_bytes<T, GRMHD_WENO5>() : batch_smem_bytes<T, GRMHD_MINMOD>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k<<<nsm * per_sm, kTileThreads, smem, s>>>(head, boxes, p);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// One launch for the whole batch: recovery, ghost fill and the one-pass RHS
// tiles of every box in a single persistent kernel.  One work counter hands
// out the items of all three phases in phase order (every recovery item,
// then every ghost item, then every tile).  When an item of box b depends on
// an earlier phase of box b (ghost fill on its recovery, the tiles on its
// ghost fill), the CTA waits until that phase's completion counter for b has
// counted all its items.  Every item waited on was handed out earlier, to a
// CTA that is running it and that waits only on items handed out earlier
// still, so the waits always end; each wait is bounded all the same (on
// giving up the kernel records GRMHD_ERR_TIMEOUT in *status and carries on).
// Data written in the launch (the recovered and ghost-filled primitives)
// are read through L2 (SrcF64Co, fill_ghost_at<..., true>); a finished item
// publishes its writes with a fence before it counts itself.
__device__ __forceinline__ void batch_item_done(unsigned* counter) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
  }
}

__device__ __forceinline__ void batch_wait(const unsigned* counter, unsigned need, int32_t* status) {
  if (threadIdx.x == 0) {
    long long polls = 0;
    while (*(volatile const unsigned*)counter < need) {
      if (++polls > kBatchWaitPolls) {
        if (status) atomicExch(status, GRMHD_ERR_TIMEOUT);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
  }
  __syncthreads();
}

// Items of box k in a phase whose begin offsets are `begin` (ascending over
// the sorted table), the last box ending at `total`.
template <int WHICH>
__device__ __forceinline__ unsigned batch_box_items(const BoxDev* __restrict__ boxes, int nbox, int k,
                                                    long long total) {
  auto begin = [&](int j) { return WHICH == 1 ? boxes[j].c2p_begin : boxes[j].gh_begin; };
  return (unsigned)((k + 1 < nbox ? begin(k + 1) : total) - begin(k));
}

// Resident CTAs per SM the one-launch kernel's registers are fitted to: the
// FP32 tiles' 3 on flat boxes; 2 on curved ones, where the recovery's FP64
// metric algebra would spill at the tiles' budget; 1 in FP64, whose WENO5
// tiles fill the shared memory of an SM.
template <class T, bool CURVED>
struct FusedMinCtas { static constexpr int value = sizeof(T) == 4 ? (CURVED ? 2 : 3) : 1; };

template <class T, int RECON, bool CURVED>
__global__ void __launch_bounds__(kTileThreads, FusedMinCtas<T, CURVED>::value) batch_fused_kernel(BatchHead* head,
                                                                                      const BoxDev* __restrict__ boxes,
                                                                                      DevParams p, int32_t* nfail,
                                                                                      int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sR = sF + 8 * kMaxTileFaces;
  const int nbox = head->nbox;
  unsigned* done_c2p = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(head) + kBatchHeadBytes);
  unsigned* done_gh = done_c2p + nbox;
  const long long n0 = head->nc2p, n1 = head->ngh, total = n0 + n1 + head->ntiles;
  int myfail = 0;
  for (;;) {
    const long long it = next_item(&head->counter[0]);
    if (it >= total) break;
    if (it < n0) {
      const int k = find_box<1>(boxes, nbox, it);
      const BoxDev& b = boxes[k];
      const long long nint = (long long)b.g.n[0] * b.g.n[1] * b.g.n[2];
      const long long t = (it - b.c2p_begin) * kBatchItem + threadIdx.x;
      if (t < nint) {
        const long long c = interior_cell(b.g, t);
        // the FP32 kernel serves the mixed path, the FP64 kernel the FP64 path
        int st;
        if constexpr (sizeof(T) == 4) st = con2prim_at<true, false>(b.g, p, b.cons, b.metric, b.prim, c);
        else st = con2prim_at<false>(b.g, p, b.cons, b.metric, b.prim, c);
        myfail += (st >= 2);
      }
      batch_item_done(&done_c2p[k]);
    } else if (it < n0 + n1) {
      const long long i1 = it - n0;
      const int k = find_box<2>(boxes, nbox, i1);
      const BoxDev& b = boxes[k];
      batch_wait(&done_c2p[k], batch_box_items<1>(boxes, nbox, k, n0), status);
      const long long c = (i1 - b.gh_begin) * kBatchItem + threadIdx.x;
      if (c < b.g.ncell) fill_ghost_at<double, true>(b.g, b.bc, 8, b.prim, c);
      batch_item_done(&done_gh[k]);
    } else {
      const long long i2 = it - n0 - n1;
      const int k = find_box<0>(boxes, nbox, i2);
      const BoxDev& b = boxes[k];
      batch_wait(&done_gh[k], batch_box_items<2>(boxes, nbox, k, n1), status);
      const long long t = i2 - b.tile_begin;
      const int tx = (int)(t % b.nt[0]);
      const int ty = (int)((t / b.nt[0]) % b.nt[1]);
      const int tz = (int)(t / ((long long)b.nt[0] * b.nt[1]));
      StageEpilogue ep;
      ep.fb = nullptr;
      ep.faces = nullptr;
      ep.states = nullptr;
      ep.rhs = b.rhs;
      ep.u = nullptr;
      ep.u0 = nullptr;
      ep.acc_in = nullptr;
      ep.acc_out = nullptr;
      ep.c0 = ep.c1 = ep.cr = ep.ca = ep.wa = ep.wr = 0.0;
      SrcF64Co src;
      src.prim = b.prim;
      src.metric = b.metric;
      src.kij = nullptr;
      switch (b.tile) {
        case 1:
          rhs_tile<T, RECON, CURVED, 16, 4, 4, SrcF64Co>(b.g, p, src, ep, tx * 16, ty * 4, tz * 4, sF, sR);
          break;
        case 2:
          rhs_tile<T, RECON, CURVED, 32, 4, 2, SrcF64Co>(b.g, p, src, ep, tx * 32, ty * 4, tz * 2, sF, sR);
          break;
        case 3:
          rhs_tile<T, RECON, CURVED, 4, 8, 8, SrcF64Co>(b.g, p, src, ep, tx * 4, ty * 8, tz * 8, sF, sR);
          break;
        default:
          rhs_tile<T, RECON, CURVED, 8, 8, 4, SrcF64Co>(b.g, p, src, ep, tx * 8, ty * 8, tz * 4, sF, sR);
          break;
      }
    }
  }
  if (nfail && myfail) atomicAdd(nfail, myfail);
}

template <class T>
cudaError_t launch_batch_fused_t(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                 int32_t* nfail, int32_t* status, cudaStream_t s) {
  void (*k)(BatchHead*, const BoxDev*, DevParams, int32_t*, int32_t*) = nullptr;
  if (p.recon == GRMHD_WENO5)
    k = curved ? batch_fused_kernel<T, GRMHD_WENO5, true> : batch_fused_kernel<T, GRMHD_WENO5, false>;
  else
    k = curved ? batch_fused_kernel<T, GRMHD_MINMOD, true> : batch_fused_kernel<T, GRMHD_MINMOD, false>;
  const size_t smem = p.recon == GRMHD_WENO5 ? batch_smem_bytes<T, GRMHD_WENO5>() : batch_smem_bytes<T, GRMHD_MINMOD>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k<<<nsm * per_sm, kTileThreads, smem, s>>>(head, boxes, p, nfail, status);
  return cudaGetLastError();
}

}  // namespace grmhd
