// Batched boxes: host side of grmhd_batch_prepare / grmhd_batch_rhs.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "batch.cuh"

namespace grmhd {
cudaError_t launch_batch_rhs_fp64(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                  cudaStream_t s);
cudaError_t launch_batch_rhs_mixed(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                   cudaStream_t s);
cudaError_t launch_batch_rhs_two_pass(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved,
                                      bool three, int nsm, cudaStream_t s);
cudaError_t launch_batch_fused_fp64(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                    int32_t* nfail, int32_t* status, cudaStream_t s);
cudaError_t launch_batch_fused_mixed(BatchHead* head, const BoxDev* boxes, const DevParams& p, bool curved, int nsm,
                                     int32_t* nfail, int32_t* status, cudaStream_t s);
__global__ void __launch_bounds__(kBatchItem) batch_con2prim_kernel(BatchHead* head, const BoxDev* __restrict__ boxes,
                                                                    DevParams p, int32_t* nfail) {
  int myfail = 0;
  const int nbox = head->nbox;
  const long long total = head->nc2p;
  for (;;) {
    const long long it = next_item(&head->counter[1]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<1>(boxes, nbox, it)];
    const long long nint = (long long)b.g.n[0] * b.g.n[1] * b.g.n[2];
    const long long t = (it - b.c2p_begin) * kBatchItem + threadIdx.x;
    if (t < nint) {
      const long long c = interior_cell(b.g, t);
      // mixed precision: FP32 Newton predictor, then the FP64 Newton
      const int st = p.precision == GRMHD_MIXED ? con2prim_at<true, false>(b.g, p, b.cons, b.metric, b.prim, c)
                                                : con2prim_at<false>(b.g, p, b.cons, b.metric, b.prim, c);
      myfail += (st >= 2);
    }
  }
  if (nfail && myfail) atomicAdd(nfail, myfail);
}

__global__ void __launch_bounds__(kBatchItem) batch_ghost_kernel(BatchHead* head, const BoxDev* __restrict__ boxes) {
  const int nbox = head->nbox;
  const long long total = head->ngh;
  for (;;) {
    const long long it = next_item(&head->counter[2]);
    if (it >= total) break;
    const BoxDev& b = boxes[find_box<2>(boxes, nbox, it)];
    const long long c = (it - b.gh_begin) * kBatchItem + threadIdx.x;
    if (c < b.g.ncell) fill_ghost_at(b.g, b.bc, 8, b.prim, c);
  }
}

}  // namespace grmhd

using namespace grmhd;

namespace {

constexpr size_t kHeadBytes = kBatchHeadBytes;
static_assert(sizeof(BatchHead) <= kHeadBytes, "batch header too large");

// The box table sits after the header and the completion counters.
size_t box_table_offset(int32_t nbox) { return kHeadBytes + batch_done_bytes(nbox); }

const int kShape[4][3] = {{8, 8, 4}, {16, 4, 4}, {32, 4, 2}, {4, 8, 8}};


}  // namespace

extern "C" {

size_t grmhd_batch_workspace_bytes(int32_t nbox) {
  if (nbox < 1 || nbox > (1 << 22)) return 0;
  return box_table_offset(nbox) + (((size_t)nbox * sizeof(BoxDev) + 255) & ~(size_t)255);
}

int grmhd_batch_prepare(const grmhd_box* boxes, int32_t nbox, const grmhd_params* params, void* ws,
                        size_t ws_bytes, grmhd_batch* batch, void* stream) {
  if (!boxes || !params || !ws || !batch || nbox < 1) return GRMHD_ERR_ARG;
  if (params->eos != GRMHD_EOS_IDEAL) return GRMHD_ERR_ARG;  // batched boxes: Gamma-law only
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  const size_t need = grmhd_batch_workspace_bytes(nbox);
  if (need == 0) return GRMHD_ERR_ARG;
  if (ws_bytes < need) return GRMHD_ERR_SIZE;
  const int min_ng = params->recon == GRMHD_WENO5 ? 3 : 2;
  std::vector<BoxDev> host(nbox);
  int ncurved = 0, nfaces = 0, nstates = 0;
  for (int b = 0; b < nbox; ++b) {
    const grmhd_box& x = boxes[b];
    const grmhd_grid& gr = x.grid;
    if (gr.ng < min_ng || gr.ng > 16) return GRMHD_ERR_ARG;
    for (int d = 0; d < 3; ++d)
      if (gr.n[d] < 1 || gr.n[d] > (1 << 16) || !(gr.dx[d] > 0.0) || !std::isfinite(gr.dx[d])) return GRMHD_ERR_ARG;
    if (!x.cons || !x.prim || !x.rhs || !aligned8(x.cons) || !aligned8(x.prim) || !aligned8(x.rhs))
      return GRMHD_ERR_ARG;
    if (x.metric && !aligned8(x.metric)) return GRMHD_ERR_ARG;
    if (x.faces && !aligned8(x.faces)) return GRMHD_ERR_ARG;
    if (x.states && (!aligned8(x.states) || !x.faces)) return GRMHD_ERR_ARG;
    nfaces += x.faces != nullptr;
    nstates += x.states != nullptr;
    if (x.tile < 0 || x.tile > 3) return GRMHD_ERR_ARG;
    if (x.bc != GRMHD_BC_PERIODIC && x.bc != GRMHD_BC_COPY) return GRMHD_ERR_ARG;
    ncurved += x.metric != nullptr;
    BoxDev& h = host[b];
    h.g = make_grid(gr);
    h.cons = x.cons;
    h.prim = x.prim;
    h.metric = x.metric;
    h.rhs = x.rhs;
    h.faces = x.faces;
    h.states = x.states;
    h.tile = x.tile;
    h.bc = x.bc;
    for (int d = 0; d < 3; ++d) h.nt[d] = (gr.n[d] + kShape[x.tile][d] - 1) / kShape[x.tile][d];
  }
  if (ncurved != 0 && ncurved != nbox) return GRMHD_ERR_ARG;  // one kernel variant per batch
  if (nfaces != 0 && nfaces != nbox) return GRMHD_ERR_ARG;    // two passes for all boxes or none
  if (nstates != 0 && nstates != nbox) return GRMHD_ERR_ARG;  // three passes for all boxes or none
  // Largest boxes first (longest-processing-time order) so the dynamic work
  // counter finishes with small items.
  std::vector<int> order(nbox);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int b) { return (long long)host[b].nt[0] * host[b].nt[1] * host[b].nt[2]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<BoxDev> sorted(nbox);
  long long tiles = 0, c2p = 0, gh = 0, st = 0, fc = 0;
  for (int k = 0; k < nbox; ++k) {
    BoxDev h = host[order[k]];
    h.tile_begin = tiles;
    h.c2p_begin = c2p;
    h.gh_begin = gh;
    h.st_begin = st;
    h.fc_begin = fc;
    tiles += work(order[k]);
    if (h.states) {
      st += (state_items(h.g) + kBatchItem - 1) / kBatchItem;
      fc += (face_items(h.g) + kBatchFaces - 1) / kBatchFaces;
    }
    const long long nint = (long long)h.g.n[0] * h.g.n[1] * h.g.n[2];
    c2p += (nint + kBatchItem - 1) / kBatchItem;
    gh += (h.g.ncell + kBatchItem - 1) / kBatchItem;
    sorted[k] = h;
  }
  BatchHead head;
  head.nbox = nbox;
  head.pad = 0;
  head.ntiles = tiles;
  head.nc2p = c2p;
  head.ngh = gh;
  head.nst = st;
  head.nfc = fc;
  for (int i = 0; i < 6; ++i) head.counter[i] = 0;
  cudaStream_t s = (cudaStream_t)stream;
  // Host sources are pageable: the calls return once the data are staged.
  if (cudaMemcpyAsync(ws, &head, sizeof(head), cudaMemcpyHostToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaMemcpyAsync(static_cast<char*>(ws) + box_table_offset(nbox), sorted.data(), (size_t)nbox * sizeof(BoxDev),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GRMHD_ERR_CUDA;
  batch->ws = ws;
  batch->ws_bytes = ws_bytes;
  batch->nbox = nbox;
  batch->curved = ncurved > 0;
  batch->ntiles = tiles;
  batch->nc2p_items = c2p;
  batch->nghost_items = gh;
  batch->two_pass = nfaces == nbox;
  batch->three_pass = nstates == nbox;
  return GRMHD_OK;
}

int grmhd_batch_rhs(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail, void* stream) {
  if (!batch || !params || !batch->ws || batch->nbox < 1) return GRMHD_ERR_ARG;
  if (params->eos != GRMHD_EOS_IDEAL) return GRMHD_ERR_ARG;  // batched boxes: Gamma-law only
  if (params->recon != GRMHD_WENO5 && params->recon != GRMHD_MINMOD) return GRMHD_ERR_ARG;
  if (params->precision != GRMHD_FP64 && params->precision != GRMHD_MIXED) return GRMHD_ERR_ARG;
  if (!(params->gamma > 1.0 && params->gamma <= 3.0) || params->nr_maxit < 1 || !(params->nr_tol > 0.0))
    return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  BatchHead* head = static_cast<BatchHead*>(batch->ws);
  const BoxDev* boxes =
      reinterpret_cast<const BoxDev*>(static_cast<char*>(batch->ws) + box_table_offset(batch->nbox));
  const DevParams p = make_params(*params);
  if (cudaMemsetAsync(&head->counter[0], 0, sizeof(head->counter), s) != cudaSuccess) return GRMHD_ERR_CUDA;
  batch_con2prim_kernel<<<nsm * 8, kBatchItem, 0, s>>>(head, boxes, p, nfail);
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  batch_ghost_kernel<<<nsm * 8, kBatchItem, 0, s>>>(head, boxes);
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  const bool curved = batch->curved != 0;
  cudaError_t e;
  if (p.precision == GRMHD_MIXED) e = launch_batch_rhs_mixed(head, boxes, p, curved, nsm, s);
  else if (batch->two_pass) e = launch_batch_rhs_two_pass(head, boxes, p, curved, batch->three_pass != 0, nsm, s);
  else e = launch_batch_rhs_fp64(head, boxes, p, curved, nsm, s);
  return e == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

int grmhd_batch_rhs_fused(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail, int32_t* status,
                          void* stream) {
  if (!batch || !params || !batch->ws || batch->nbox < 1) return GRMHD_ERR_ARG;
  if (params->eos != GRMHD_EOS_IDEAL) return GRMHD_ERR_ARG;  // batched boxes: Gamma-law only
  if (params->recon != GRMHD_WENO5 && params->recon != GRMHD_MINMOD) return GRMHD_ERR_ARG;
  if (params->precision != GRMHD_FP64 && params->precision != GRMHD_MIXED) return GRMHD_ERR_ARG;
  if (!(params->gamma > 1.0 && params->gamma <= 3.0) || params->nr_maxit < 1 || !(params->nr_tol > 0.0))
    return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  if (status && (reinterpret_cast<uintptr_t>(status) & 3u)) return GRMHD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  BatchHead* head = static_cast<BatchHead*>(batch->ws);
  const BoxDev* boxes =
      reinterpret_cast<const BoxDev*>(static_cast<char*>(batch->ws) + box_table_offset(batch->nbox));
  const DevParams p = make_params(*params);
  // one memset: the work counters (the header's last bytes) and the completion counters after them
  char* zero_from = reinterpret_cast<char*>(&head->counter[0]);
  const size_t zero_bytes = static_cast<size_t>(static_cast<char*>(batch->ws) + box_table_offset(batch->nbox) - zero_from);
  if (cudaMemsetAsync(zero_from, 0, zero_bytes, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  const bool curved = batch->curved != 0;
  const cudaError_t e = p.precision == GRMHD_MIXED
                            ? launch_batch_fused_mixed(head, boxes, p, curved, nsm, nfail, status, s)
                            : launch_batch_fused_fp64(head, boxes, p, curved, nsm, nfail, status, s);
  return e == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

// A library-owned graph of one grmhd_batch_rhs: captured once on a private
// stream (nothing runs while capturing), replayed with one launch per batch
// evaluation.
struct grmhd_batch_graph_t {
  cudaGraphExec_t exec;
};

int grmhd_batch_graph_create(const grmhd_batch* batch, const grmhd_params* params, int32_t* nfail,
                             grmhd_batch_graph* graph) {
  if (!graph) return GRMHD_ERR_ARG;
  *graph = nullptr;
  if (!batch || !params) return GRMHD_ERR_ARG;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(s);
    return GRMHD_ERR_CUDA;
  }
  const int rc = grmhd_batch_rhs(batch, params, nfail, s);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &g);
  cudaStreamDestroy(s);
  if (rc != GRMHD_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return rc != GRMHD_OK ? rc : GRMHD_ERR_CUDA;
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return GRMHD_ERR_CUDA;
  grmhd_batch_graph_t* h = new (std::nothrow) grmhd_batch_graph_t;
  if (!h) {
    cudaGraphExecDestroy(x);
    return GRMHD_ERR_CUDA;
  }
  h->exec = x;
  *graph = h;
  return GRMHD_OK;
}

int grmhd_batch_graph_launch(grmhd_batch_graph graph, void* stream) {
  if (!graph || !graph->exec) return GRMHD_ERR_ARG;
  return cudaGraphLaunch(graph->exec, (cudaStream_t)stream) == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

int grmhd_batch_graph_destroy(grmhd_batch_graph graph) {
  if (!graph) return GRMHD_OK;
  const cudaError_t e = graph->exec ? cudaGraphExecDestroy(graph->exec) : cudaSuccess;
  delete graph;
  return e == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

}  // extern "C"
