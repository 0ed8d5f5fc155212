// Per-cell kernels of a single block: conserved -> primitive recovery,
// primitive -> conserved, ghost-zone fill.
#include "recovery.cuh"

namespace grmhd {

__global__ void con2prim_kernel(DevGrid g, DevParams p, const double* __restrict__ cons,
                                const double* __restrict__ metric, double* __restrict__ prim,
                                int8_t* __restrict__ status, int32_t* __restrict__ nfail) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  int myfail = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    const int st = con2prim_at(g, p, cons, metric, prim, c);
    myfail += (st >= 2);
    if (status) status[c] = (int8_t)st;
  }
  if (nfail && myfail) atomicAdd(nfail, myfail);
}

__global__ void prim2con_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                const double* __restrict__ metric, double* __restrict__ cons) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double pr[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pr[q] = __ldg(prim + q * g.ncell + c);
    Geom<double> m;
    if (metric) {
      CellMetric cm;
      cell_metric(metric, g.ncell, c, cm);
      m.alpha = __ldg(metric + c);
#pragma unroll
      for (int i = 0; i < 3; ++i) m.beta[i] = __ldg(metric + (1 + i) * g.ncell + c);
#pragma unroll
      for (int i = 0; i < 6; ++i) m.g[i] = cm.g[i];
      m.sqrtg = cm.sqrtg;
      m.gup_dd = cm.gu[0];
      Side<double> s;
      side_state<double, true, 0>(pr, m, p.gamma, p.gfac, s);
#pragma unroll
      for (int q = 0; q < 8; ++q) cons[q * g.ncell + c] = s.U[q];
    } else {
      Side<double> s;
      side_state<double, false, 0>(pr, m, p.gamma, p.gfac, s);
#pragma unroll
      for (int q = 0; q < 8; ++q) cons[q * g.ncell + c] = s.U[q];
    }
  }
}

__global__ void fill_ghosts_kernel(DevGrid g, int bc, int nvar, double* __restrict__ f) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
       c += (long long)gridDim.x * blockDim.x)
    fill_ghost_at(g, bc, nvar, f, c);
}

static int grid_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  const long long cap = 152LL * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_con2prim(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                            double* prim, int8_t* status, int32_t* nfail, cudaStream_t s) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  con2prim_kernel<<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, prim, status, nfail);
  return cudaGetLastError();
}

cudaError_t launch_prim2con(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                            double* cons, cudaStream_t s) {
  prim2con_kernel<<<grid_blocks(g.ncell, 128), 128, 0, s>>>(g, p, prim, metric, cons);
  return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(const DevGrid& g, int bc, int nvar, double* field, cudaStream_t s) {
  fill_ghosts_kernel<<<grid_blocks(g.ncell, 256), 256, 0, s>>>(g, bc, nvar, field);
  return cudaGetLastError();
}

}  // namespace grmhd
