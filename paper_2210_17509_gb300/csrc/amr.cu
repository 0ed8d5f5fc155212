// Two-level block AMR without subcycling (Sec. 3): restriction of the
// conserved variables, prolongation of the primitives into fine ghost zones,
// flux restriction at the coarse-fine interface, and the composite step.
//
// Placement: a fine grid at lo (coarse interior indices) halves the coarse
// spacing; its interior cell i lies in the coarse interior cell
// lo + floor(i / 2) along each axis.
#include <cmath>
#include <vector>

#include "recovery.cuh"
#include "rhs.cuh"

namespace grmhd {

namespace {

__device__ __forceinline__ int floor_half(int i) { return i >= 0 ? i / 2 : -((1 - i) / 2); }

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)b;
}

// Covered coarse cell I (x fastest), variable q: the mean of its 8 children,
// summed with x fastest, then y, then z.
__global__ void restrict_kernel(DevGrid c, double* __restrict__ coarse, DevGrid f, const double* __restrict__ fine,
                                int lox, int loy, int loz, int nvar) {
  const int mx = f.n[0] / 2, my = f.n[1] / 2, mz = f.n[2] / 2;
  const long long ncov = (long long)mx * my * mz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncov * nvar;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / ncov);
    const long long r = t - (long long)q * ncov;
    const int I = (int)(r % mx), J = (int)((r / mx) % my), K = (int)(r / ((long long)mx * my));
    const double* u = fine + (long long)q * f.ncell;
    double sum = 0.0;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx)
          sum += u[(long long)(f.ng + 2 * K + cz) * f.sz + (long long)(f.ng + 2 * J + cy) * f.sy +
                   (f.ng + 2 * I + cx)];
    coarse[(long long)q * c.ncell + (long long)(c.ng + loz + K) * c.sz + (long long)(c.ng + loy + J) * c.sy +
           (c.ng + lox + I)] = sum / 8.0;
  }
}

// Number of ghost points of a block: two z slabs of full extent, two y slabs
// over the interior z range, two x slabs over the interior y and z ranges.
__host__ __device__ __forceinline__ long long ghost_count(const DevGrid& f) {
  return 2LL * f.ng * f.N[0] * f.N[1] + 2LL * f.ng * f.N[0] * f.n[2] + 2LL * f.ng * f.n[1] * f.n[2];
}

// Interior-relative coordinates of the g-th ghost point (slab order above).
__device__ __forceinline__ void ghost_point(const DevGrid& f, long long g, int fi[3]) {
  const long long zs = (long long)f.ng * f.N[0] * f.N[1];
  const long long ys = (long long)f.ng * f.N[0] * f.n[2];
  if (g < 2 * zs) {
    const int side = (int)(g / zs);
    const long long r = g - side * zs;
    fi[0] = (int)(r % f.N[0]) - f.ng;
    fi[1] = (int)((r / f.N[0]) % f.N[1]) - f.ng;
    const int k = (int)(r / ((long long)f.N[0] * f.N[1]));
    fi[2] = side ? f.n[2] + k : k - f.ng;
    return;
  }
  g -= 2 * zs;
  if (g < 2 * ys) {
    const int side = (int)(g / ys);
    const long long r = g - side * ys;
    fi[0] = (int)(r % f.N[0]) - f.ng;
    const int j = (int)((r / f.N[0]) % f.ng);
    fi[1] = side ? f.n[1] + j : j - f.ng;
    fi[2] = (int)(r / ((long long)f.N[0] * f.ng));
    return;
  }
  g -= 2 * ys;
  const long long xs = (long long)f.ng * f.n[1] * f.n[2];
  const int side = (int)(g / xs);
  const long long r = g - side * xs;
  const int i = (int)(r % f.ng);
  fi[0] = side ? f.n[0] + i : i - f.ng;
  fi[1] = (int)((r / f.ng) % f.n[1]);
  fi[2] = (int)(r / ((long long)f.ng * f.n[1]));
}

// Fine point (all points, x fastest, or the ghost points only), variable q:
// parent value plus the minmod-limited slope per axis times the child's
// offset (+-1/4).
__global__ void prolongate_kernel(DevGrid c, const double* __restrict__ coarse, DevGrid f, double* __restrict__ fine,
                                  int lox, int loy, int loz, int nvar, int ghosts_only) {
  const long long npts = ghosts_only ? ghost_count(f) : f.ncell;
  const int lo[3] = {lox, loy, loz};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npts * nvar;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / npts);
    const long long k = t - (long long)q * npts;
    int fi[3];
    if (ghosts_only) {
      ghost_point(f, k, fi);
    } else {
      fi[0] = (int)(k % f.N[0]) - f.ng;
      fi[1] = (int)((k / f.N[0]) % f.N[1]) - f.ng;
      fi[2] = (int)(k / ((long long)f.N[0] * f.N[1])) - f.ng;
    }
    const long long pt = (long long)(fi[2] + f.ng) * f.sz + (long long)(fi[1] + f.ng) * f.sy + (fi[0] + f.ng);
    long long pc = 0;
    int par[3];
    double off[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int h = floor_half(fi[d]);
      par[d] = c.ng + lo[d] + h;
      off[d] = (fi[d] - 2 * h == 0) ? -0.25 : 0.25;
    }
    pc = (long long)par[2] * c.sz + (long long)par[1] * c.sy + par[0];
    const double* u = coarse + (long long)q * c.ncell;
    const double u0 = u[pc];
    double val = u0;
    const long long st[3] = {1, c.sy, c.sz};
#pragma unroll
    for (int d = 0; d < 3; ++d) val += off[d] * minmod<double>(u0 - u[pc - st[d]], u[pc + st[d]] - u0);
    fine[(long long)q * f.ncell + pt] = val;
  }
}

// Interface faces: kFacesPerBlock coarse faces per CTA, five flux
// evaluations each (the coarse face, then its four fine faces) on five
// threads; the fluxes meet in shared memory and are combined in a fixed
// order, so the result does not depend on scheduling.
constexpr int kFacesPerBlock = 32;
constexpr int kRefluxThreads = 5 * kFacesPerBlock;

template <int RECON, bool CURVED, bool POLY>
__global__ void __launch_bounds__(kRefluxThreads) reflux_kernel(
    DevGrid c, DevParams p, const double* __restrict__ cprim, const double* __restrict__ cmetric, DevGrid f,
    const double* __restrict__ fprim, const double* __restrict__ fmetric, int lox, int loy, int loz, double scale,
    double* __restrict__ out, double acc_scale, double* __restrict__ acc) {
  __shared__ double sF[kFacesPerBlock][5][8];
  __shared__ long long sCell[kFacesPerBlock];
  __shared__ double sW[kFacesPerBlock];
  const int nc[3] = {f.n[0] / 2, f.n[1] / 2, f.n[2] / 2};
  const int lo[3] = {lox, loy, loz};
  const long long per[3] = {(long long)nc[1] * nc[2], (long long)nc[2] * nc[0], (long long)nc[0] * nc[1]};
  const long long total = 2 * (per[0] + per[1] + per[2]);
  const int fl = threadIdx.x / 5, role = threadIdx.x % 5;
  for (long long base = (long long)blockIdx.x * kFacesPerBlock; base < total;
       base += (long long)gridDim.x * kFacesPerBlock) {
    const long long t = base + fl;
    if (t < total) {
      long long r = t;
      int d = 0;
      while (r >= 2 * per[d]) { r -= 2 * per[d]; ++d; }
      const int side = (int)(r / per[d]);
      r -= side * per[d];
      const int a = (d + 1) % 3, b = (d + 2) % 3;
      const int A = (int)(r % nc[a]), B = (int)(r / nc[a]);
      double F[8];
      if (role == 0) {
        int Ic[3];
        Ic[d] = lo[d] + (side ? nc[d] : 0);
        Ic[a] = lo[a] + A;
        Ic[b] = lo[b] + B;
        const long long cface =
            (long long)(c.ng + Ic[2]) * c.sz + (long long)(c.ng + Ic[1]) * c.sy + (c.ng + Ic[0]);
        face_flux_one<RECON, CURVED, POLY>(c, p, cprim, cmetric, cface, d, F);
        // the uncovered cell: below the face on the low side (the face is its
        // upper face), above it on the high side (its lower face)
        const long long st = d == 0 ? 1 : (d == 1 ? c.sy : c.sz);
        sCell[fl] = side ? cface : cface - st;
        sW[fl] = (side ? 1.0 : -1.0) * c.idx[d];
      } else {
        int If[3];
        If[d] = side ? f.n[d] : 0;
        If[a] = 2 * A + ((role - 1) & 1);
        If[b] = 2 * B + ((role - 1) >> 1);
        const long long fface =
            (long long)(f.ng + If[2]) * f.sz + (long long)(f.ng + If[1]) * f.sy + (f.ng + If[0]);
        face_flux_one<RECON, CURVED, POLY>(f, p, fprim, fmetric, fface, d, F);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) sF[fl][role][q] = F[q];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kFacesPerBlock * 8; idx += kRefluxThreads) {
      const int j = idx >> 3, q = idx & 7;
      if (base + j < total) {
        const double ff = ((sF[j][1][q] + sF[j][2][q]) + sF[j][3][q]) + sF[j][4][q];
        const double dl = sW[j] * (0.25 * ff - sF[j][0][q]);
        const long long o = (long long)q * c.ncell + sCell[j];
        out[o] += scale * dl;
        if (acc) acc[o] += acc_scale * dl;
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_restrict(const DevGrid& c, double* coarse, const DevGrid& f, const double* fine, const int lo[3],
                            int nvar, cudaStream_t s) {
  const long long n = (long long)(f.n[0] / 2) * (f.n[1] / 2) * (f.n[2] / 2) * nvar;
  restrict_kernel<<<blocks_for(n, 256), 256, 0, s>>>(c, coarse, f, fine, lo[0], lo[1], lo[2], nvar);
  return cudaGetLastError();
}

cudaError_t launch_prolongate(const DevGrid& c, const double* coarse, const DevGrid& f, double* fine,
                              const int lo[3], int nvar, bool ghosts_only, cudaStream_t s) {
  const long long n = (ghosts_only ? ghost_count(f) : f.ncell) * nvar;
  prolongate_kernel<<<blocks_for(n, 256), 256, 0, s>>>(c, coarse, f, fine, lo[0], lo[1], lo[2], nvar,
                                                        ghosts_only ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_reflux(const DevGrid& c, const DevParams& p, const double* cprim, const double* cmetric,
                          const DevGrid& f, const double* fprim, const double* fmetric, const int lo[3],
                          double scale, double* out, double acc_scale, double* acc, cudaStream_t s) {
  const long long nf = 2LL * ((long long)(f.n[1] / 2) * (f.n[2] / 2) + (long long)(f.n[2] / 2) * (f.n[0] / 2) +
                              (long long)(f.n[0] / 2) * (f.n[1] / 2));
  const int blocks = blocks_for(nf, kFacesPerBlock);
  using K = void (*)(DevGrid, DevParams, const double*, const double*, DevGrid, const double*, const double*, int,
                     int, int, double, double*, double, double*);
  // [polytrope][WENO5][curved]
  static const K table[2][2][2] = {
      {{reflux_kernel<GRMHD_MINMOD, false, false>, reflux_kernel<GRMHD_MINMOD, true, false>},
       {reflux_kernel<GRMHD_WENO5, false, false>, reflux_kernel<GRMHD_WENO5, true, false>}},
      {{reflux_kernel<GRMHD_MINMOD, false, true>, reflux_kernel<GRMHD_MINMOD, true, true>},
       {reflux_kernel<GRMHD_WENO5, false, true>, reflux_kernel<GRMHD_WENO5, true, true>}}};
  const K k = table[p.eos == GRMHD_EOS_POLYTROPE][p.recon == GRMHD_WENO5][cmetric != nullptr];
  k<<<blocks, kRefluxThreads, 0, s>>>(c, p, cprim, cmetric, f, fprim, fmetric, lo[0], lo[1], lo[2], scale, out,
                                      acc_scale, acc);
  return cudaGetLastError();
}

}  // namespace grmhd

using namespace grmhd;

namespace {

// Fine grid against its coarse parent: same ghost width (>= 2), even n,
// half the spacing, placement inside the coarse interior.
int check_placement(const grmhd_grid* c, const grmhd_grid* f, const int32_t* lo) {
  if (check_grid(c, 2) || check_grid(f, 2) || !lo) return GRMHD_ERR_ARG;
  if (f->ng != c->ng) return GRMHD_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (f->n[d] % 2) return GRMHD_ERR_ARG;
    if (std::fabs(2.0 * f->dx[d] - c->dx[d]) > 1e-12 * c->dx[d]) return GRMHD_ERR_ARG;
    if (lo[d] < 0 || lo[d] + f->n[d] / 2 > c->n[d]) return GRMHD_ERR_ARG;
  }
  return GRMHD_OK;
}

}  // namespace

extern "C" {

int grmhd_restrict(const grmhd_grid* coarse, double* coarse_field, const grmhd_grid* fine,
                   const double* fine_field, const int32_t lo[3], int32_t nvar, void* stream) {
  int e = check_placement(coarse, fine, lo);
  if (e) return e;
  if (nvar < 1 || nvar > 64 || !coarse_field || !fine_field || !aligned8(coarse_field) || !aligned8(fine_field))
    return GRMHD_ERR_ARG;
  const int l[3] = {lo[0], lo[1], lo[2]};
  return cuda_status(launch_restrict(make_grid(*coarse), coarse_field, make_grid(*fine), fine_field, l, nvar,
                                     (cudaStream_t)stream));
}

int grmhd_prolongate(const grmhd_grid* coarse, const double* coarse_field, const grmhd_grid* fine,
                     double* fine_field, const int32_t lo[3], int32_t nvar, int32_t ghosts_only, void* stream) {
  int e = check_placement(coarse, fine, lo);
  if (e) return e;
  if (nvar < 1 || nvar > 64 || !coarse_field || !fine_field || !aligned8(coarse_field) || !aligned8(fine_field))
    return GRMHD_ERR_ARG;
  const int l[3] = {lo[0], lo[1], lo[2]};
  return cuda_status(launch_prolongate(make_grid(*coarse), coarse_field, make_grid(*fine), fine_field, l, nvar,
                                       ghosts_only != 0, (cudaStream_t)stream));
}

int grmhd_reflux(const grmhd_grid* coarse, const grmhd_params* params, const double* coarse_prim,
                 const double* coarse_metric, const grmhd_grid* fine, const double* fine_prim,
                 const double* fine_metric, const int32_t lo[3], double scale, double* coarse_out,
                 double acc_scale, double* acc, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if ((e = check_placement(coarse, fine, lo))) return e;
  if (coarse->ng < min_ghosts(params, coarse_metric)) return GRMHD_ERR_ARG;
  if (!coarse_prim || !fine_prim || !coarse_out || !aligned8(coarse_prim) || !aligned8(fine_prim) ||
      !aligned8(coarse_out) || (acc && !aligned8(acc)))
    return GRMHD_ERR_ARG;
  if ((coarse_metric == nullptr) != (fine_metric == nullptr)) return GRMHD_ERR_ARG;
  if ((coarse_metric && !aligned8(coarse_metric)) || (fine_metric && !aligned8(fine_metric))) return GRMHD_ERR_ARG;
  if (!std::isfinite(scale) || !std::isfinite(acc_scale)) return GRMHD_ERR_ARG;
  const int l[3] = {lo[0], lo[1], lo[2]};
  return cuda_status(launch_reflux(make_grid(*coarse), make_params(*params), coarse_prim, coarse_metric,
                                   make_grid(*fine), fine_prim, fine_metric, l, scale, coarse_out, acc_scale, acc,
                                   (cudaStream_t)stream));
}

size_t grmhd_amr2_workspace_bytes(const grmhd_grid* coarse, int32_t nfine, const grmhd_grid* fine,
                                  int32_t scheme) {
  if (check_grid(coarse, 0) || nfine < 0 || nfine > 4096 || (nfine > 0 && !fine)) return 0;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3 && scheme != GRMHD_RK4) return 0;
  const int per = scheme == GRMHD_RK4 ? 2 : 1;  // u0 (+ acc)
  size_t total = per * round256((size_t)8 * make_grid(*coarse).ncell * sizeof(double));
  for (int i = 0; i < nfine; ++i) {
    if (check_grid(&fine[i], 0)) return 0;
    total += per * round256((size_t)8 * make_grid(fine[i]).ncell * sizeof(double));
  }
  return total;
}

int grmhd_amr2_step(const grmhd_grid* coarse, const grmhd_params* params, int32_t scheme, double dt,
                    double* coarse_cons, double* coarse_prim, const double* coarse_metric, int32_t nfine,
                    const grmhd_grid* fine, double* const* fine_cons, double* const* fine_prim,
                    const double* const* fine_metric, const int32_t* lo, void* ws, size_t ws_bytes,
                    int32_t* nfail, void* stream) {
  int e = check_params(params);
  if (e) return e;
  if (params->precision != GRMHD_FP64) return GRMHD_ERR_ARG;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3 && scheme != GRMHD_RK4) return GRMHD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return GRMHD_ERR_ARG;
  if ((e = check_grid(coarse, min_ghosts(params, coarse_metric)))) return e;
  if (nfine < 0 || nfine > 4096 || (nfine > 0 && (!fine || !fine_cons || !fine_prim || !lo))) return GRMHD_ERR_ARG;
  if (!coarse_cons || !coarse_prim || !aligned8(coarse_cons) || !aligned8(coarse_prim)) return GRMHD_ERR_ARG;
  if (coarse_metric && !aligned8(coarse_metric)) return GRMHD_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return GRMHD_ERR_ARG;
  if (nfail && (reinterpret_cast<uintptr_t>(nfail) & 3u)) return GRMHD_ERR_ARG;
  for (int i = 0; i < nfine; ++i) {
    if ((e = check_placement(coarse, &fine[i], lo + 3 * i))) return e;
    const double* fm = fine_metric ? fine_metric[i] : nullptr;
    if ((coarse_metric == nullptr) != (fm == nullptr)) return GRMHD_ERR_ARG;
    if (!fine_cons[i] || !fine_prim[i] || !aligned8(fine_cons[i]) || !aligned8(fine_prim[i]) ||
        (fm && !aligned8(fm)))
      return GRMHD_ERR_ARG;
    // a gap of one coarse cell to the coarse boundary and to the other fine grids
    for (int d = 0; d < 3; ++d)
      if (lo[3 * i + d] < 1 || lo[3 * i + d] + fine[i].n[d] / 2 > coarse->n[d] - 1) return GRMHD_ERR_ARG;
    for (int j = 0; j < i; ++j) {
      bool apart = false;
      for (int d = 0; d < 3; ++d) {
        const int a0 = lo[3 * i + d], a1 = a0 + fine[i].n[d] / 2;
        const int b0 = lo[3 * j + d], b1 = b0 + fine[j].n[d] / 2;
        if (a1 + 1 <= b0 || b1 + 1 <= a0) apart = true;
      }
      if (!apart) return GRMHD_ERR_ARG;
    }
  }
  if (ws_bytes < grmhd_amr2_workspace_bytes(coarse, nfine, fine, scheme)) return GRMHD_ERR_SIZE;

  cudaStream_t s = (cudaStream_t)stream;
  const DevParams p = make_params(*params);
  const int nb = nfine + 1;
  std::vector<DevGrid> g(nb);
  std::vector<double*> U(nb), P(nb), U0(nb), acc(nb, nullptr);
  std::vector<const double*> M(nb);
  g[0] = make_grid(*coarse);
  U[0] = coarse_cons;
  P[0] = coarse_prim;
  M[0] = coarse_metric;
  for (int i = 0; i < nfine; ++i) {
    g[i + 1] = make_grid(fine[i]);
    U[i + 1] = fine_cons[i];
    P[i + 1] = fine_prim[i];
    M[i + 1] = fine_metric ? fine_metric[i] : nullptr;
  }
  char* w = static_cast<char*>(ws);
  for (int b = 0; b < nb; ++b) {
    const size_t bytes = (size_t)8 * g[b].ncell * sizeof(double);
    U0[b] = reinterpret_cast<double*>(w);
    w += round256(bytes);
    if (scheme == GRMHD_RK4) {
      acc[b] = reinterpret_cast<double*>(w);
      w += round256(bytes);
    }
    if (cudaMemcpyAsync(U0[b], U[b], bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  }
  RkStage st[4];
  const int ns = rk_stages(scheme, dt, st);
  for (int k = 0; k < ns; ++k) {
    // fused RHS + stage update of every block
    for (int b = 0; b < nb; ++b) {
      StageEpilogue ep = no_epilogue();
      ep.u = U[b];
      ep.u0 = U0[b];
      ep.acc_in = st[k].acc_in ? acc[b] : nullptr;
      ep.acc_out = st[k].acc_out ? acc[b] : nullptr;
      ep.c0 = st[k].c0;
      ep.c1 = st[k].c1;
      ep.cr = st[k].cr;
      ep.ca = st[k].ca;
      ep.wa = st[k].wa;
      ep.wr = st[k].wr;
      if (launch_rhs_fp64(g[b], p, P[b], M[b], nullptr, ep, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
    // flux restriction onto the coarse update (and the RK4 accumulator),
    // from the primitives the RHS used; then the covered coarse cells
    for (int i = 0; i < nfine; ++i) {
      const int l[3] = {lo[3 * i], lo[3 * i + 1], lo[3 * i + 2]};
      if (launch_reflux(g[0], p, P[0], M[0], g[i + 1], P[i + 1], M[i + 1], l, st[k].cr, U[0], st[k].wr,
                        st[k].acc_out ? acc[0] : nullptr, s) != cudaSuccess)
        return GRMHD_ERR_CUDA;
    }
    for (int i = 0; i < nfine; ++i) {
      const int l[3] = {lo[3 * i], lo[3 * i + 1], lo[3 * i + 2]};
      if (launch_restrict(g[0], U[0], g[i + 1], U[i + 1], l, 8, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
    for (int b = 0; b < nb; ++b)
      if (launch_con2prim(g[b], p, U[b], M[b], P[b], nullptr, nfail, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (launch_fill_ghosts(g[0], p.bc, 8, P[0], s) != cudaSuccess) return GRMHD_ERR_CUDA;
    for (int i = 0; i < nfine; ++i) {
      const int l[3] = {lo[3 * i], lo[3 * i + 1], lo[3 * i + 2]};
      if (launch_prolongate(g[0], P[0], g[i + 1], P[i + 1], l, 8, true, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
  }
  return GRMHD_OK;
}

}  // extern "C"
