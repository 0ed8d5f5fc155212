// Per-cell kernels of a single block: conserved -> primitive recovery,
// primitive -> conserved, ghost-zone fill.
#include "recovery.cuh"

namespace grmhd {

template <bool POLY>
__global__ void con2prim_kernel(DevGrid g, DevParams p, const double* __restrict__ cons,
                                const double* __restrict__ metric, double* __restrict__ prim,
                                int8_t* __restrict__ status, int32_t* __restrict__ nfail) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  int myfail = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    const int st = con2prim_at<false, false, true, POLY>(g, p, cons, metric, prim, c);
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
    if (p.eos == GRMHD_EOS_POLYTROPE && pr[0] > 0.0) pr[4] = pr[0] * poly_k_rho_gm1<double>(p, pr[0]);
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

// Mixed path: FP32-predicted FP64 recovery, writing FP64 and FP32 primitives.
template <bool RESULT64, bool POLY>
__global__ void con2prim_mixed_kernel(DevGrid g, DevParams p, const double* __restrict__ cons,
                                      const double* __restrict__ metric, double* __restrict__ prim,
                                      float* __restrict__ prim32, const double* __restrict__ mcache,
                                      const float* __restrict__ geom32, int32_t* __restrict__ nfail) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  int myfail = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    myfail += (con2prim_at<true, true, RESULT64, POLY>(g, p, cons, metric, prim, c, prim32, mcache, geom32) >= 2);
  }
  if (nfail && myfail) atomicAdd(nfail, myfail);
}

// The FP32 primitive copy of the mixed path holds the primitives in pairs,
// [q/2][ncell] float2 (q even in .x, q odd in .y): its ghost fill copies
// npair float2 components.
__global__ void fill_ghosts_f32_kernel(DevGrid g, int bc, int npair, float2* __restrict__ f) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
       c += (long long)gridDim.x * blockDim.x)
    fill_ghost_at(g, bc, npair, f, c);
}

// FP32 pair copy of the FP64 primitives [8][n] (conversions on the integer
// pipe, fpbits.cuh).
__global__ void prim_to_f32_pairs_kernel(long long n, const double* __restrict__ a, float2* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int h = 0; h < 4; ++h)
      b[h * n + i] = make_float2(f64_to_f32i(__ldg(a + 2 * h * n + i)), f64_to_f32i(__ldg(a + (2 * h + 1) * n + i)));
  }
}

// Geometry cache of a static metric (layout in rhs.cuh, kGeomCacheComps values per
// point): every FP64 quantity the mixed RHS needs, computed once in FP64.
// mcache (FP64, 7 components per point): 1/sqrt(gamma) and gamma^ij for the
// primitive recovery.
template <class GT>
__global__ void geom_cache_kernel(DevGrid g, const double* __restrict__ metric, GT* __restrict__ geom,
                                  double* __restrict__ mcache) {
  const long long n = g.ncell;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    idx[0] = (int)(c % g.N[0]);
    idx[1] = (int)((c / g.N[0]) % g.N[1]);
    idx[2] = (int)(c / ((long long)g.N[0] * g.N[1]));
    // the FP32 cache's values are converted on the integer pipe (fpbits.cuh;
    // the bits of the conversion instruction for normal FP32 values)
    auto cvt = [](double x) -> GT {
      if constexpr (sizeof(GT) == 4) return f64_to_f32i(x);
      else return x;
    };
    double a[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      a[q] = __ldg(metric + q * n + c);
      geom[q * n + c] = cvt(a[q]);
      // FP32 cache: half the metric values; a face's metric is the sum of its
      // two cells' halves (the FP64 cache holds the face metric itself)
      if constexpr (sizeof(GT) == 4) geom[(kGeomCacheHalf32 + q) * n + c] = cvt(0.5 * a[q]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long s = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
      GT sgf = GT(1), gupf = GT(1);
      // the face metric, the mean of the two cells (0.5 (a_below + a): the
      // halving is exact, so the value has the bits of 0.5 a_below + 0.5 a)
      double fm[10];
#pragma unroll
      for (int q = 0; q < 10; ++q)
        fm[q] = idx[d] >= 1 ? 0.5 * (__ldg(metric + q * n + c - s) + a[q]) : (q == 0 ? 1.0 : 0.0);
      if constexpr (sizeof(GT) == 8) {
        // FP64 cache: the face metric and its 1/alpha; points without a lower
        // neighbour have no face that any kernel computes
#pragma unroll
        for (int q = 0; q < 10; ++q) geom[(kGeomCacheFace + 10 * d + q) * n + c] = fm[q];
        geom[(kGeomCacheFaceIa + d) * n + c] = 1.0 / fm[0];
      }
      if (idx[d] >= 1) {
        const double* m = fm + 4;
        const double cxx = m[3] * m[5] - m[4] * m[4];
        const double cyy = m[0] * m[5] - m[2] * m[2];
        const double czz = m[0] * m[3] - m[1] * m[1];
        const double det = m[0] * cxx - m[1] * (m[1] * m[5] - m[4] * m[2]) + m[2] * (m[1] * m[4] - m[3] * m[2]);
        const double cdd = d == 0 ? cxx : (d == 1 ? cyy : czz);
        sgf = cvt(sqrt(det));
        gupf = cvt(cdd / det);
      }
      geom[(10 + d) * n + c] = sgf;
      geom[(13 + d) * n + c] = gupf;
    }
    {
      const double gxx = a[4], gxy = a[5], gxz = a[6], gyy = a[7], gyz = a[8], gzz = a[9];
      const double cxx = gyy * gzz - gyz * gyz, cxy = gxz * gyz - gxy * gzz, cxz = gxy * gyz - gxz * gyy;
      const double cyy = gxx * gzz - gxz * gxz, cyz = gxy * gxz - gxx * gyz, czz = gxx * gyy - gxy * gxy;
      const double det = gxx * cxx + gxy * cxy + gxz * cxz;
      const double idet = 1.0 / det;
      const double sgd = sqrt(det);
      geom[16 * n + c] = cvt(sgd);
      mcache[c] = 1.0 / sgd;
      mcache[1 * n + c] = cxx * idet;
      mcache[2 * n + c] = cxy * idet;
      mcache[3 * n + c] = cxz * idet;
      mcache[4 * n + c] = cyy * idet;
      mcache[5 * n + c] = cyz * idet;
      mcache[6 * n + c] = czz * idet;
      geom[17 * n + c] = cvt(cxx * idet);
      geom[18 * n + c] = cvt(cxy * idet);
      geom[19 * n + c] = cvt(cxz * idet);
      geom[20 * n + c] = cvt(cyy * idet);
      geom[21 * n + c] = cvt(cyz * idet);
      geom[22 * n + c] = cvt(czz * idet);
    }
    const bool inner = idx[0] >= 2 && idx[0] < g.N[0] - 2 && idx[1] >= 2 && idx[1] < g.N[1] - 2 && idx[2] >= 2 &&
                       idx[2] < g.N[2] - 2;
    double da[3];  // d_e alpha
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const long long s = e == 0 ? 1 : (e == 1 ? g.sy : g.sz);
      const double w = g.idx[e] * (1.0 / 12.0);
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        double v = 0.0;
        if (inner) {
          const double* mm = metric + q * n + c;
          v = (8.0 * (__ldg(mm + s) - __ldg(mm - s)) - (__ldg(mm + 2 * s) - __ldg(mm - 2 * s))) * w;
        }
        if (q == 0) da[e] = v;
        geom[(23 + 10 * e + q) * n + c] = cvt(v);
      }
    }
    if constexpr (sizeof(GT) == 8) {
      // the metric factors of the sources (SrcStatics, in its order), formed
      // from the values the RHS reads from this cache
      const double beta[3] = {a[1], a[2], a[3]};
      const double gm[6] = {a[4], a[5], a[6], a[7], a[8], a[9]};
      double gu[6], sgc;
#pragma unroll
      for (int i = 0; i < 6; ++i) gu[i] = geom[(17 + i) * n + c];
      sgc = geom[16 * n + c];
      SrcStatics<double> st;
      source_statics<double>(a[0], beta, gm, sgc, gu, da, st);
      double* q = geom + (long long)kGeomCacheStat * n + c;
      q[0] = st.ia;
      q[n] = st.ia2;
#pragma unroll
      for (int i = 0; i < 3; ++i) q[(2 + i) * n] = st.bia2[i];
#pragma unroll
      for (int k = 0; k < 6; ++k) q[(5 + k) * n] = st.M[k];
#pragma unroll
      for (int i = 0; i < 3; ++i) q[(11 + i) * n] = st.betal[i];
      q[14 * n] = st.asg;
#pragma unroll
      for (int k = 0; k < 6; ++k) q[(15 + k) * n] = st.bb[k];
      q[21 * n] = st.bda;
    }
  }
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
  if (p.eos == GRMHD_EOS_POLYTROPE)
    con2prim_kernel<true><<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, prim, status, nfail);
  else
    con2prim_kernel<false><<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, prim, status, nfail);
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

namespace grmhd {

cudaError_t launch_con2prim_mixed(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                                  double* prim, float* prim32, const double* mcache, const float* geom32,
                                  bool result64, int32_t* nfail, cudaStream_t s) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  void (*k)(DevGrid, DevParams, const double*, const double*, double*, float*, const double*, const float*,
            int32_t*);
  if (p.eos == GRMHD_EOS_POLYTROPE)
    k = result64 ? con2prim_mixed_kernel<true, true> : con2prim_mixed_kernel<false, true>;
  else
    k = result64 ? con2prim_mixed_kernel<true, false> : con2prim_mixed_kernel<false, false>;
  k<<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, prim, prim32, mcache, geom32, nfail);
  return cudaGetLastError();
}

cudaError_t launch_fill_ghosts_f32(const DevGrid& g, int bc, int nvar, float* field, cudaStream_t s) {
  fill_ghosts_f32_kernel<<<grid_blocks(g.ncell, 256), 256, 0, s>>>(g, bc, nvar / 2, reinterpret_cast<float2*>(field));
  return cudaGetLastError();
}

cudaError_t launch_prim_to_f32_pairs(long long ncell, const double* prim, float* prim32, cudaStream_t s) {
  prim_to_f32_pairs_kernel<<<grid_blocks(ncell, 256), 256, 0, s>>>(ncell, prim, reinterpret_cast<float2*>(prim32));
  return cudaGetLastError();
}

cudaError_t launch_geom_cache(const DevGrid& g, const double* metric, void* geom, bool fp64, double* mcache,
                              cudaStream_t s) {
  if (fp64)
    geom_cache_kernel<double><<<grid_blocks(g.ncell, 128), 128, 0, s>>>(g, metric, static_cast<double*>(geom), mcache);
  else
    geom_cache_kernel<float><<<grid_blocks(g.ncell, 128), 128, 0, s>>>(g, metric, static_cast<float*>(geom), mcache);
  return cudaGetLastError();
}

template <bool POLY>
__global__ void con2prim_cached_kernel(DevGrid g, DevParams p, const double* __restrict__ cons,
                                       const double* __restrict__ metric, const double* __restrict__ mcache,
                                       double* __restrict__ prim, int32_t* __restrict__ nfail) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  int myfail = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    // FP64 recovery from the FP32 predictor's guess (Gamma-law; the polytrope has its own)
    myfail += (con2prim_at<!POLY, false, true, POLY>(g, p, cons, metric, prim, c, nullptr, mcache) >= 2);
  }
  if (nfail && myfail) atomicAdd(nfail, myfail);
}

cudaError_t launch_con2prim_cached(const DevGrid& g, const DevParams& p, const double* cons, const double* metric,
                                   const double* mcache, double* prim, int32_t* nfail, cudaStream_t s) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  if (p.eos == GRMHD_EOS_POLYTROPE)
    con2prim_cached_kernel<true><<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, mcache, prim, nfail);
  else
    con2prim_cached_kernel<false><<<grid_blocks(nint, 128), 128, 0, s>>>(g, p, cons, metric, mcache, prim, nfail);
  return cudaGetLastError();
}

}  // namespace grmhd
