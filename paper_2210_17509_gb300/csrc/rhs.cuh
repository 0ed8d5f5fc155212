// Fused method-of-lines RHS kernel: reconstruction + face metric + HLLE +
// flux divergence + source terms + RK stage epilogue, one launch.
//
// Work decomposition: a CTA owns a TX x TY x TZ tile of interior cells.  It
// computes every face flux of the tile exactly once -- (TX+1) TY TZ x-faces,
// TX (TY+1) TZ y-faces, TX TY (TZ+1) z-faces, one flat list spread over all
// threads -- into shared memory (SoA [comp][face], conflict-free), then each
// thread differences the six faces of its cell, adds the Eq. 13 source
// (3+1 form, curved metric only) and applies the stage epilogue.
#pragma once

#include "physics.cuh"

namespace grmhd {

// Where the kernels read their inputs from.
//  SrcF64:   primitives and metric as stored (FP64); the FP64 path, and the
//            mixed path when no workspace for the caches is available.
//  SrcCache: FP32 copy of the primitives plus the FP32 geometry cache (metric
//            values, face and cell sqrt(gamma) and inverse-metric entries and
//            metric derivatives, all computed in FP64 once per step); the fast
//            mixed path.
struct SrcF64 {
  const double* __restrict__ prim;
  const double* __restrict__ metric;
  const double* __restrict__ kij;
};
template <class PT, class GT>
struct SrcCacheT {
  const PT* __restrict__ prim;
  const GT* __restrict__ geom;
  const double* __restrict__ kij;
};
typedef SrcCacheT<float, float> SrcCache;      // mixed: FP32 primitives + FP32 geometry cache
typedef SrcCacheT<double, double> SrcCache64;  // FP64: FP64 primitives + FP64 geometry cache

// Geometry cache layout ([comp][ncell] floats, every point of the block):
//   0..9    metric (alpha, beta^i, gamma_ij)
//   10..12  sqrt(gamma) on the lower x / y / z face of the point
//   13..15  gamma^{dd} on the lower x / y / z face
//   16      sqrt(gamma) at the point;  17..22 gamma^{ij} at the point
//   23..52  4th-order derivatives d_e of the 10 metric entries (index 23 + 10 e + q)
constexpr int kGeomComps = 53;

template <class T>
__device__ __forceinline__ T ld_prim(const SrcF64& s, long long i) { return (T)__ldg(s.prim + i); }
template <class T, class PT, class GT>
__device__ __forceinline__ T ld_prim(const SrcCacheT<PT, GT>& s, long long i) { return (T)__ldg(s.prim + i); }

// Load the 8 primitives at the six-point stencil of the face between cell
// c - stride and c, reconstruct both states.
template <class T, int RECON, class S>
__device__ __forceinline__ void reconstruct_face(const S& src, long long ncell, long long c, long long stride, T eps,
                                                 T pL[8], T pR[8]) {
  if (RECON == GRMHD_WENO5 && sizeof(T) == 8) {
    // FP64: the four normalisations of two variables share one division
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      double n[4], d[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long a = (q + h) * ncell + c;
        const double um3 = ld_prim<double>(src, a - 3 * stride), um2 = ld_prim<double>(src, a - 2 * stride);
        const double um1 = ld_prim<double>(src, a - stride), u0 = ld_prim<double>(src, a);
        const double up1 = ld_prim<double>(src, a + stride), up2 = ld_prim<double>(src, a + 2 * stride);
        weno5_parts(um3, um2, um1, u0, up1, (double)eps, n[2 * h], d[2 * h]);
        weno5_parts(up2, up1, u0, um1, um2, (double)eps, n[2 * h + 1], d[2 * h + 1]);
      }
      const double d01 = d[0] * d[1], d23 = d[2] * d[3];
      const double X = 1.0 / (d01 * d23);
      const double x01 = d23 * X, x23 = d01 * X;
      pL[q] = (T)(n[0] * (d[1] * x01));
      pR[q] = (T)(n[1] * (d[0] * x01));
      pL[q + 1] = (T)(n[2] * (d[3] * x23));
      pR[q + 1] = (T)(n[3] * (d[2] * x23));
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long a = q * ncell + c;
    if (RECON == GRMHD_WENO5) {
      const T um3 = ld_prim<T>(src, a - 3 * stride), um2 = ld_prim<T>(src, a - 2 * stride);
      const T um1 = ld_prim<T>(src, a - stride), u0 = ld_prim<T>(src, a);
      const T up1 = ld_prim<T>(src, a + stride), up2 = ld_prim<T>(src, a + 2 * stride);
      weno5_pair<T>(um3, um2, um1, u0, up1, up2, eps, pL[q], pR[q]);
    } else {
      const T um2 = ld_prim<T>(src, a - 2 * stride), um1 = ld_prim<T>(src, a - stride);
      const T u0 = ld_prim<T>(src, a), up1 = ld_prim<T>(src, a + stride);
      pL[q] = um1 + T(0.5) * minmod<T>(um1 - um2, u0 - um1);
      pR[q] = u0 - T(0.5) * minmod<T>(u0 - um1, up1 - u0);
    }
  }
}

// Legacy form used by the adjoint (FP64 primitives).
template <class T, int RECON>
__device__ __forceinline__ void reconstruct_face(const double* __restrict__ prim, long long ncell, long long c,
                                                 long long stride, T eps, T pL[8], T pR[8]) {
  SrcF64 s;
  s.prim = prim;
  s.metric = nullptr;
  s.kij = nullptr;
  reconstruct_face<T, RECON, SrcF64>(s, ncell, c, stride, eps, pL, pR);
}

// Face metric from the inputs (FP64 mean, FP64 sqrt(gamma) and gamma^dd).
template <class T, int DIR>
__device__ __forceinline__ void face_geometry(const SrcF64& s, long long ncell, long long c, long long stride,
                                              Geom<T>& m) {
  face_geom<T, DIR>(s.metric, ncell, c, stride, m);
}

// Face metric from the cache: mean of the two cells (in the compute type),
// cached sqrt(gamma) and gamma^dd of the face.
template <class T, int DIR, class PT, class GT>
__device__ __forceinline__ void face_geometry(const SrcCacheT<PT, GT>& s, long long ncell, long long c,
                                              long long stride, Geom<T>& m) {
  const GT* gm = s.geom;
  T a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = T(0.5) * ((T)__ldg(gm + q * ncell + c - stride) + (T)__ldg(gm + q * ncell + c));
  m.alpha = a[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = a[1 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = a[4 + i];
  m.sqrtg = (T)__ldg(gm + (10 + DIR) * ncell + c);
  m.gup_dd = (T)__ldg(gm + (13 + DIR) * ncell + c);
}

// Face metric with a run-time face normal.
template <class T>
__device__ __forceinline__ void face_geometry_rt(const SrcF64& s, long long ncell, long long c, long long stride,
                                                 int dir, Geom<T>& m) {
  face_geom_rt<T>(s.metric, ncell, c, stride, dir, m);
}
template <class T, class PT, class GT>
__device__ __forceinline__ void face_geometry_rt(const SrcCacheT<PT, GT>& s, long long ncell, long long c,
                                                 long long stride, int dir, Geom<T>& m) {
  const GT* gm = s.geom;
  T a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = T(0.5) * ((T)__ldg(gm + q * ncell + c - stride) + (T)__ldg(gm + q * ncell + c));
  m.alpha = a[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = a[1 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = a[4 + i];
  m.sqrtg = (T)__ldg(gm + (10 + dir) * ncell + c);
  m.gup_dd = (T)__ldg(gm + (13 + dir) * ncell + c);
}

// Flux through a face whose normal dir is known only at run time: the
// states and the metric are relabelled so the normal is the first axis,
// one x-face computation runs, and the flux is relabelled back (one copy of
// the face code instead of three keeps the kernel small).
template <class T, int RECON, bool CURVED, class S>
__device__ __forceinline__ void face_flux_rt(const DevGrid& g, const DevParams& p, const S& src, long long c, int dir,
                                             T F[8]) {
  const long long stride = (dir == 0) ? 1 : ((dir == 1) ? g.sy : g.sz);
  T pL[8], pR[8];
  reconstruct_face<T, RECON, S>(src, g.ncell, c, stride, (T)p.weno_eps, pL, pR);
  Geom<T> m;
  if (CURVED) face_geometry_rt<T>(src, g.ncell, c, stride, dir, m);
  if (!physical_state<T, CURVED>(pL, m)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pL[q] = ld_prim<T>(src, q * g.ncell + c - stride);
  }
  if (!physical_state<T, CURVED>(pR, m)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pR[q] = ld_prim<T>(src, q * g.ncell + c);
  }
  T rL[8], rR[8], Fr[8];
  rotate_state(dir, pL, rL);
  rotate_state(dir, pR, rR);
  if (CURVED) rotate_metric(dir, m);
  Side<T> L, R;
  side_state<T, CURVED, 0>(rL, m, (T)p.gamma, (T)p.gfac, L);
  side_state<T, CURVED, 0>(rR, m, (T)p.gamma, (T)p.gfac, R);
  hlle_combine<T>(L, R, Fr);
  unrotate_flux(dir, Fr, F);
}

template <class T, int RECON, bool CURVED, int DIR, class S>
__device__ __forceinline__ void face_flux(const DevGrid& g, const DevParams& p, const S& src, long long c, T F[8]) {
  const long long stride = (DIR == 0) ? 1 : ((DIR == 1) ? g.sy : g.sz);
  T pL[8], pR[8];
  reconstruct_face<T, RECON, S>(src, g.ncell, c, stride, (T)p.weno_eps, pL, pR);
  Geom<T> m;
  if (CURVED) face_geometry<T, DIR>(src, g.ncell, c, stride, m);
  // A face state with rho <= 0, P <= 0 or v^2 >= 1 falls back to the state of
  // the cell it was reconstructed from (rare; WENO5 overshoot at sharp
  // gradients of under-resolved data).
  if (!physical_state<T, CURVED>(pL, m)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pL[q] = ld_prim<T>(src, q * g.ncell + c - stride);
  }
  if (!physical_state<T, CURVED>(pR, m)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pR[q] = ld_prim<T>(src, q * g.ncell + c);
  }
  Side<T> L, R;
  side_state<T, CURVED, DIR>(pL, m, (T)p.gamma, (T)p.gfac, L);
  side_state<T, CURVED, DIR>(pR, m, (T)p.gamma, (T)p.gfac, R);
  hlle_combine<T>(L, R, F);
}

// Eq. 13 in 3+1 form for a static-in-time lapse and shift:
//   S_{S_j} = alpha sqrt(gamma) [ T^00 (beta^i beta^k d_j g_ik / 2 - alpha d_j alpha)
//             + T^0i beta^k d_j g_ik + T^0_i d_j beta^i + T^ik d_j g_ik / 2 ]
//   S_tau   = alpha sqrt(gamma) [ T^00 (beta^i beta^j K_ij - beta^i d_i alpha)
//             + T^0i (2 beta^j K_ij - d_i alpha) + T^ij K_ij ]
// Metric derivatives by 4th-order centred differences of the cell-centred
// metric; the spatial inverse and sqrt(gamma) in FP64.
// Eq. 13 in 3+1 form for a static-in-time lapse and shift:
//   S_{S_j} = alpha sqrt(gamma) [ T^00 (beta^i beta^k d_j g_ik / 2 - alpha d_j alpha)
//             + T^0i beta^k d_j g_ik + T^0_i d_j beta^i + T^ik d_j g_ik / 2 ]
//   S_tau   = alpha sqrt(gamma) [ T^00 (beta^i beta^j K_ij - beta^i d_i alpha)
//             + T^0i (2 beta^j K_ij - d_i alpha) + T^ij K_ij ]
// from the cell's metric (alpha, beta, gamma_ij, sqrt(gamma), gamma^ij) and
// the metric derivatives dA[e][q].
template <class T, class S>
__device__ __forceinline__ void source_core(const DevGrid& g, const DevParams& p, const S& src, long long c,
                                            const T alpha, const T beta[3], const T gm[6], const T sg, const T gu[6],
                                            const T dA[3][10], T out[8]) {
  // fluid at the cell centre
  const T rho = ld_prim<T>(src, c), P = ld_prim<T>(src, c + 4 * g.ncell);
  const T v[3] = {ld_prim<T>(src, c + g.ncell), ld_prim<T>(src, c + 2 * g.ncell), ld_prim<T>(src, c + 3 * g.ncell)};
  const T B[3] = {ld_prim<T>(src, c + 5 * g.ncell), ld_prim<T>(src, c + 6 * g.ncell),
                  ld_prim<T>(src, c + 7 * g.ncell)};
  T vl[3], Bl[3], bl_[3];
  lower(gm, v, vl);
  lower(gm, B, Bl);
  (void)bl_;
  const T v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  const T Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const T B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const T omv2 = T(1) - v2;
  const T W = xrsqrt(omv2);
  const T iW = omv2 * W;
  const T ab0 = W * Bv;
  const T b2 = B2 * omv2 + Bv * Bv;
  const T hs = rho + (T)p.gfac * P + b2;
  const T Ps = P + T(0.5) * b2;
  const T ia = T(1) / alpha;
  const T ia2 = ia * ia;
  const T b0 = ab0 * ia;
  T vt[3], bu[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vt[i] = v[i] - beta[i] * ia;
    bu[i] = B[i] * iW + ab0 * vt[i];
  }
  const T hW2 = hs * W * W;
  const T T00 = (hW2 - Ps) * ia2 - b0 * b0;
  T T0[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) T0[i] = hW2 * vt[i] * ia + Ps * beta[i] * ia2 - b0 * bu[i];
  // T^{ij}, symmetric, packed like gamma
  const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
  T Tij[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = I6[s], j = J6[s];
    Tij[s] = hW2 * vt[i] * vt[j] + Ps * (gu[s] - beta[i] * beta[j] * ia2) - bu[i] * bu[j];
  }
  T betal[3];
  lower(gm, beta, betal);
  T T0l[3];  // T^0_i = beta_i T^00 + gamma_ij T^0j
  lower(gm, T0, T0l);
#pragma unroll
  for (int i = 0; i < 3; ++i) T0l[i] += betal[i] * T00;
  const T asg = alpha * sg;
  // symmetric contraction weights: off-diagonal entries count twice
  const T wsym[6] = {T(1), T(2), T(2), T(1), T(2), T(1)};
  out[0] = T(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T bbdg = T(0), t0dg = T(0), tdg = T(0);
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const int i = I6[s], k = J6[s];
      const T dg = dA[j][4 + s] * wsym[s];
      bbdg += beta[i] * beta[k] * dg;
      // T^0i beta^k d_j g_ik summed over i, k: symmetric part
      t0dg += T(0.5) * (T0[i] * beta[k] + T0[k] * beta[i]) * dg;
      tdg += Tij[s] * dg;
    }
    const T t0db = T0l[0] * dA[j][1] + T0l[1] * dA[j][2] + T0l[2] * dA[j][3];
    out[1 + j] = asg * (T00 * (T(0.5) * bbdg - alpha * dA[j][0]) + t0dg + t0db + T(0.5) * tdg);
  }
  {
    T t = -(T0[0] * dA[0][0] + T0[1] * dA[1][0] + T0[2] * dA[2][0]);
    t -= T00 * (beta[0] * dA[0][0] + beta[1] * dA[1][0] + beta[2] * dA[2][0]);
    if (src.kij) {
      T K[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) K[s] = (T)__ldg(src.kij + s * g.ncell + c);
      T bK[3];
      lower(K, beta, bK);  // K_ij beta^j
      const T bbK = beta[0] * bK[0] + beta[1] * bK[1] + beta[2] * bK[2];
      const T tK = T0[0] * bK[0] + T0[1] * bK[1] + T0[2] * bK[2];
      T TK = T(0);
#pragma unroll
      for (int s = 0; s < 6; ++s) TK += Tij[s] * K[s] * wsym[s];
      t += T00 * bbK + T(2) * tK + TK;
    }
    out[4] = asg * t;
  }
  out[5] = out[6] = out[7] = T(0);
}

// Metric quantities from the FP64 inputs: inverse and sqrt(gamma) in FP64,
// 4th-order centred differences of the cell-centred metric.
template <class T>
__device__ __forceinline__ void source_terms(const DevGrid& g, const DevParams& p, const SrcF64& src, long long c,
                                             T out[8]) {
  const double* __restrict__ metric = src.metric;
  double a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = __ldg(metric + q * g.ncell + c);
  const double gxx = a[4], gxy = a[5], gxz = a[6], gyy = a[7], gyz = a[8], gzz = a[9];
  const double cxx = gyy * gzz - gyz * gyz, cxy = gxz * gyz - gxy * gzz, cxz = gxy * gyz - gxz * gyy;
  const double cyy = gxx * gzz - gxz * gxz, cyz = gxy * gxz - gxx * gyz, czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx + gxy * cxy + gxz * cxz;
  const double idet = 1.0 / det;
  const T sg = (T)sqrt(det);
  const T gu[6] = {(T)(cxx * idet), (T)(cxy * idet), (T)(cxz * idet),
                   (T)(cyy * idet), (T)(cyz * idet), (T)(czz * idet)};
  const T alpha = (T)a[0];
  const T beta[3] = {(T)a[1], (T)a[2], (T)a[3]};
  const T gm[6] = {(T)gxx, (T)gxy, (T)gxz, (T)gyy, (T)gyz, (T)gzz};
  // derivatives d[e][q] of the 10 metric components
  T dA[3][10];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const long long s = (e == 0) ? 1 : ((e == 1) ? g.sy : g.sz);
    const double w = g.idx[e] * (1.0 / 12.0);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const double* m = metric + q * g.ncell + c;
      dA[e][q] = (T)((8.0 * (__ldg(m + s) - __ldg(m - s)) - (__ldg(m + 2 * s) - __ldg(m - 2 * s))) * w);
    }
  }
  source_core<T, SrcF64>(g, p, src, c, alpha, beta, gm, sg, gu, dA, out);
}

// Metric quantities from the geometry cache.
template <class T, class PT, class GT>
__device__ __forceinline__ void source_terms(const DevGrid& g, const DevParams& p, const SrcCacheT<PT, GT>& src,
                                             long long c, T out[8]) {
  const GT* gc = src.geom;
  const long long n = g.ncell;
  const T alpha = (T)__ldg(gc + c);
  const T beta[3] = {(T)__ldg(gc + n + c), (T)__ldg(gc + 2 * n + c), (T)__ldg(gc + 3 * n + c)};
  T gm[6], gu[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    gm[i] = (T)__ldg(gc + (4 + i) * n + c);
    gu[i] = (T)__ldg(gc + (17 + i) * n + c);
  }
  const T sg = (T)__ldg(gc + 16 * n + c);
  T dA[3][10];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int q = 0; q < 10; ++q) dA[e][q] = (T)__ldg(gc + (23 + 10 * e + q) * n + c);
  source_core<T, SrcCacheT<PT, GT>>(g, p, src, c, alpha, beta, gm, sg, gu, dA, out);
}

// Tile shapes the kernels are instantiated for (cells per axis, 256 cells each).
template <int S> struct TileShape;
template <> struct TileShape<0> { static constexpr int X = 8, Y = 8, Z = 4; };
template <> struct TileShape<1> { static constexpr int X = 16, Y = 4, Z = 4; };
template <> struct TileShape<2> { static constexpr int X = 32, Y = 4, Z = 2; };
template <> struct TileShape<3> { static constexpr int X = 4, Y = 8, Z = 8; };
template <> struct TileShape<4> { static constexpr int X = 8, Y = 8, Z = 8; };  // 2 cells per thread
constexpr int kNumTileShapes = 5;
constexpr int kTileThreads = 256;

template <int TX, int TY, int TZ>
struct TileFaces {
  static constexpr int NFX = (TX + 1) * TY * TZ;
  static constexpr int NFY = TX * (TY + 1) * TZ;
  static constexpr int NFZ = TX * TY * (TZ + 1);
  static constexpr int NF = NFX + NFY + NFZ;
};
// Largest face count over the 256-cell shapes 0..3 (the batched kernel's
// shared face buffer); single-block launches size it per shape.
constexpr int kMaxTileFaces = 968;

// One tile of the RHS: all face fluxes of the tile (each once) into the
// shared buffer sF [8][NF], then each thread differences its cell's faces,
// adds the sources and applies the stage epilogue.  Called by all threads of
// the CTA (contains __syncthreads); kTileThreads threads, each handling one
// or more cells of the TX*TY*TZ tile.
template <class T, int RECON, bool CURVED, int TX, int TY, int TZ, class S>
__device__ __forceinline__ void rhs_tile(const DevGrid& g, const DevParams& p, const S& src, const StageEpilogue& ep,
                                         int x0, int y0, int z0, T* sF) {
  constexpr int NT = kTileThreads;
  constexpr int NC = TX * TY * TZ;
  constexpr int NFX = TileFaces<TX, TY, TZ>::NFX;
  constexpr int NFY = TileFaces<TX, TY, TZ>::NFY;
  constexpr int NF = TileFaces<TX, TY, TZ>::NF;
  const int ng = g.ng;
  for (int f = threadIdx.x; f < NF; f += NT) {
    T F[8];
    int dir, xi, yi, zi;
    bool ok;
    if (f < NFX) {
      const int a = f % (TX + 1), r = f / (TX + 1);
      dir = 0;
      xi = x0 + a; yi = y0 + r % TY; zi = z0 + r / TY;
      ok = (xi <= g.n[0]) && (yi < g.n[1]) && (zi < g.n[2]);
    } else if (f < NFX + NFY) {
      const int ff = f - NFX;
      const int r = ff / TX;
      dir = 1;
      xi = x0 + ff % TX; yi = y0 + r % (TY + 1); zi = z0 + r / (TY + 1);
      ok = (xi < g.n[0]) && (yi <= g.n[1]) && (zi < g.n[2]);
    } else {
      const int ff = f - NFX - NFY;
      const int r = ff / TX;
      dir = 2;
      xi = x0 + ff % TX; yi = y0 + r % TY; zi = z0 + r / TY;
      ok = (xi < g.n[0]) && (yi < g.n[1]) && (zi <= g.n[2]);
    }
    if (ok) {
      const long long c = (long long)(zi + ng) * g.sz + (long long)(yi + ng) * g.sy + (xi + ng);
      face_flux_rt<T, RECON, CURVED, S>(g, p, src, c, dir, F);
    }
    if (ok) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sF[q * NF + f] = F[q];
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int cl = threadIdx.x; cl < NC; cl += NT) {
  const int ci = cl % TX, cj = (cl / TX) % TY, ck = cl / (TX * TY);
  const int xi = x0 + ci, yi = y0 + cj, zi = z0 + ck;
  if (xi < g.n[0] && yi < g.n[1] && zi < g.n[2]) {
    const long long c = (long long)(zi + ng) * g.sz + (long long)(yi + ng) * g.sy + (xi + ng);
    const int fx = (ck * TY + cj) * (TX + 1) + ci;
    const int fy = NFX + (ck * (TY + 1) + cj) * TX + ci;
    const int fz = NFX + NFY + (ck * TY + cj) * TX + ci;
    const T ix = (T)g.idx[0], iy = (T)g.idx[1], iz = (T)g.idx[2];
    T r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const T* s = sF + q * NF;
      T acc = -(s[fx + 1] - s[fx]) * ix;
      acc -= (s[fy + TX] - s[fy]) * iy;
      acc -= (s[fz + TX * TY] - s[fz]) * iz;
      r[q] = acc;
    }
    if (CURVED) {
      T sv[8];
      source_terms<T>(g, p, src, c, sv);
#pragma unroll
      for (int q = 0; q < 8; ++q) r[q] += sv[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long o = q * g.ncell + c;
      const double rq = (double)r[q];
      if (ep.rhs) ep.rhs[o] = rq;
      const double ain = ep.acc_in ? ep.acc_in[o] : 0.0;
      if (ep.u) ep.u[o] = ep.c0 * ep.u0[o] + ep.c1 * ep.u[o] + ep.cr * rq + ep.ca * ain;
      if (ep.acc_out) ep.acc_out[o] = ep.wa * ain + ep.wr * rq;
    }
  }
  }
}

// Resident CTAs per SM the register budget is fitted to: 3 for the FP32
// (mixed) kernels, which are latency bound, 1 for FP64 (pipe bound).
template <class T>
struct MinCtas { static constexpr int value = sizeof(T) == 4 ? 3 : 1; };

template <class T, int RECON, bool CURVED, int SHAPE, class S>
__global__ void __launch_bounds__(kTileThreads, MinCtas<T>::value) rhs_kernel(DevGrid g, DevParams p, S src,
                                                                             StageEpilogue ep) {
  using TS = TileShape<SHAPE>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  rhs_tile<T, RECON, CURVED, TS::X, TS::Y, TS::Z, S>(g, p, src, ep, blockIdx.x * TS::X, blockIdx.y * TS::Y,
                                                      blockIdx.z * TS::Z, sF);
}

template <class T, int RECON, bool CURVED, class S>
cudaError_t launch_rhs_shape(int shape, const DevGrid& g, const DevParams& p, const S& src, const StageEpilogue& ep,
                             cudaStream_t s) {
  void (*k)(DevGrid, DevParams, S, StageEpilogue) = nullptr;
  int tx = 8, ty = 8, tz = 4;
  int nf = TileFaces<8, 8, 4>::NF;
  switch (shape) {
    case 4: k = rhs_kernel<T, RECON, CURVED, 4, S>; tx = TileShape<4>::X; ty = TileShape<4>::Y; tz = TileShape<4>::Z;
            nf = TileFaces<8, 8, 8>::NF; break;
    case 1: k = rhs_kernel<T, RECON, CURVED, 1, S>; tx = TileShape<1>::X; ty = TileShape<1>::Y; tz = TileShape<1>::Z; break;
    case 2: k = rhs_kernel<T, RECON, CURVED, 2, S>; tx = TileShape<2>::X; ty = TileShape<2>::Y; tz = TileShape<2>::Z; break;
    case 3: k = rhs_kernel<T, RECON, CURVED, 3, S>; tx = TileShape<3>::X; ty = TileShape<3>::Y; tz = TileShape<3>::Z; break;
    default: k = rhs_kernel<T, RECON, CURVED, 0, S>; break;
  }
  if (shape >= 1 && shape <= 3) nf = kMaxTileFaces;
  const size_t smem = (size_t)8 * nf * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((g.n[0] + tx - 1) / tx, (g.n[1] + ty - 1) / ty, (g.n[2] + tz - 1) / tz);
  k<<<grid, kTileThreads, smem, s>>>(g, p, src, ep);
  return cudaGetLastError();
}

// Host-side launcher for one precision and input source.
template <class T, class S>
cudaError_t launch_rhs_src(const DevGrid& g, const DevParams& p, const S& src, bool curved, const StageEpilogue& ep,
                           cudaStream_t s) {
  const int shape = p.tile;
  if (p.recon == GRMHD_WENO5)
    return curved ? launch_rhs_shape<T, GRMHD_WENO5, true, S>(shape, g, p, src, ep, s)
                  : launch_rhs_shape<T, GRMHD_WENO5, false, S>(shape, g, p, src, ep, s);
  return curved ? launch_rhs_shape<T, GRMHD_MINMOD, true, S>(shape, g, p, src, ep, s)
                : launch_rhs_shape<T, GRMHD_MINMOD, false, S>(shape, g, p, src, ep, s);
}

template <class T>
cudaError_t launch_rhs_t(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                         const double* kij, const StageEpilogue& ep, cudaStream_t s) {
  SrcF64 src;
  src.prim = prim;
  src.metric = metric;
  src.kij = kij;
  return launch_rhs_src<T, SrcF64>(g, p, src, metric != nullptr, ep, s);
}

}  // namespace grmhd
