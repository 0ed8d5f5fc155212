// Fused method-of-lines RHS kernel: reconstruction + face metric + HLLE +
// flux divergence + source terms + RK stage epilogue, one launch.
//
// Work decomposition: a CTA owns a TX x TY x TZ tile of interior cells.  It
// computes every face flux of the tile exactly once -- (TX+1) TY TZ x-faces,
// TX (TY+1) TZ y-faces, TX TY (TZ+1) z-faces, one flat list spread over all
// threads -- into shared memory (SoA [comp][face], conflict-free), then each
// thread differences the six faces of its cell, adds the Eq. 13 source
// (3+1 form, curved metric only) and applies the stage epilogue.  For FP64
// WENO5 the reconstruction runs per cell before the face pass: every cell of
// the tile extended by one along each direction forms its face states from
// one stencil into a shared-memory stage, which the faces then read.  One
// face routine serves all three directions, the states, metric and flux
// being relabelled so that the face normal is the first axis.
#pragma once

#include <type_traits>

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
//   FP64 cache (the FP64 RHS is bound by its FP64 instructions: the face
//   metric read whole saves ten additions and a division per face):
//   53..82  the metric on the lower d-face of the point, 0.5 a_below + 0.5 a
//           (index 53 + 10 d + q; the two halvings are exact, so the value
//           has the bits of the mean of the two cells)
//   83..85  1 / alpha on the lower d-face
//   86..107 the metric factors of the sources at the point (SrcStatics:
//           1/alpha, 1/alpha^2, beta^i / alpha^2, gamma^ij - beta^i beta^j /
//           alpha^2, beta_i, alpha sqrt(gamma), beta^i beta^j, beta^i d_i alpha)
//   FP32 cache (the FP32 RHS is latency bound: ten arrays that all three
//   face directions share stay in L1 better than thirty):
//   53..62  half the metric values, 0.5 (alpha, beta^i, gamma_ij): a face's
//           metric is the sum of its two cells' entries
static_assert(kGeomCacheComps == 108 && kGeomCacheFace == 53 && kGeomCacheFaceIa == 83 && kGeomCacheHalf32 == 53 &&
                  kGeomCacheStat == 86,
              "geometry cache layout");

// (SrcStatics and source_statics, the metric factors of the sources: physics.cuh)

// SrcStatics as stored in the FP64 geometry cache (component k at index
// kGeomCacheStat + k, in the order of the struct).
template <class T>
__device__ __forceinline__ void load_statics(const double* __restrict__ gc, long long n, long long c,
                                             SrcStatics<T>& st) {
  const double* q = gc + (long long)kGeomCacheStat * n + c;
  st.ia = (T)__ldg(q);
  st.ia2 = (T)__ldg(q + n);
#pragma unroll
  for (int i = 0; i < 3; ++i) st.bia2[i] = (T)__ldg(q + (2 + i) * n);
#pragma unroll
  for (int s = 0; s < 6; ++s) st.M[s] = (T)__ldg(q + (5 + s) * n);
#pragma unroll
  for (int i = 0; i < 3; ++i) st.betal[i] = (T)__ldg(q + (11 + i) * n);
  st.asg = (T)__ldg(q + 14 * n);
#pragma unroll
  for (int s = 0; s < 6; ++s) st.bb[s] = (T)__ldg(q + (15 + s) * n);
  st.bda = (T)__ldg(q + 21 * n);
}

// SrcF64 whose primitives are written in the same launch (the one-launch
// batch: recovered and ghost-filled by other CTAs before the tile reads
// them): the primitives are read through L2 (ld.global.cg), not the
// read-only path, which is not coherent with writes made during a launch.
// The metric stays read-only.
struct SrcF64Co : SrcF64 {};

template <class T>
__device__ __forceinline__ T ld_prim(const SrcF64& s, long long i) { return (T)__ldg(s.prim + i); }
template <class T>
__device__ __forceinline__ T ld_prim(const SrcF64Co& s, long long i) { return (T)__ldcg(s.prim + i); }
template <class T, class GT>
__device__ __forceinline__ T ld_prim(const SrcCacheT<double, GT>& s, long long i) { return (T)__ldg(s.prim + i); }

// Primitive q of point i.  The FP64 sources hold the primitives as
// [q][ncell]; the FP32 copy of the mixed path (SrcCacheT<float, GT>) holds
// them in pairs, [q/2][ncell] float2 (q even in .x, q odd in .y), so that
// the two variables of a paired FP32 instruction (weno5_x2) arrive in one
// 8-byte load.
template <class T, class S>
__device__ __forceinline__ T ld_pq(const S& s, long long ncell, int q, long long i) {
  return ld_prim<T>(s, q * ncell + i);
}
template <class T, class GT>
__device__ __forceinline__ T ld_pq(const SrcCacheT<float, GT>& s, long long ncell, int q, long long i) {
  return (T)__ldg(s.prim + 2 * ((q >> 1) * ncell + i) + (q & 1));
}
// Primitives 2h and 2h+1 of point i.
template <class S>
__device__ __forceinline__ float2 ld_pair(const S& s, long long ncell, int h, long long i) {
  return make_float2(ld_pq<float>(s, ncell, 2 * h, i), ld_pq<float>(s, ncell, 2 * h + 1, i));
}
template <class GT>
__device__ __forceinline__ float2 ld_pair(const SrcCacheT<float, GT>& s, long long ncell, int h, long long i) {
  return __ldg(reinterpret_cast<const float2*>(s.prim) + h * ncell + i);
}

// Load the 8 primitives at the six-point stencil of the face between cell
// c - stride and c, reconstruct both states.
template <class T, int RECON, class S>
__device__ __forceinline__ void reconstruct_face(const S& src, long long ncell, long long c, long long stride, T eps,
                                                 T pL[8], T pR[8]) {
  if constexpr (RECON == GRMHD_WENO5 && sizeof(T) == 8) {
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
  } else if constexpr (RECON == GRMHD_WENO5 && sizeof(T) == 4) {
    // FP32: two variables per paired instruction (weno5_x2, the bits of weno5<float>)
    const float2 e2 = make_float2(eps, eps);
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const int h = q >> 1;
      const float2 um3 = ld_pair(src, ncell, h, c - 3 * stride), um2 = ld_pair(src, ncell, h, c - 2 * stride);
      const float2 um1 = ld_pair(src, ncell, h, c - stride), u0 = ld_pair(src, ncell, h, c);
      const float2 up1 = ld_pair(src, ncell, h, c + stride), up2 = ld_pair(src, ncell, h, c + 2 * stride);
      const float2 vL = weno5_x2(um3, um2, um1, u0, up1, e2);
      const float2 vR = weno5_x2(up2, up1, u0, um1, um2, e2);
      pL[q] = vL.x;
      pL[q + 1] = vL.y;
      pR[q] = vR.x;
      pR[q + 1] = vR.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if constexpr (RECON == GRMHD_WENO5) {
        const T um3 = ld_pq<T>(src, ncell, q, c - 3 * stride), um2 = ld_pq<T>(src, ncell, q, c - 2 * stride);
        const T um1 = ld_pq<T>(src, ncell, q, c - stride), u0 = ld_pq<T>(src, ncell, q, c);
        const T up1 = ld_pq<T>(src, ncell, q, c + stride), up2 = ld_pq<T>(src, ncell, q, c + 2 * stride);
        weno5_pair<T>(um3, um2, um1, u0, up1, up2, eps, pL[q], pR[q]);
      } else {
        const T um2 = ld_pq<T>(src, ncell, q, c - 2 * stride), um1 = ld_pq<T>(src, ncell, q, c - stride);
        const T u0 = ld_pq<T>(src, ncell, q, c), up1 = ld_pq<T>(src, ncell, q, c + stride);
        pL[q] = um1 + T(0.5) * minmod<T>(um1 - um2, u0 - um1);
        pR[q] = u0 - T(0.5) * minmod<T>(u0 - um1, up1 - u0);
      }
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

// FP64 WENO5: both states of cell c for the primitives 2h and 2h+1 into v
// (minus and plus of 2h, then of 2h+1); the four values share one division.
template <class S>
__device__ __forceinline__ void weno5_cell_pair_states(const S& src, long long ncell, long long c, long long stride,
                                                       int h, double eps13, double v[4]) {
  double nm[2], dm[2], np[2], dp[2], u0[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const long long a = (2 * h + k) * ncell + c;
    u0[k] = ld_prim<double>(src, a);
    weno5_cell_parts(ld_prim<double>(src, a - 2 * stride), ld_prim<double>(src, a - stride), u0[k],
                     ld_prim<double>(src, a + stride), ld_prim<double>(src, a + 2 * stride), eps13, nm[k], dm[k],
                     np[k], dp[k]);
  }
  const double a0 = __dmul_rn(dm[0], dp[0]), a1 = __dmul_rn(dm[1], dp[1]);
  const double X = 1.0 / __dmul_rn(__dmul_rn(6.0, a0), a1);
  const double x0 = __dmul_rn(a1, X), x1 = __dmul_rn(a0, X);
  v[0] = weno5_cell_state(u0[0], nm[0], __dmul_rn(dp[0], x0));
  v[1] = weno5_cell_state(u0[0], np[0], __dmul_rn(dm[0], x0));
  v[2] = weno5_cell_state(u0[1], nm[1], __dmul_rn(dp[1], x1));
  v[3] = weno5_cell_state(u0[1], np[1], __dmul_rn(dm[1], x1));
}

// Both reconstructed states of cell c (value at its lower face, "minus", and
// at its upper face, "plus") for the primitives 2h and 2h+1, written to the
// stage buffer sR at [2q][e] (minus) and [2q+1][e] (plus), ne entries per
// component.  eps13 = (12/13) weno_eps (see weno5_cell_parts).
// which: 0 both states, 1 the minus state only, 2 the plus state only (the
// cells at the ends of an extended box need one of the two).
template <class T, int RECON, class S>
__device__ __forceinline__ void reconstruct_cell_pair(const S& src, long long ncell, long long c, long long stride,
                                                      int h, T eps13, T* __restrict__ sR, int ne, int e,
                                                      int which = 0) {
  if constexpr (RECON == GRMHD_WENO5 && sizeof(T) == 8) {
    if (which != 0) {
      // one state of each of the two variables; the division as below, so
      // the value is the same to the bit as when both states are formed
      double n[2], dm[2], dp[2], u0[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const long long a = (2 * h + k) * ncell + c;
        u0[k] = ld_prim<double>(src, a);
        weno5_cell_parts_one(ld_prim<double>(src, a - 2 * stride), ld_prim<double>(src, a - stride), u0[k],
                             ld_prim<double>(src, a + stride), ld_prim<double>(src, a + 2 * stride), (double)eps13,
                             which == 2, n[k], dm[k], dp[k]);
      }
      const double a0 = __dmul_rn(dm[0], dp[0]), a1 = __dmul_rn(dm[1], dp[1]);
      const double X = 1.0 / __dmul_rn(__dmul_rn(6.0, a0), a1);
      const double x0 = __dmul_rn(a1, X), x1 = __dmul_rn(a0, X);
      if (which == 2) {
        sR[(4 * h + 1) * ne + e] = (T)weno5_cell_state(u0[0], n[0], __dmul_rn(dm[0], x0));
        sR[(4 * h + 3) * ne + e] = (T)weno5_cell_state(u0[1], n[1], __dmul_rn(dm[1], x1));
      } else {
        sR[(4 * h + 0) * ne + e] = (T)weno5_cell_state(u0[0], n[0], __dmul_rn(dp[0], x0));
        sR[(4 * h + 2) * ne + e] = (T)weno5_cell_state(u0[1], n[1], __dmul_rn(dp[1], x1));
      }
      return;
    }
    double v[4];
    weno5_cell_pair_states<S>(src, ncell, c, stride, h, (double)eps13, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) sR[(4 * h + k) * ne + e] = (T)v[k];
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = 2 * h + k;
      T vm, vp;
      if constexpr (RECON == GRMHD_WENO5) {
        weno5_cell((float)ld_pq<T>(src, ncell, q, c - 2 * stride), (float)ld_pq<T>(src, ncell, q, c - stride),
                   (float)ld_pq<T>(src, ncell, q, c), (float)ld_pq<T>(src, ncell, q, c + stride),
                   (float)ld_pq<T>(src, ncell, q, c + 2 * stride), (float)eps13, vm, vp);
      } else {
        minmod_cell<T>(ld_pq<T>(src, ncell, q, c - stride), ld_pq<T>(src, ncell, q, c),
                       ld_pq<T>(src, ncell, q, c + stride), vm, vp);
      }
      sR[(4 * h + 2 * k) * ne + e] = vm;
      sR[(4 * h + 2 * k + 1) * ne + e] = vp;
    }
  }
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
  if constexpr (sizeof(GT) == 8) {
#pragma unroll
    for (int q = 0; q < 10; ++q) a[q] = (T)__ldg(gm + (kGeomCacheFace + 10 * dir + q) * ncell + c);
  } else {
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const GT* h = gm + (kGeomCacheHalf32 + q) * ncell + c;
      a[q] = (T)__ldg(h - stride) + (T)__ldg(h);
    }
  }
  m.alpha = a[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = a[1 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = a[4 + i];
  m.sqrtg = (T)__ldg(gm + (10 + dir) * ncell + c);
  m.gup_dd = (T)__ldg(gm + (13 + dir) * ncell + c);
  if constexpr (sizeof(GT) == 8) m.ia = (T)__ldg(gm + (kGeomCacheFaceIa + dir) * ncell + c);
  else m.ia = T(1) / m.alpha;
}

// Flux through a face whose normal dir is known only at run time, from its
// reconstructed left / right states: the states and the metric are
// relabelled so the normal is the first axis, one x-face computation runs,
// and the flux is relabelled back (one copy of the face code instead of
// three keeps the kernel small).  c is the cell above the face.
template <class T, bool CURVED, class S, bool POLY = false>
__device__ __forceinline__ void face_flux_states(const DevGrid& g, const DevParams& p, const S& src, long long c,
                                                 int dir, long long stride, T pL[8], T pR[8], T F[8]) {
  // polytrope (a separate instantiation, so that the Gamma-law kernels carry
  // none of it): the face pressure follows from the face density
  if constexpr (POLY) apply_polytrope_pair<T>(p, pL, pR);
  Geom<T> m;
  if (CURVED) face_geometry_rt<T>(src, g.ncell, c, stride, dir, m);
  T rL[8], rR[8], Fr[8];
  Side<T> L, R;
  const T ia = CURVED ? m.ia : T(1);  // 1/alpha of the face, shared by both sides
  if constexpr (sizeof(T) == 8) {
    // FP64 (pipe bound): the check's lowered velocity and v^2 feed the side states
    T vlL[3], vlR[3], v2L, v2R, rvL[3], rvR[3];
    if (!physical_state_v<T, CURVED>(pL, m, vlL, v2L)) {
#pragma unroll
      for (int q = 0; q < 8; ++q) pL[q] = ld_pq<T>(src, g.ncell, q, c - stride);
      physical_state_v<T, CURVED>(pL, m, vlL, v2L);
    }
    if (!physical_state_v<T, CURVED>(pR, m, vlR, v2R)) {
#pragma unroll
      for (int q = 0; q < 8; ++q) pR[q] = ld_pq<T>(src, g.ncell, q, c);
      physical_state_v<T, CURVED>(pR, m, vlR, v2R);
    }
    rotate_state(dir, pL, rL);
    rotate_state(dir, pR, rR);
    rotate_vec(dir, vlL, rvL);
    rotate_vec(dir, vlR, rvR);
    if (CURVED) rotate_metric(dir, m);
    side_state<T, CURVED, 0, true, true>(rL, m, par_t<T>(p.gamma, p.gammaf), par_t<T>(p.gfac, p.gfacf), L, ia, rvL, v2L);
    side_state<T, CURVED, 0, true, true>(rR, m, par_t<T>(p.gamma, p.gammaf), par_t<T>(p.gfac, p.gfacf), R, ia, rvR, v2R);
  } else {
    // FP32: both sides in paired instructions (one side per lane)
    bool okL, okR;
    physical_states_x2<CURVED>(pL, pR, m, okL, okR);
    if (!okL) {
#pragma unroll
      for (int q = 0; q < 8; ++q) pL[q] = ld_pq<T>(src, g.ncell, q, c - stride);
    }
    if (!okR) {
#pragma unroll
      for (int q = 0; q < 8; ++q) pR[q] = ld_pq<T>(src, g.ncell, q, c);
    }
    rotate_state(dir, pL, rL);
    rotate_state(dir, pR, rR);
    if (CURVED) rotate_metric(dir, m);
    side_states_x2<CURVED>(rL, rR, m, p.gammaf, p.gfacf, ia, L, R);
  }
  finish_speeds<T, CURVED, 0>(m, L, R);
  hlle_combine_scaled<T>(L, R, CURVED ? m.alpha : T(1), CURVED ? m.sqrtg : T(1), Fr);
  unrotate_flux(dir, Fr, F);
}

// Eq. 13 in 3+1 form for a static-in-time lapse and shift:
//   S_{S_j} = alpha sqrt(gamma) [ T^00 (beta^i beta^k d_j g_ik / 2 - alpha d_j alpha)
//             + T^0i beta^k d_j g_ik + T^0_i d_j beta^i + T^ik d_j g_ik / 2 ]
//   S_tau   = alpha sqrt(gamma) [ T^00 (beta^i beta^j K_ij - beta^i d_i alpha)
//             + T^0i (2 beta^j K_ij - d_i alpha) + T^ij K_ij ]
// from the cell's metric (alpha, beta, gamma_ij, sqrt(gamma), gamma^ij) and
// the metric derivatives dA[e][q].
template <class T, class S>
__device__ __forceinline__ void source_core(const DevGrid& g, const DevParams& p, const S& src, long long c,
                                            const T alpha, const T beta[3], const T gm[6], const T dA[3][10],
                                            const SrcStatics<T>& st, T out[8]) {
  // fluid at the cell centre
  const long long n = g.ncell;
  const T rho = ld_pq<T>(src, n, 0, c), P = ld_pq<T>(src, n, 4, c);
  const T v[3] = {ld_pq<T>(src, n, 1, c), ld_pq<T>(src, n, 2, c), ld_pq<T>(src, n, 3, c)};
  const T B[3] = {ld_pq<T>(src, n, 5, c), ld_pq<T>(src, n, 6, c), ld_pq<T>(src, n, 7, c)};
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
  const T hs = rho + par_t<T>(p.gfac, p.gfacf) * P + b2;
  const T Ps = P + T(0.5) * b2;
  const T ia = st.ia, ia2 = st.ia2;
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
  for (int i = 0; i < 3; ++i) T0[i] = hW2 * vt[i] * ia + Ps * st.bia2[i] - b0 * bu[i];
  // T^{ij}, symmetric, packed like gamma
  const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
  T Tij[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = I6[s], j = J6[s];
    Tij[s] = hW2 * vt[i] * vt[j] + Ps * st.M[s] - bu[i] * bu[j];
  }
  T T0l[3];  // T^0_i = beta_i T^00 + gamma_ij T^0j
  lower(gm, T0, T0l);
#pragma unroll
  for (int i = 0; i < 3; ++i) T0l[i] += st.betal[i] * T00;
  const T asg = st.asg;
  // symmetric contraction weights: off-diagonal entries count twice
  const T wsym[6] = {T(1), T(2), T(2), T(1), T(2), T(1)};
  out[0] = T(0);
  // The momentum source is sum_{ik} d_j gamma_ik [T00 beta^i beta^k / 2 +
  // T^0i beta^k + T^ik / 2] - T00 alpha d_j alpha + T^0_i d_j beta^i; the
  // bracket does not depend on j, so it is formed once per packed (i, k),
  // with the symmetric weight and the factor 1/2 folded in.
  T Wg[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = I6[s], k = J6[s];
    Wg[s] = (T(0.5) * wsym[s]) * (T00 * st.bb[s] + (T0[i] * beta[k] + T0[k] * beta[i]) + Tij[s]);
  }
  const T T00a = T00 * alpha;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T acc = T0l[0] * dA[j][1] + T0l[1] * dA[j][2] + T0l[2] * dA[j][3] - T00a * dA[j][0];
#pragma unroll
    for (int s = 0; s < 6; ++s) acc += Wg[s] * dA[j][4 + s];
    out[1 + j] = asg * acc;
  }
  {
    T t = -(T0[0] * dA[0][0] + T0[1] * dA[1][0] + T0[2] * dA[2][0]);
    t -= T00 * st.bda;
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
// 4th-order centred differences of the cell-centred metric (S: SrcF64 or
// SrcF64Co, which differ in how the primitives are read).
template <class T, class S>
__device__ __forceinline__ void source_terms_f64(const DevGrid& g, const DevParams& p, const S& src, long long c,
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
  SrcStatics<T> st;
  const T da[3] = {dA[0][0], dA[1][0], dA[2][0]};
  source_statics<T>(alpha, beta, gm, sg, gu, da, st);
  source_core<T, S>(g, p, src, c, alpha, beta, gm, dA, st, out);
}

template <class T>
__device__ __forceinline__ void source_terms(const DevGrid& g, const DevParams& p, const SrcF64& src, long long c,
                                             T out[8]) {
  source_terms_f64<T, SrcF64>(g, p, src, c, out);
}
template <class T>
__device__ __forceinline__ void source_terms(const DevGrid& g, const DevParams& p, const SrcF64Co& src, long long c,
                                             T out[8]) {
  source_terms_f64<T, SrcF64Co>(g, p, src, c, out);
}

// A value the cell phase reads once (the sources' geometry, the stage
// update's U0 and U): the FP32 kernels read it through L2 only
// (ld.global.cg), leaving L1 to the primitive stencils and face metrics that
// the face pass re-reads (measured: the FP32 RHS is sensitive to L1 space);
// the FP64 kernels, bound by the FP64 pipe, keep the read-only path.
template <bool L2ONLY, class V>
__device__ __forceinline__ V ld_once(const V* p) {
  if constexpr (L2ONLY) return __ldcg(p);
  else return __ldg(p);
}

// Metric quantities from the geometry cache.
template <class T, class PT, class GT>
__device__ __forceinline__ void source_terms(const DevGrid& g, const DevParams& p, const SrcCacheT<PT, GT>& src,
                                             long long c, T out[8]) {
  constexpr bool F32 = sizeof(GT) == 4;
  const GT* gc = src.geom;
  const long long n = g.ncell;
  const T alpha = (T)ld_once<F32>(gc + c);
  const T beta[3] = {(T)ld_once<F32>(gc + n + c), (T)ld_once<F32>(gc + 2 * n + c), (T)ld_once<F32>(gc + 3 * n + c)};
  T gm[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) gm[i] = (T)ld_once<F32>(gc + (4 + i) * n + c);
  T dA[3][10];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int q = 0; q < 10; ++q) dA[e][q] = (T)ld_once<F32>(gc + (23 + 10 * e + q) * n + c);
  SrcStatics<T> st;
  if constexpr (sizeof(GT) == 8) {
    // FP64 cache: the metric factors formed once (the FP64 sources are bound by the FP64 pipe)
    load_statics<T>(gc, n, c, st);
  } else {
    T gu[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) gu[i] = (T)ld_once<F32>(gc + (17 + i) * n + c);
    const T sg = (T)ld_once<F32>(gc + 16 * n + c);
    const T da[3] = {dA[0][0], dA[1][0], dA[2][0]};
    source_statics<T>(alpha, beta, gm, sg, gu, da, st);
  }
  source_core<T, SrcCacheT<PT, GT>>(g, p, src, c, alpha, beta, gm, dA, st, out);
}

// A compute-type RHS value in FP64 for the stage epilogue: FP32 is widened on
// the integer pipe (fpbits.cuh), which on this GPU would otherwise take an
// FP64-pipe slot per value.  The result is the exact FP64 value, except that
// FP32 subnormals (magnitude below 2^-126) become zero.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64i(x); }

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
// Reconstruction stage: per direction, the tile extended by one cell on
// both sides along that direction (EXX, EYY, EZZ cells); NE is the largest
// of the three, NEA their sum.
template <int TX, int TY, int TZ>
struct TileStage {
  static constexpr int EXX = (TX + 2) * TY * TZ, EYY = TX * (TY + 2) * TZ, EZZ = TX * TY * (TZ + 2);
  static constexpr int NE = EXX > EYY ? (EXX > EZZ ? EXX : EZZ) : (EYY > EZZ ? EYY : EZZ);
  static constexpr int NEA = EXX + EYY + EZZ;
};

// Reconstruction per cell (both face states of a cell from one stencil,
// staged in shared memory) pays off where the reconstruction dominates:
// FP64 WENO5.  FP32 and minmod reconstruct per face, inline.
template <class T, int RECON>
struct CellRecon { static constexpr bool value = RECON == GRMHD_WENO5 && sizeof(T) == 8; };

constexpr size_t kMaxTileSmem = 227 * 1024;

// Stage layout of a tile: all three directions at once (one face pass over
// every face of the tile) when the shared memory allows, else one direction
// at a time (three face passes).
template <class T, int RECON, int TX, int TY, int TZ>
struct TileSmem {
  static constexpr size_t faces = (size_t)8 * TileFaces<TX, TY, TZ>::NF * sizeof(T);
  static constexpr size_t all = faces + (size_t)16 * TileStage<TX, TY, TZ>::NEA * sizeof(T);
  static constexpr bool stage_all = CellRecon<T, RECON>::value && all <= kMaxTileSmem;
  static constexpr size_t bytes = !CellRecon<T, RECON>::value
                                      ? faces
                                      : (stage_all ? all : faces + (size_t)16 * TileStage<TX, TY, TZ>::NE * sizeof(T));
  // stage entries per component
  static constexpr int ns = stage_all ? TileStage<TX, TY, TZ>::NEA : TileStage<TX, TY, TZ>::NE;
};

template <class T, int RECON, int TX, int TY, int TZ>
constexpr size_t tile_smem_bytes() { return TileSmem<T, RECON, TX, TY, TZ>::bytes; }

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// Batched kernel (one buffer for the shapes 0..3): face buffer
// [8][kMaxTileFaces], then the stage [16][batch_stage_entries].
constexpr int kMaxTileFaces = 968;  // largest NF over the shapes 0..3
template <class T, int RECON>
constexpr int batch_stage_entries() {
  return !CellRecon<T, RECON>::value
             ? 0
             : (int)cmax(cmax(TileSmem<T, RECON, 8, 8, 4>::ns, TileSmem<T, RECON, 16, 4, 4>::ns),
                         cmax(TileSmem<T, RECON, 32, 4, 2>::ns, TileSmem<T, RECON, 4, 8, 8>::ns));
}
template <class T, int RECON>
constexpr size_t batch_smem_bytes() {
  return (size_t)(8 * kMaxTileFaces + 16 * batch_stage_entries<T, RECON>()) * sizeof(T);
}

// Flux of the face between cell c - stride and cell c along dir, as the
// RHS kernels compute it with per-face reconstruction (used outside the
// tiles: AMR interface faces, constrained-transport ring faces).
template <int RECON, bool CURVED, bool POLY = false>
__device__ __forceinline__ void face_flux_one(const DevGrid& g, const DevParams& p, const double* prim,
                                              const double* metric, long long c, int dir, double F[8]) {
  SrcF64 src;
  src.prim = prim;
  src.metric = metric;
  src.kij = nullptr;
  const long long stride = dir == 0 ? 1 : (dir == 1 ? g.sy : g.sz);
  double pL[8], pR[8];
  reconstruct_face<double, RECON, SrcF64>(src, g.ncell, c, stride, p.weno_eps, pL, pR);
  face_flux_states<double, CURVED, SrcF64, POLY>(g, p, src, c, dir, stride, pL, pR, F);
}

// Flux of the dir-face at tile face coordinates (fx, fy, fz), i.e. the
// lower dir-face of tile cell (fx, fy, fz) (fx = TX etc. for the tile's
// upper boundary faces), into F; false (F untouched) outside the block.
// With a stage, the face states come from sR (stage index of the cell below
// the face: eoff[dir] + its index in that direction's extended box);
// otherwise they are reconstructed here.  cell: array index of the cell
// above the face.
template <class T, int RECON, bool CURVED, int TX, int TY, int TZ, class S, bool POLY = false>
__device__ __forceinline__ bool tile_face_at(const DevGrid& g, const DevParams& p, const S& src, int x0, int y0,
                                             int z0, int dir, int fx, int fy, int fz, const T* __restrict__ sR, int ns,
                                             int eoff_y, int eoff_z, T F[8], long long& cell) {
  const int ux = dir == 0, uy = dir == 1, uz = dir == 2;
  const int xi = x0 + fx, yi = y0 + fy, zi = z0 + fz;
  if (!(xi < g.n[0] + ux && yi < g.n[1] + uy && zi < g.n[2] + uz)) return false;
  const int ng = g.ng;
  const long long c = (long long)(zi + ng) * g.sz + (long long)(yi + ng) * g.sy + (xi + ng);
  const long long stride = (dir == 0) ? 1 : ((dir == 1) ? g.sy : g.sz);
  T pL[8], pR[8];
  if constexpr (CellRecon<T, RECON>::value) {
    // extended box of this direction: one more cell on each side along dir
    const int ex_n = TX + 2 * ux, ey_n = TY + 2 * uy;
    const int eL = (dir == 0 ? 0 : (dir == 1 ? eoff_y : eoff_z)) + (fz * ey_n + fy) * ex_n + fx;
    const int eR = eL + (dir == 0 ? 1 : (dir == 1 ? ex_n : ex_n * ey_n));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      pL[q] = sR[(2 * q + 1) * ns + eL];
      pR[q] = sR[(2 * q) * ns + eR];
    }
  } else {
    reconstruct_face<T, RECON, S>(src, g.ncell, c, stride, par_t<T>(p.weno_eps, p.weno_epsf), pL, pR);
  }
  face_flux_states<T, CURVED, S, POLY>(g, p, src, c, dir, stride, pL, pR, F);
  cell = c;
  return true;
}

// Face flux of face f (flat index over the NFX x-, NFY y- and NFZ z-faces of
// the tile) into sF [8][NF].
template <class T, int RECON, bool CURVED, int TX, int TY, int TZ, class S, bool POLY = false>
__device__ __forceinline__ void tile_face(const DevGrid& g, const DevParams& p, const S& src, int x0, int y0, int z0,
                                          int f, T* __restrict__ sF, const T* __restrict__ sR, int ns, int eoff_y,
                                          int eoff_z) {
  constexpr int NFX = TileFaces<TX, TY, TZ>::NFX;
  constexpr int NFY = TileFaces<TX, TY, TZ>::NFY;
  constexpr int NF = TileFaces<TX, TY, TZ>::NF;
  // face coordinates in the tile (compile-time divisors per direction)
  int dir, fx, fy, fz;
  if (f < NFX) {
    dir = 0;
    fx = f % (TX + 1); fy = (f / (TX + 1)) % TY; fz = f / ((TX + 1) * TY);
  } else if (f < NFX + NFY) {
    const int fl = f - NFX;
    dir = 1;
    fx = fl % TX; fy = (fl / TX) % (TY + 1); fz = fl / (TX * (TY + 1));
  } else {
    const int fl = f - NFX - NFY;
    dir = 2;
    fx = fl % TX; fy = (fl / TX) % TY; fz = fl / (TX * TY);
  }
  T F[8];
  long long c;
  if (!tile_face_at<T, RECON, CURVED, TX, TY, TZ, S, POLY>(g, p, src, x0, y0, z0, dir, fx, fy, fz, sR, ns, eoff_y,
                                                           eoff_z, F, c))
    return;
#pragma unroll
  for (int q = 0; q < 8; ++q) sF[q * NF + f] = F[q];
}

// Stage item it of the directions [d0, d1]: cell e of the extended box of
// its direction, variable pair h; written at stage index eoff + e.
template <class T, int RECON, int TX, int TY, int TZ, class S>
__device__ __forceinline__ void tile_stage_item(const DevGrid& g, const S& src, int x0, int y0, int z0, int dir, int e,
                                                int h, int eoff, T eps13, T* __restrict__ sR, int ns, int which = 0) {
  const int ux = dir == 0, uy = dir == 1, uz = dir == 2;
  int ex, ey, ez;  // compile-time divisors per direction
  if (dir == 0) {
    ex = e % (TX + 2); ey = (e / (TX + 2)) % TY; ez = e / ((TX + 2) * TY);
  } else if (dir == 1) {
    ex = e % TX; ey = (e / TX) % (TY + 2); ez = e / (TX * (TY + 2));
  } else {
    ex = e % TX; ey = (e / TX) % TY; ez = e / (TX * TY);
  }
  const int xi = x0 + ex - ux, yi = y0 + ey - uy, zi = z0 + ez - uz;
  // cells -1 .. n along dir (ghosts have >= 3 layers), interior across
  if (xi < g.n[0] + ux && yi < g.n[1] + uy && zi < g.n[2] + uz) {
    const int ng = g.ng;
    const long long c = (long long)(zi + ng) * g.sz + (long long)(yi + ng) * g.sy + (xi + ng);
    const long long stride = (dir == 0) ? 1 : ((dir == 1) ? g.sy : g.sz);
    reconstruct_cell_pair<T, RECON, S>(src, g.ncell, c, stride, h, eps13, sR, ns, eoff + e, which);
  }
}

// Constrained transport: the transverse field components of the tile's face
// fluxes (B^a through a d-face, a != d) into fb [(3 d + a) * ncell + cell
// above the face], each face written by one tile only (its lower faces, and
// the upper faces on the block's upper boundaries).
template <class T, int TX, int TY, int TZ>
__device__ __noinline__ void tile_export_field_fluxes(const DevGrid& g, int x0, int y0, int z0,
                                                      const T* __restrict__ sF, double* __restrict__ fb) {
  constexpr int NFX = TileFaces<TX, TY, TZ>::NFX;
  constexpr int NFY = TileFaces<TX, TY, TZ>::NFY;
  constexpr int NF = TileFaces<TX, TY, TZ>::NF;
  for (int f = threadIdx.x; f < NF; f += kTileThreads) {
    int dir, fx, fy, fz;
    if (f < NFX) {
      dir = 0;
      fx = f % (TX + 1); fy = (f / (TX + 1)) % TY; fz = f / ((TX + 1) * TY);
    } else if (f < NFX + NFY) {
      const int fl = f - NFX;
      dir = 1;
      fx = fl % TX; fy = (fl / TX) % (TY + 1); fz = fl / (TX * (TY + 1));
    } else {
      const int fl = f - NFX - NFY;
      dir = 2;
      fx = fl % TX; fy = (fl / TX) % TY; fz = fl / (TX * TY);
    }
    const int xi = x0 + fx, yi = y0 + fy, zi = z0 + fz;
    const int ux = dir == 0, uy = dir == 1, uz = dir == 2;
    if (!(xi < g.n[0] + ux && yi < g.n[1] + uy && zi < g.n[2] + uz)) continue;
    // the tile's upper face along dir belongs to the next tile unless it is the block's
    const int fl = dir == 0 ? fx : (dir == 1 ? fy : fz);
    const int tl = dir == 0 ? TX : (dir == 1 ? TY : TZ);
    if (fl == tl && (dir == 0 ? xi : (dir == 1 ? yi : zi)) != g.n[dir]) continue;
    const long long c = (long long)(zi + g.ng) * g.sz + (long long)(yi + g.ng) * g.sy + (xi + g.ng);
    // F_d(B^d) is read by no edge field
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a != dir) fb[(3 * dir + a) * g.ncell + c] = (double)sF[(5 + a) * NF + f];
  }
}

// One tile of the RHS.  Every face flux of the tile is computed once into
// the face buffer sF [8][NF].  For FP64 WENO5 the reconstruction runs per
// cell first: every cell of the tile extended by one along a direction
// reconstructs both of its face states in that direction into the stage
// buffer sR [16][ns] (all three directions at once, or one at a time when
// the shared memory is short), and each face takes its left state (plus
// state of the cell below) and right state (minus state of the cell above)
// from there.  Then each thread differences its cell's six faces, adds the
// sources and applies the stage epilogue.  Called by all threads of the CTA
// (contains __syncthreads); kTileThreads threads, each handling one or more
// cells of the TX*TY*TZ tile.
template <class T, int RECON, bool CURVED, int TX, int TY, int TZ, class S, bool POLY = false>
__device__ __forceinline__ void rhs_tile(const DevGrid& g, const DevParams& p, const S& src, const StageEpilogue& ep,
                                         int x0, int y0, int z0, T* sF, T* sR) {
  constexpr int NT = kTileThreads;
  constexpr int NC = TX * TY * TZ;
  constexpr int NFX = TileFaces<TX, TY, TZ>::NFX;
  constexpr int NFY = TileFaces<TX, TY, TZ>::NFY;
  constexpr int NFZ = TileFaces<TX, TY, TZ>::NFZ;
  constexpr int NF = TileFaces<TX, TY, TZ>::NF;
  using ST = TileStage<TX, TY, TZ>;
  using SM = TileSmem<T, RECON, TX, TY, TZ>;
  const int ng = g.ng;
  if constexpr (!CellRecon<T, RECON>::value) {
    for (int f = threadIdx.x; f < NF; f += NT)
      tile_face<T, RECON, CURVED, TX, TY, TZ, S, POLY>(g, p, src, x0, y0, z0, f, sF, sR, 0, 0, 0);
    __syncthreads();
  } else if constexpr (SM::stage_all) {
    const T eps13 = par_t<T>(p.weno_eps * (12.0 / 13.0), p.eps13f);
    // (a) the tile's own cells, both states, per direction; (b) the two end
    // cells of every line of the extended box, one state each (the plus
    // state below the tile, the minus state above it).  The two groups are
    // separate ranges of the item index, so warps stay uniform.
    constexpr int NBX = 2 * TY * TZ, NBY = 2 * TX * TZ, NBZ = 2 * TX * TY;
    for (int it = threadIdx.x; it < 12 * NC + 4 * (NBX + NBY + NBZ); it += NT) {
      int dir, e, h, which = 0;
      if (it < 12 * NC) {
        dir = it / (4 * NC);
        const int r = it - dir * 4 * NC;
        h = r / NC;
        const int l = r - h * NC;
        const int cx = l % TX, cy = (l / TX) % TY, cz = l / (TX * TY);
        if (dir == 0) e = (cz * TY + cy) * (TX + 2) + cx + 1;
        else if (dir == 1) e = (cz * (TY + 2) + cy + 1) * TX + cx;
        else e = ((cz + 1) * TY + cy) * TX + cx;
      } else {
        int r = it - 12 * NC;
        const int nb = r < 4 * NBX ? NBX : (r < 4 * (NBX + NBY) ? NBY : NBZ);
        dir = r < 4 * NBX ? 0 : (r < 4 * (NBX + NBY) ? 1 : 2);
        r -= dir == 0 ? 0 : (dir == 1 ? 4 * NBX : 4 * (NBX + NBY));
        h = r / nb;
        const int b = r - h * nb;
        const int side = b / (nb / 2), t = b - side * (nb / 2);
        which = side ? 1 : 2;
        if (dir == 0) e = (t / TY * TY + t % TY) * (TX + 2) + (side ? TX + 1 : 0);
        else if (dir == 1) e = ((t / TX) * (TY + 2) + (side ? TY + 1 : 0)) * TX + t % TX;
        else e = ((side ? TZ + 1 : 0) * TY + t / TX) * TX + t % TX;
      }
      const int eoff = dir == 0 ? 0 : (dir == 1 ? ST::EXX : ST::EXX + ST::EYY);
      tile_stage_item<T, RECON, TX, TY, TZ, S>(g, src, x0, y0, z0, dir, e, h, eoff, eps13, sR, ST::NEA, which);
    }
    __syncthreads();
    for (int f = threadIdx.x; f < NF; f += NT)
      tile_face<T, RECON, CURVED, TX, TY, TZ, S, POLY>(g, p, src, x0, y0, z0, f, sF, sR, ST::NEA, ST::EXX,
                                                  ST::EXX + ST::EYY);
    __syncthreads();
  } else {
    const T eps13 = par_t<T>(p.weno_eps * (12.0 / 13.0), p.eps13f);
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int ne = dir == 0 ? ST::EXX : (dir == 1 ? ST::EYY : ST::EZZ);
      for (int it = threadIdx.x; it < 4 * ne; it += NT)
        tile_stage_item<T, RECON, TX, TY, TZ, S>(g, src, x0, y0, z0, dir, it % ne, it / ne, 0, eps13, sR, ST::NE);
      __syncthreads();
      const int f0 = dir == 0 ? 0 : (dir == 1 ? NFX : NFX + NFY);
      const int nfd = dir == 0 ? NFX : (dir == 1 ? NFY : NFZ);
      for (int f = threadIdx.x; f < nfd; f += NT)
        tile_face<T, RECON, CURVED, TX, TY, TZ, S, POLY>(g, p, src, x0, y0, z0, f0 + f, sF, sR, ST::NE, 0, 0);
      __syncthreads();
    }
  }

  if (ep.fb) tile_export_field_fluxes<T, TX, TY, TZ>(g, x0, y0, z0, sF, ep.fb);

#pragma unroll 1
  for (int cl = threadIdx.x; cl < NC; cl += NT) {
  const int ci = cl % TX, cj = (cl / TX) % TY, ck = cl / (TX * TY);
  const int xi = x0 + ci, yi = y0 + cj, zi = z0 + ck;
  if (xi < g.n[0] && yi < g.n[1] && zi < g.n[2]) {
    const long long c = (long long)(zi + ng) * g.sz + (long long)(yi + ng) * g.sy + (xi + ng);
    const int fx = (ck * TY + cj) * (TX + 1) + ci;
    const int fy = NFX + (ck * (TY + 1) + cj) * TX + ci;
    const int fz = NFX + NFY + (ck * TY + cj) * TX + ci;
    const T ix = par_t<T>(g.idx[0], g.idxf[0]), iy = par_t<T>(g.idx[1], g.idxf[1]), iz = par_t<T>(g.idx[2], g.idxf[2]);
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
      const double rq = to_f64(r[q]);
      if (ep.rhs) {
        if constexpr (sizeof(T) == 4) __stcg(ep.rhs + o, rq);
        else ep.rhs[o] = rq;
      }
      const double ain = ep.acc_in ? ep.acc_in[o] : 0.0;
      // FP64 (pipe bound): without an accumulator the ca term, an exact zero, is left out
      // (the same bits); the FP32 kernels keep the one expression, which measured faster there
      if constexpr (sizeof(T) == 8) {
        if (ep.u) ep.u[o] = ep.acc_in ? ep.c0 * ep.u0[o] + ep.c1 * ep.u[o] + ep.cr * rq + ep.ca * ain
                                      : ep.c0 * ep.u0[o] + ep.c1 * ep.u[o] + ep.cr * rq;
      } else {
        if (ep.u) __stcg(ep.u + o, ep.c0 * ld_once<true>(ep.u0 + o) + ep.c1 * ld_once<true>(ep.u + o) + ep.cr * rq + ep.ca * ain);
      }
      if (ep.acc_out) ep.acc_out[o] = ep.wa * ain + ep.wr * rq;
    }
  }
  }
}

// Resident CTAs per SM the register budget is fitted to: 3 for the FP32
// (mixed) kernels, which are latency bound, 1 for FP64 (pipe bound).
template <class T>
struct MinCtas { static constexpr int value = sizeof(T) == 4 ? 3 : 1; };

// ---------------------------------------------------------------------------
// Two-pass FP64 RHS.  FP64 issue is what bounds the RHS on this GPU, and HBM
// bandwidth is plentiful, so the FP64 path can spend bytes to save flops:
// pass 1 computes every face flux of the block exactly once into a face
// buffer Ff [(8 dir + q) * ncell + cell above the face] (192 B per cell
// written and read back), and pass 2 differences the buffer per cell, adds
// the sources and applies the stage epilogue, with the same operations in
// the same order as the single-pass cell loop.  The single-pass tile
// computes the faces on its upper boundaries too (896 face fluxes for 768
// faces in an 8x8x4 tile, in four rounds of 256 threads instead of three)
// and reconstructs one more end cell per line.

// Pass 1, one tile: the lower faces of its cells (3 per cell; the cell
// beyond the block's upper end along dir, when the tile is ragged there,
// gives the block's upper boundary face) and, when the tile ends exactly at
// the block's upper end along dir, that boundary face layer.  The stage
// skips the end cells above the tile except there.  fb (nullable): the
// transverse field fluxes for constrained transport, as the tile export
// writes them.
template <class T, int RECON, bool CURVED, int TX, int TY, int TZ, class S, bool POLY>
__device__ __forceinline__ void faces_tile(const DevGrid& g, const DevParams& p, const S& src, int x0, int y0, int z0,
                                           double* __restrict__ Ff, double* __restrict__ fb, T* sR) {
  constexpr int NT = kTileThreads;
  constexpr int NC = TX * TY * TZ;
  using ST = TileStage<TX, TY, TZ>;
  constexpr int NBX = TY * TZ, NBY = TX * TZ, NBZ = TX * TY;  // lines (boundary faces) per direction
  const bool top[3] = {x0 + TX == g.n[0], y0 + TY == g.n[1], z0 + TZ == g.n[2]};
  if constexpr (CellRecon<T, RECON>::value) {
    static_assert(TileSmem<T, RECON, TX, TY, TZ>::stage_all, "two-pass RHS needs the all-direction stage");
    const T eps13 = par_t<T>(p.weno_eps * (12.0 / 13.0), p.eps13f);
    // (a) the tile's own cells, both states; (b) the end cell below every
    // line, plus state; (c) the end cell above every line of the directions
    // in which the tile ends at the block's upper end, minus state
    const int nb_up = 4 * ((top[0] ? NBX : 0) + (top[1] ? NBY : 0) + (top[2] ? NBZ : 0));
    const int nitems = 12 * NC + 4 * (NBX + NBY + NBZ) + nb_up;
    for (int it = threadIdx.x; it < nitems; it += NT) {
      int dir, e, h, which = 0;
      if (it < 12 * NC) {
        dir = it / (4 * NC);
        const int r = it - dir * 4 * NC;
        h = r / NC;
        const int l = r - h * NC;
        const int cx = l % TX, cy = (l / TX) % TY, cz = l / (TX * TY);
        if (dir == 0) e = (cz * TY + cy) * (TX + 2) + cx + 1;
        else if (dir == 1) e = (cz * (TY + 2) + cy + 1) * TX + cx;
        else e = ((cz + 1) * TY + cy) * TX + cx;
      } else {
        int r = it - 12 * NC;
        int side = 0;
        if (r >= 4 * (NBX + NBY + NBZ)) {
          // upper end cells of the top directions, in x, y, z order
          side = 1;
          r -= 4 * (NBX + NBY + NBZ);
          if (!top[0]) r += 4 * NBX;
          if (!top[1] && r >= 4 * NBX) r += 4 * NBY;
        }
        const int nb = r < 4 * NBX ? NBX : (r < 4 * (NBX + NBY) ? NBY : NBZ);
        dir = r < 4 * NBX ? 0 : (r < 4 * (NBX + NBY) ? 1 : 2);
        r -= dir == 0 ? 0 : (dir == 1 ? 4 * NBX : 4 * (NBX + NBY));
        h = r / nb;
        const int t = r - h * nb;
        which = side ? 1 : 2;
        if (dir == 0) e = (t / TY * TY + t % TY) * (TX + 2) + (side ? TX + 1 : 0);
        else if (dir == 1) e = ((t / TX) * (TY + 2) + (side ? TY + 1 : 0)) * TX + t % TX;
        else e = ((side ? TZ + 1 : 0) * TY + t / TX) * TX + t % TX;
      }
      const int eoff = dir == 0 ? 0 : (dir == 1 ? ST::EXX : ST::EXX + ST::EYY);
      tile_stage_item<T, RECON, TX, TY, TZ, S>(g, src, x0, y0, z0, dir, e, h, eoff, eps13, sR, ST::NEA, which);
    }
    __syncthreads();
  }
  auto store = [&](int dir, int fx, int fy, int fz) {
    T F[8];
    long long c;
    if (!tile_face_at<T, RECON, CURVED, TX, TY, TZ, S, POLY>(g, p, src, x0, y0, z0, dir, fx, fy, fz, sR, ST::NEA,
                                                             ST::EXX, ST::EXX + ST::EYY, F, c))
      return;
#pragma unroll
    for (int q = 0; q < 8; ++q) Ff[(8 * dir + q) * g.ncell + c] = (double)F[q];
    if (fb) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a != dir) fb[(3 * dir + a) * g.ncell + c] = (double)F[5 + a];
    }
  };
  // the lower faces of the tile's cells: 3 NC faces, a whole number of rounds
  for (int f = threadIdx.x; f < 3 * NC; f += NT) {
    const int dir = f / NC, l = f - dir * NC;
    store(dir, l % TX, (l / TX) % TY, l / (TX * TY));
  }
  // the block's upper boundary faces where the tile ends exactly there
  if (top[0])
    for (int f = threadIdx.x; f < NBX; f += NT) store(0, TX, f % TY, f / TY);
  if (top[1])
    for (int f = threadIdx.x; f < NBY; f += NT) store(1, f % TX, TY, f / TX);
  if (top[2])
    for (int f = threadIdx.x; f < NBZ; f += NT) store(2, f % TX, f / TX, TZ);
}

template <class T, int RECON, bool CURVED, class S, bool POLY>
__global__ void __launch_bounds__(kTileThreads, MinCtas<T>::value) rhs_faces_kernel(DevGrid g, DevParams p, S src,
                                                                                    double* Ff, double* fb) {
  using TS = TileShape<0>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sR = reinterpret_cast<T*>(smem_raw);  // the stage only: no face buffer in shared memory
  faces_tile<T, RECON, CURVED, TS::X, TS::Y, TS::Z, S, POLY>(g, p, src, blockIdx.x * TS::X, blockIdx.y * TS::Y,
                                                             blockIdx.z * TS::Z, Ff, fb, sR);
}

// Pass 2 at interior cell c (array index): the flux differences, the
// sources and the stage epilogue (the single-pass cell loop's operations, in
// its order).
template <class T, bool CURVED, class S>
__device__ __forceinline__ void div_cell(const DevGrid& g, const DevParams& p, const S& src,
                                         const double* __restrict__ Ff, long long c, const StageEpilogue& ep) {
  const T ix = par_t<T>(g.idx[0], g.idxf[0]), iy = par_t<T>(g.idx[1], g.idxf[1]), iz = par_t<T>(g.idx[2], g.idxf[2]);
  T r[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double* fx = Ff + (0 * 8 + q) * g.ncell + c;
    const double* fy = Ff + (1 * 8 + q) * g.ncell + c;
    const double* fz = Ff + (2 * 8 + q) * g.ncell + c;
    T acc = -((T)__ldg(fx + 1) - (T)__ldg(fx)) * ix;
    acc -= ((T)__ldg(fy + g.sy) - (T)__ldg(fy)) * iy;
    acc -= ((T)__ldg(fz + g.sz) - (T)__ldg(fz)) * iz;
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
    const double rq = to_f64(r[q]);
    if (ep.rhs) ep.rhs[o] = rq;
    const double ain = ep.acc_in ? ep.acc_in[o] : 0.0;
    // without an accumulator the ca term (an exact zero) is left out: the same bits
    if (ep.u) ep.u[o] = ep.acc_in ? ep.c0 * ep.u0[o] + ep.c1 * ep.u[o] + ep.cr * rq + ep.ca * ain
                                  : ep.c0 * ep.u0[o] + ep.c1 * ep.u[o] + ep.cr * rq;
    if (ep.acc_out) ep.acc_out[o] = ep.wa * ain + ep.wr * rq;
  }
}

// Pass 2 over the interior cells of one block: 128-thread CTAs, registers
// fitted to 3 per SM (12 warps; the FP64 curved sources otherwise take 212
// registers and leave 8 warps per SM).
constexpr int kDivThreads = 128;
template <class T, bool CURVED, class S>
__global__ void __launch_bounds__(kDivThreads, 3) rhs_div_kernel(DevGrid g, DevParams p, S src, const double* __restrict__ Ff,
                                                      StageEpilogue ep) {
  const long long nx = g.n[0], ny = g.n[1], nint = nx * ny * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q0 = t / nx;
    const long long c = (q0 / ny + g.ng) * g.sz + (q0 % ny + g.ng) * g.sy + (t - q0 * nx + g.ng);
    div_cell<T, CURVED, S>(g, p, src, Ff, c, ep);
  }
}

// Constrained transport: the field fluxes of the faces outside the tiles,
// i.e. the d-faces (d-index 0 .. n_d) on the ring of ghost rows around the
// block (transverse (A, B) on the border of -1 .. n_a by -1 .. n_b, a = d + 1,
// b = d + 2 cyclic: the rows B = -1 and B = n_b, then the columns A = -1 and
// A = n_a), from the same inputs as the tiles, into fb as the tiles write it.
__host__ __device__ __forceinline__ long long ct_ring_faces(const DevGrid& g, int d) {
  const int na = g.n[(d + 1) % 3], nb = g.n[(d + 2) % 3];
  return (long long)(g.n[d] + 1) * (2LL * (na + 2) + 2LL * nb);
}

constexpr int kRingThreads = 128;

template <class T, int RECON, bool CURVED, class S, bool POLY = false>
__global__ void __launch_bounds__(kRingThreads) ct_ring_kernel(DevGrid g, DevParams p, S src,
                                                               double* __restrict__ fb) {
  const long long r0 = ct_ring_faces(g, 0), r1 = ct_ring_faces(g, 1), total = r0 + r1 + ct_ring_faces(g, 2);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int d = t < r0 ? 0 : (t < r0 + r1 ? 1 : 2);
    const long long r = t - (d == 0 ? 0 : (d == 1 ? r0 : r0 + r1));
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    const int na = g.n[a], nb = g.n[b];
    const long long per = 2LL * (na + 2) + 2LL * nb;
    const int id = (int)(r / per);
    const int m = (int)(r - id * per);
    int A, B;
    if (m < na + 2) {
      A = m - 1; B = -1;
    } else if (m < 2 * (na + 2)) {
      A = m - (na + 2) - 1; B = nb;
    } else if (m < 2 * (na + 2) + nb) {
      A = -1; B = m - 2 * (na + 2);
    } else {
      A = na; B = m - 2 * (na + 2) - nb;
    }
    int I[3];
    I[d] = id; I[a] = A; I[b] = B;
    const long long c = (long long)(I[2] + g.ng) * g.sz + (long long)(I[1] + g.ng) * g.sy + (I[0] + g.ng);
    const long long stride = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
    T pL[8], pR[8], F[8];
    reconstruct_face<T, RECON, S>(src, g.ncell, c, stride, par_t<T>(p.weno_eps, p.weno_epsf), pL, pR);
    face_flux_states<T, CURVED, S, POLY>(g, p, src, c, d, stride, pL, pR, F);
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q != d) fb[(3 * d + q) * g.ncell + c] = (double)F[5 + q];
  }
}

template <class T, int RECON, bool CURVED, int SHAPE, class S, bool POLY = false>
__global__ void __launch_bounds__(kTileThreads, MinCtas<T>::value) rhs_kernel(DevGrid g, DevParams p, S src,
                                                                             StageEpilogue ep) {
  using TS = TileShape<SHAPE>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sR = sF + 8 * TileFaces<TS::X, TS::Y, TS::Z>::NF;  // stage (FP64 WENO5 only)
  rhs_tile<T, RECON, CURVED, TS::X, TS::Y, TS::Z, S, POLY>(g, p, src, ep, blockIdx.x * TS::X, blockIdx.y * TS::Y,
                                                      blockIdx.z * TS::Z, sF, sR);
}

// ---------------------------------------------------------------------------
// Three-pass FP64 WENO5 RHS (the cached paths, with a state buffer in
// ep.states).  The tile stage of the faces kernel reconstructs, besides its
// own cells, the end cell below every line of the tile (about 8% of the
// kernel's FP64 work); without tiles no cell is reconstructed twice:
//   pass 1, rhs_states_kernel: per direction d, both face states of every
//     cell on the lines of cells -1 .. n_d along d (interior across), into
//     St [(16 d + 2 q + s) ncell + cell], s = 0 for the value at the cell's
//     lower face (minus), 1 at its upper face (plus);
//   pass 2, rhs_face_kernel: the flux of every d-face 0 .. n_d from the
//     plus state of the cell below and the minus state of the cell above,
//     into the face buffer (and the field fluxes for constrained transport)
//     as faces_tile writes them;
//   pass 3, rhs_div_kernel.
// The operations and their inputs are those of the tiles, so the results
// have the same bits.  The buffer costs 768 B of traffic per cell (written
// once, read once), against an FP64-pipe-bound pass.
constexpr int kStatesThreads = 256, kFaceThreads = 128;

// State units of direction d: the cells -1 .. n_d of each line along d in
// pairs ((n_d + 3) / 2 pairs, the last one a single cell when n_d is odd),
// interior across.
__host__ __device__ __forceinline__ long long state_units(const DevGrid& g, int d) {
  return (long long)(d == 0 ? (g.n[0] + 3) / 2 : g.n[0]) * (d == 1 ? (g.n[1] + 3) / 2 : g.n[1]) *
         (d == 2 ? (g.n[2] + 3) / 2 : g.n[2]);
}
// Faces of direction d: n_d + 1 along d, interior across.
__host__ __device__ __forceinline__ long long face_count(const DevGrid& g, int d) {
  return (long long)(g.n[0] + (d == 0)) * (g.n[1] + (d == 1)) * (g.n[2] + (d == 2));
}

// State items of a block: direction, then variable pair, then the cell
// pairs of the direction's lines (x fastest).
__host__ __device__ __forceinline__ long long state_items(const DevGrid& g) {
  return 4 * (state_units(g, 0) + state_units(g, 1) + state_units(g, 2));
}
__host__ __device__ __forceinline__ long long face_items(const DevGrid& g) {
  return face_count(g, 0) + face_count(g, 1) + face_count(g, 2);
}

// The four states of weno5_cell_pair_states from the parts of its two
// variables (one shared division).
__device__ __forceinline__ void weno5_pair_states_from_parts(const double u0[2], const double nm[2],
                                                             const double dm[2], const double np[2],
                                                             const double dp[2], double v[4]) {
  const double a0 = __dmul_rn(dm[0], dp[0]), a1 = __dmul_rn(dm[1], dp[1]);
  const double X = 1.0 / __dmul_rn(__dmul_rn(6.0, a0), a1);
  const double x0 = __dmul_rn(a1, X), x1 = __dmul_rn(a0, X);
  v[0] = weno5_cell_state(u0[0], nm[0], __dmul_rn(dp[0], x0));
  v[1] = weno5_cell_state(u0[0], np[0], __dmul_rn(dm[0], x0));
  v[2] = weno5_cell_state(u0[1], nm[1], __dmul_rn(dp[1], x1));
  v[3] = weno5_cell_state(u0[1], np[1], __dmul_rn(dm[1], x1));
}

// FP64 WENO5 of the two neighbouring cells c and c + stride of a line (the
// second one only if two): both states of each for the primitives 2h and
// 2h+1 into v0 and v1, as weno5_cell_pair_states forms them (the same bits),
// from the six values of each variable that the two stencils cover.
template <class S>
__device__ __forceinline__ void weno5_two_cell_pair_states(const S& src, long long ncell, long long c,
                                                           long long stride, int h, double eps13, bool two,
                                                           double v0[4], double v1[4]) {
  // parts of cell 0 (A) and cell 1 (B) for the two variables
  double nmA[2], dmA[2], npA[2], dpA[2], uA[2], nmB[2], dmB[2], npB[2], dpB[2], uB[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const long long a = (2 * h + k) * ncell + c;
    double u[6];
    u[0] = ld_prim<double>(src, a - 2 * stride);
    u[1] = ld_prim<double>(src, a - stride);
    u[2] = ld_prim<double>(src, a);
    u[3] = ld_prim<double>(src, a + stride);
    u[4] = ld_prim<double>(src, a + 2 * stride);
    u[5] = two ? ld_prim<double>(src, a + 3 * stride) : u[4];
    weno5_two_cell_parts(u, eps13, two, nmA[k], dmA[k], npA[k], dpA[k], nmB[k], dmB[k], npB[k], dpB[k]);
    uA[k] = u[2];
    uB[k] = u[3];
  }
  weno5_pair_states_from_parts(uA, nmA, dmA, npA, dpA, v0);
  if (two) weno5_pair_states_from_parts(uB, nmB, dmB, npB, dpB, v1);
}

// State item t (0 <= t < state_items(g)) of pass 1: one cell pair of a line
// along d, one variable pair.  The two cells share four of their six stencil
// values (and three first and two second differences of them).
template <class S>
__device__ __forceinline__ void rhs_state_item(const DevGrid& g, const DevParams& p, const S& src,
                                               double* __restrict__ St, long long t) {
  const long long m0 = state_units(g, 0), m1 = state_units(g, 1), m2 = state_units(g, 2);
  int d = 0;
  long long r = t;
  if (r >= 4 * m0) {
    r -= 4 * m0;
    d = 1;
    if (r >= 4 * m1) {
      r -= 4 * m1;
      d = 2;
    }
  }
  const long long m = d == 0 ? m0 : (d == 1 ? m1 : m2);
  const int h = (int)(r / m);
  const long long l = r - h * m;
  const int ex = d == 0 ? (g.n[0] + 3) / 2 : g.n[0], ey = d == 1 ? (g.n[1] + 3) / 2 : g.n[1];
  const long long lxy = l / ex;
  int i = (int)(l - lxy * ex), j = (int)(lxy % ey), k = (int)(lxy / ey);
  // the first cell of the pair along d: -1, 1, 3, ...
  if (d == 0) i = 2 * i - 1;
  else if (d == 1) j = 2 * j - 1;
  else k = 2 * k - 1;
  const bool two = (d == 0 ? i : (d == 1 ? j : k)) + 1 <= g.n[d];
  const long long c = (long long)(k + g.ng) * g.sz + (long long)(j + g.ng) * g.sy + (i + g.ng);
  const long long stride = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
  double v0[4], v1[4];
  weno5_two_cell_pair_states<S>(src, g.ncell, c, stride, h, p.weno_eps * (12.0 / 13.0), two, v0, v1);
  double* o = St + (16LL * d + 4 * h) * g.ncell + c;
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q * g.ncell] = v0[q];
  if (two) {
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q * g.ncell + stride] = v1[q];
  }
}

// Face item t (0 <= t < face_items(g)) of pass 2.
template <bool CURVED, class S, bool POLY>
__device__ __forceinline__ void rhs_face_item(const DevGrid& g, const DevParams& p, const S& src,
                                              const double* __restrict__ St, double* __restrict__ Ff,
                                              double* __restrict__ fb, long long t) {
  const long long f0 = face_count(g, 0), f1 = face_count(g, 1);
  const int d = t < f0 ? 0 : (t < f0 + f1 ? 1 : 2);
  const long long l = t - (d == 0 ? 0 : (d == 1 ? f0 : f0 + f1));
  const int ex = g.n[0] + (d == 0), ey = g.n[1] + (d == 1);
  const long long lxy = l / ex;
  const int i = (int)(l - lxy * ex), j = (int)(lxy % ey), k = (int)(lxy / ey);
  // c: the cell above the face
  const long long c = (long long)(k + g.ng) * g.sz + (long long)(j + g.ng) * g.sy + (i + g.ng);
  const long long stride = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
  const double* Sd = St + 16LL * d * g.ncell;
  double pL[8], pR[8], F[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    pL[q] = __ldg(Sd + (2 * q + 1) * g.ncell + c - stride);
    pR[q] = __ldg(Sd + (2 * q) * g.ncell + c);
  }
  face_flux_states<double, CURVED, S, POLY>(g, p, src, c, d, stride, pL, pR, F);
#pragma unroll
  for (int q = 0; q < 8; ++q) Ff[(8 * d + q) * g.ncell + c] = F[q];
  if (fb) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a != d) fb[(3 * d + a) * g.ncell + c] = F[5 + a];
  }
}

template <class S>
__global__ void __launch_bounds__(kStatesThreads) rhs_states_kernel(DevGrid g, DevParams p, S src,
                                                                    double* __restrict__ St) {
  const long long total = state_items(g);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    rhs_state_item<S>(g, p, src, St, t);
}

template <bool CURVED, class S, bool POLY>
__global__ void __launch_bounds__(kFaceThreads) rhs_face_kernel(DevGrid g, DevParams p, S src,
                                                                const double* __restrict__ St,
                                                                double* __restrict__ Ff, double* __restrict__ fb) {
  const long long total = face_items(g);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    rhs_face_item<CURVED, S, POLY>(g, p, src, St, Ff, fb, t);
}

// Multi-pass launch (FP64 with the geometry cache and a face buffer in
// ep.faces): the face fluxes (for WENO5 with a state buffer in ep.states the
// state and face kernels, otherwise the 8x8x4 tile kernel), the
// constrained-transport ring if asked for, then the per-cell pass.
template <class T, int RECON, bool CURVED, class S>
cudaError_t launch_rhs_two_pass(const DevGrid& g, const DevParams& p, const S& src, const StageEpilogue& ep,
                                cudaStream_t s) {
  using TS = TileShape<0>;
  const bool poly = p.eos == GRMHD_EOS_POLYTROPE;
  if (CellRecon<T, RECON>::value && ep.states) {
    // three passes: states, faces (then the ring and the per-cell pass below)
    const long long ns = state_items(g);
    long long bs = (ns + kStatesThreads - 1) / kStatesThreads;
    if (bs > 152LL * 32) bs = 152LL * 32;
    rhs_states_kernel<S><<<(int)bs, kStatesThreads, 0, s>>>(g, p, src, ep.states);
    const long long nf = face_items(g);
    long long bf = (nf + kFaceThreads - 1) / kFaceThreads;
    if (bf > 152LL * 32) bf = 152LL * 32;
    if (poly)
      rhs_face_kernel<CURVED, S, true><<<(int)bf, kFaceThreads, 0, s>>>(g, p, src, ep.states, ep.faces, ep.fb);
    else
      rhs_face_kernel<CURVED, S, false><<<(int)bf, kFaceThreads, 0, s>>>(g, p, src, ep.states, ep.faces, ep.fb);
  } else {
    void (*k)(DevGrid, DevParams, S, double*, double*) =
        poly ? rhs_faces_kernel<T, RECON, CURVED, S, true> : rhs_faces_kernel<T, RECON, CURVED, S, false>;
    const size_t smem =
        CellRecon<T, RECON>::value ? (size_t)16 * TileStage<TS::X, TS::Y, TS::Z>::NEA * sizeof(T) : (size_t)0;
    if (smem) {
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const dim3 grid((g.n[0] + TS::X - 1) / TS::X, (g.n[1] + TS::Y - 1) / TS::Y, (g.n[2] + TS::Z - 1) / TS::Z);
    k<<<grid, kTileThreads, smem, s>>>(g, p, src, ep.faces, ep.fb);
  }
  if (ep.fb) {
    const long long nring = ct_ring_faces(g, 0) + ct_ring_faces(g, 1) + ct_ring_faces(g, 2);
    long long blocks = (nring + kRingThreads - 1) / kRingThreads;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    if (poly)
      ct_ring_kernel<T, RECON, CURVED, S, true><<<(int)blocks, kRingThreads, 0, s>>>(g, p, src, ep.fb);
    else
      ct_ring_kernel<T, RECON, CURVED, S><<<(int)blocks, kRingThreads, 0, s>>>(g, p, src, ep.fb);
  }
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  long long blocks = (nint + kDivThreads - 1) / kDivThreads;
  if (blocks > 152LL * 24) blocks = 152LL * 24;
  rhs_div_kernel<T, CURVED, S><<<(int)blocks, kDivThreads, 0, s>>>(g, p, src, ep.faces, ep);
  return cudaGetLastError();
}

template <class T, int RECON, bool CURVED, class S>
cudaError_t launch_rhs_shape(int shape, const DevGrid& g, const DevParams& p, const S& src, const StageEpilogue& ep,
                             cudaStream_t s) {
  if constexpr (sizeof(T) == 8 && std::is_same<S, SrcCache64>::value) {
    if (ep.faces) return launch_rhs_two_pass<T, RECON, CURVED, S>(g, p, src, ep, s);
  }
  void (*k)(DevGrid, DevParams, S, StageEpilogue) = nullptr;
  int tx, ty, tz;
  size_t smem;
  const bool poly = p.eos == GRMHD_EOS_POLYTROPE;
  // the polytrope runs on the default tile shape only
  if (poly) shape = -1;
  switch (shape) {
#define GRMHD_SHAPE_CASE(SH)                                                          \
  case SH:                                                                            \
    k = rhs_kernel<T, RECON, CURVED, SH, S>;                                          \
    tx = TileShape<SH>::X; ty = TileShape<SH>::Y; tz = TileShape<SH>::Z;              \
    smem = tile_smem_bytes<T, RECON, TileShape<SH>::X, TileShape<SH>::Y, TileShape<SH>::Z>(); \
    break;
    GRMHD_SHAPE_CASE(1)
    GRMHD_SHAPE_CASE(2)
    GRMHD_SHAPE_CASE(3)
    GRMHD_SHAPE_CASE(4)
    case -1:
      k = rhs_kernel<T, RECON, CURVED, 0, S, true>;
      tx = TileShape<0>::X; ty = TileShape<0>::Y; tz = TileShape<0>::Z;
      smem = tile_smem_bytes<T, RECON, TileShape<0>::X, TileShape<0>::Y, TileShape<0>::Z>();
      break;
    default:
    GRMHD_SHAPE_CASE(0)
#undef GRMHD_SHAPE_CASE
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((g.n[0] + tx - 1) / tx, (g.n[1] + ty - 1) / ty, (g.n[2] + tz - 1) / tz);
  k<<<grid, kTileThreads, smem, s>>>(g, p, src, ep);
  if (ep.fb) {
    // the rest of the field-flux register: the ring faces
    const long long nring = ct_ring_faces(g, 0) + ct_ring_faces(g, 1) + ct_ring_faces(g, 2);
    long long blocks = (nring + kRingThreads - 1) / kRingThreads;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    if (poly)
      ct_ring_kernel<T, RECON, CURVED, S, true><<<(int)blocks, kRingThreads, 0, s>>>(g, p, src, ep.fb);
    else
      ct_ring_kernel<T, RECON, CURVED, S><<<(int)blocks, kRingThreads, 0, s>>>(g, p, src, ep.fb);
  }
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
