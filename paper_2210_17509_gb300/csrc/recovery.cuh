// Per-cell primitive recovery and ghost fill as device functions, shared by
// the single-block kernels and the persistent batched kernels.
#pragma once

#include "fpbits.cuh"
#include "physics.cuh"

namespace grmhd {

// Spatial metric of a cell: gamma_ij packed (xx, xy, xz, yy, yz, zz), its
// inverse and sqrt(det), all FP64.  Minkowski when metric == NULL.
struct CellMetric {
  double g[6], gu[6], sqrtg;
};

__device__ __forceinline__ void cell_metric(const double* __restrict__ metric, long long ncell, long long c,
                                            CellMetric& m) {
  if (!metric) {
    m.g[0] = m.g[3] = m.g[5] = 1.0;
    m.g[1] = m.g[2] = m.g[4] = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) m.gu[i] = m.g[i];
    m.sqrtg = 1.0;
    return;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = __ldg(metric + (4 + i) * ncell + c);
  const double gxx = m.g[0], gxy = m.g[1], gxz = m.g[2], gyy = m.g[3], gyz = m.g[4], gzz = m.g[5];
  const double cxx = gyy * gzz - gyz * gyz, cxy = gxz * gyz - gxy * gzz, cxz = gxy * gyz - gxz * gyy;
  const double cyy = gxx * gzz - gxz * gxz, cyz = gxy * gxz - gxx * gyz, czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx + gxy * cxy + gxz * cxz;
  const double idet = 1.0 / det;
  m.gu[0] = cxx * idet; m.gu[1] = cxy * idet; m.gu[2] = cxz * idet;
  m.gu[3] = cyy * idet; m.gu[4] = cyz * idet; m.gu[5] = czz * idet;
  m.sqrtg = sqrt(det);
}

// Undensitised inputs of the recovery of one cell (Sec. 2.3): the momentum
// equation S_i = (z + B^2) v_i - (B.v) B_i with B.v = (B.S)/z reduces the
// unknowns to z = rho h W^2 and W.
struct C2PIn {
  double D, tau, S2, B2, BS2;
};

// Energy residual at (z, W) and the S^2 residual, Gamma-law pressure
// P = (Gamma - 1)/Gamma (z / W^2 - D / W).
__device__ __forceinline__ double c2p_v2_of_z(const C2PIn& in, double z) {
  const double zb = z + in.B2;
  const double iz = 1.0 / z;
  return (in.S2 + in.BS2 * (2.0 * z + in.B2) * iz * iz) / (zb * zb);
}

__device__ __forceinline__ double c2p_energy_of_z(const C2PIn& in, double z, double v2, double gm1g) {
  const double iw2 = 1.0 - v2;
  const double iw = sqrt(iw2);
  const double P = gm1g * (z * iw2 - in.D * iw);
  return in.tau + in.D - z - in.B2 + 0.5 * in.B2 * iw2 + 0.5 * in.BS2 / (z * z) + P;
}

// Bracketed bisection of the energy residual in z, with W(z) from the S^2
// equation; z below the v = 1 boundary counts as "too small".  A root needs
// a sign change of the residual inside v < 1: if the lower end of the final
// bracket is "too small" only through v >= 1, the bracket has closed on the
// v = 1 boundary and there is no root (which side of v = 1 the midpoint
// lands on is round-off).  Returns 1 (root found) or 2 (no root); z, W on
// exit.
static __device__ int c2p_bisect(const C2PIn& in, const DevParams& p, double& z, double& W) {
  const double gm1g = p.gm1g;
  double zlo = 0.0, zhi = 2.0 * (in.tau + in.D) / gm1g + in.B2 + 1e-300;
  // 0: residual <= 0 inside v < 1; 1: residual > 0 inside v < 1; 2: v >= 1
  auto sign_class = [&](double zz) {
    const double v2 = c2p_v2_of_z(in, zz);
    if (!(v2 < 1.0)) return 2;
    return c2p_energy_of_z(in, zz, v2, gm1g) > 0.0 ? 1 : 0;
  };
  bool lo_energy = false;
  int k = 0;
  for (int c = sign_class(zhi); c != 0 && k < 200; c = sign_class(zhi)) {
    zlo = zhi;
    lo_energy = c == 1;
    zhi *= 2.0;
    ++k;
  }
  if (k >= 200 || !isfinite(zhi)) return 2;
  for (int it = 0; it < 400 && zhi - zlo > 1e-15 * zhi; ++it) {
    const double zm = 0.5 * (zlo + zhi);
    const int c = sign_class(zm);
    if (c != 0) {
      zlo = zm;
      lo_energy = c == 1;
    } else {
      zhi = zm;
    }
  }
  if (!lo_energy) return 2;
  z = 0.5 * (zlo + zhi);
  const double v2 = c2p_v2_of_z(in, z);
  if (!(v2 < 1.0)) return 2;
  W = 1.0 / sqrt(1.0 - v2);
  return 1;
}

// A Newton root is accepted only if it is physical: W >= 1, rho = D / W >=
// rho_atm and P = (Gamma - 1)/Gamma (z / W^2 - D / W) > 0, i.e. z > D W.
// Otherwise (the iteration can settle on a spurious root from a poor guess,
// e.g. next to an atmosphere cell) the bracketed bisection decides.
__device__ __forceinline__ bool c2p_root_physical(const C2PIn& in, const DevParams& p, double z, double W) {
  // (the comparisons on the integer pipe, fpbits.cuh; D W and rho_atm W are >= 0)
  return dge1i(W) && dfinitei(W) && dgtci(z, in.D * W) && dgeci(in.D, p.rho_atm * W);
}

// Newman-Hamlin iteration over the pressure (Sec. 2.3, the paper's fallback
// "Newman's method"): with E = tau + D, a = E + P + B^2/2 and
// d = (B^2 S^2 - (B.S)^2)/2, the energy and momentum equations give
// f(eps) = eps^3 - a eps^2 + d = 0 for eps = B^2 + z, whose physical root is
// the largest.  f(a) = d >= 0 and f is increasing and convex above 2a/3, so
// Newton's iteration on f from eps = a descends monotonically onto it (no
// trigonometric closed form needed); then v^2(z) from the momentum equation
// and the Gamma-law pressure of (z, W) give the next P.  The fixed point is
// accelerated by Aitken's delta-squared extrapolation every third iterate.
// Returns true with (z, W) when the pressure changes by at most nr_tol
// (relative) within 3 * nr_maxit steps.
static __device__ bool c2p_newman_hamlin(const C2PIn& in, const DevParams& p, double P, double& z, double& W) {
  const double E = in.tau + in.D;
  const double d = fmax(0.5 * (in.B2 * in.S2 - in.BS2), 0.0);  // >= 0 (Cauchy-Schwarz) up to round-off
  double Pm1 = 0.0;
  const int maxit = 3 * p.nr_maxit;
  for (int it = 0; it < maxit; ++it) {
    const double a = E + P + 0.5 * in.B2;
    if (!(a > 0.0) || !(27.0 * d <= 4.0 * a * a * a)) return false;  // no root above 2a/3
    double eps = a;
    for (int k = 0; k < 60; ++k) {
      const double fe = eps * eps * (eps - a) + d;
      const double de = eps * fma(3.0, eps, -2.0 * a);
      const double step = fe / de;
      eps -= step;
      if (!(fabs(step) > 1e-16 * eps)) break;
    }
    const double zz = eps - in.B2;
    if (!(zz > 0.0)) return false;
    const double v2 = c2p_v2_of_z(in, zz);
    if (!(v2 < 1.0)) return false;
    const double iw = sqrt(1.0 - v2);
    double Pn = p.gm1g * (zz * (1.0 - v2) - in.D * iw);
    if (fabs(Pn - P) <= p.nr_tol * fabs(Pn)) {
      z = zz;
      W = 1.0 / iw;
      return isfinite(z) && isfinite(W);
    }
    // Aitken extrapolation from the last three iterates (P_{k-1}, P_k, P_{k+1})
    if (it % 3 == 2) {
      const double den = Pn - 2.0 * P + Pm1;
      const double Pa = Pn - (Pn - P) * (Pn - P) / den;
      if (den != 0.0 && Pa > 0.0 && isfinite(Pa)) Pn = Pa;
    }
    Pm1 = P;
    P = Pn;
  }
  return false;
}

// Returns 0 (Newton converged), 1 (bisection), 2 (failed); z, W on exit.
// The Newton steps must fall below nr_tol (relative).  P0 (> 0) starts the
// Newman-Hamlin iteration, which follows a failed Newton iteration or, with
// GRMHD_NEWMAN_HAMLIN, replaces it; status 0 covers both.
static __device__ int c2p_solve(const C2PIn& in, const DevParams& p, double& z, double& W, double P0) {
  const double gm1g = p.gm1g;
  const double D = in.D, B2 = in.B2, BS2 = in.BS2, S2 = in.S2, tau = in.tau;
  bool ok = false;
  const bool newman_first = (p.flags & GRMHD_NEWMAN_HAMLIN) != 0;
  // (the comparisons on the integer pipe, fpbits.cuh)
  if (!newman_first && dgt0i(z) && dge1i(W) && dfinitei(z) && dfinitei(W)) {
    for (int it = 0; it < p.nr_maxit; ++it) {
      const double izW = 1.0 / (z * W);  // 1/z and 1/W from one division
      const double iz = W * izW, iW = z * izW;
      const double iW2 = iW * iW, iW3 = iW2 * iW, iz2 = iz * iz, iz3 = iz2 * iz;
      const double zb = z + B2;
      const double f1 = zb * zb * (1.0 - iW2) - S2 - BS2 * (2.0 * z + B2) * iz2;
      const double f2 = tau + D - z - B2 + 0.5 * B2 * iW2 + 0.5 * BS2 * iz2 + gm1g * (z * iW2 - D * iW);
      const double J11 = 2.0 * zb * (1.0 - iW2) + 2.0 * BS2 * zb * iz3;
      const double J12 = 2.0 * zb * zb * iW3;
      const double J21 = -1.0 - BS2 * iz3 + gm1g * iW2;
      const double J22 = -B2 * iW3 + gm1g * (D * iW2 - 2.0 * z * iW3);
      const double idet = 1.0 / (J11 * J22 - J12 * J21);
      const double dz = (f1 * J22 - f2 * J12) * idet;
      const double dW = (J11 * f2 - J21 * f1) * idet;
      if (!dfinitei(dz) || !dfinitei(dW)) break;
      const bool conv = dabsleci(dz, p.nr_tol * z) && dabsleci(dW, p.nr_tol * W);  // z > 0, W >= 1
      double zn = z - dz, Wn = W - dW;
      if (!dgt0i(zn)) zn = 0.5 * z;
      if (!dge1i(Wn)) Wn = 0.5 * (W + 1.0);
      z = zn;
      W = Wn;
      if (conv) { ok = true; break; }
    }
  }
  if (ok && c2p_root_physical(in, p, z, W)) return 0;
  if (c2p_newman_hamlin(in, p, P0, z, W) && c2p_root_physical(in, p, z, W)) return 0;
  return c2p_bisect(in, p, z, W);
}

// FP32 Newton starting point of the FP64 recovery: iterates the same 2D
// system in single precision to a relative step of 1e-6 and returns the
// improved (z, W) (unchanged if it fails); the FP64 Newton of c2p_solve then
// finishes to nr_tol, normally in one or two steps.
__device__ __forceinline__ bool c2p_predict_fp32(const C2PIn& in, const DevParams& p, double& z, double& W) {
  const float gm1g = p.gm1gf;
  // conversions on the integer pipe (fpbits.cuh; the bits of the hardware conversions)
  const float D = f64_to_f32i(in.D), B2 = f64_to_f32i(in.B2), BS2 = f64_to_f32i(in.BS2), S2 = f64_to_f32i(in.S2),
              tau = f64_to_f32i(in.tau);
  float zf = f64_to_f32i(z), Wf = f64_to_f32i(W);
  if (!(zf > 0.0f) || !(Wf >= 1.0f)) return false;
  bool converged = false;
  for (int it = 0; it < 30; ++it) {
    const float iz = 1.0f / zf, iW = 1.0f / Wf;
    const float iW2 = iW * iW, iW3 = iW2 * iW, iz2 = iz * iz, iz3 = iz2 * iz;
    const float zb = zf + B2;
    const float f1 = zb * zb * (1.0f - iW2) - S2 - BS2 * (2.0f * zf + B2) * iz2;
    const float f2 = tau + D - zf - B2 + 0.5f * B2 * iW2 + 0.5f * BS2 * iz2 + gm1g * (zf * iW2 - D * iW);
    const float J11 = 2.0f * zb * (1.0f - iW2) + 2.0f * BS2 * zb * iz3;
    const float J12 = 2.0f * zb * zb * iW3;
    const float J21 = -1.0f - BS2 * iz3 + gm1g * iW2;
    const float J22 = -B2 * iW3 + gm1g * (D * iW2 - 2.0f * zf * iW3);
    const float idet = 1.0f / (J11 * J22 - J12 * J21);
    const float dz = (f1 * J22 - f2 * J12) * idet;
    const float dW = (J11 * f2 - J21 * f1) * idet;
    if (!isfinite(dz) || !isfinite(dW)) return false;
    float zn = zf - dz, Wn = Wf - dW;
    if (!(zn > 0.0f)) zn = 0.5f * zf;
    if (!(Wn >= 1.0f)) Wn = 0.5f * (Wf + 1.0f);
    const bool conv = fabsf(dz) <= 1e-6f * zf && fabsf(dW) <= 1e-6f * Wf;
    zf = zn;
    Wf = Wn;
    if (conv) { converged = true; break; }
  }
  if (zf > 0.0f && Wf >= 1.0f && isfinite(zf) && isfinite(Wf)) {
    z = f32_to_f64i(zf);
    W = f32_to_f64i(Wf);
    return converged;
  }
  return false;
}

// Mixed-path recovery of the Gamma-law system (Sec. 2.3), from the FP32
// guess (zf, Wf).
//
// (1) FP32 Newton predictor on the same 2D system, to a relative step of
// 1e-6.  The loop is warp-uniform: a vote keeps every lane of the warp
// iterating until all have converged (a converged lane holds its values), so
// the FP64 code that follows runs once per warp with all lanes rather than
// once per exit iteration.  1/z and 1/W come from one fast reciprocal; the
// predictor's accuracy does not depend on them, only its convergence rate.
//
// (2) One step of mixed-precision iterative refinement (Wilkinson): the
// residual of the 2D system at the predicted (z, W) in FP64 and the
// correction from the FP32 Jacobian at that point.  Both equations
// multiplied by W^2 z^2 need no division in FP64; the factor is divided out
// in FP32, where only the correction's relative accuracy matters.  The
// Jacobian's v^2 = (W^2 - 1)/W^2 comes from the FP64 W^2 - 1 (exact: W is an
// FP32 value), so slow flows lose no digits to the cancellation in 1 - 1/W^2
// and the Jacobian carries only FP32 rounding.  The error after the step is
// the predictor's times that rounding plus its square, i.e. of order 1e-13
// relative, as after a full FP64 Newton step.  A correction above 1e-6
// (relative), a failed predictor or an unphysical root hands the solve to
// the FP64 Newton of c2p_solve, from the best point.  Pg: the guess's
// pressure, which starts the Newman-Hamlin fallback.
__device__ __forceinline__ int c2p_solve_mixed(const C2PIn& in, const DevParams& p, float zf, float Wf, float Pg,
                                               double& z, double& W) {
  const float gm1g = p.gm1gf;
  // conversions between the FP32 and FP64 parts on the integer pipe (fpbits.cuh)
  const float D = f64_to_f32i(in.D), B2 = f64_to_f32i(in.B2), BS2 = f64_to_f32i(in.BS2), S2 = f64_to_f32i(in.S2),
              tau = f64_to_f32i(in.tau);
  bool active = zf > 0.0f && Wf >= 1.0f && isfinite(zf) && isfinite(Wf);
  bool converged = false;
  const unsigned mask = __activemask();
  for (int it = 0; it < 30 && __any_sync(mask, active); ++it) {
    if (active) {
      const float r = __fdividef(1.0f, zf * Wf);
      const float iz = Wf * r, iW = zf * r;
      const float iW2 = iW * iW, iW3 = iW2 * iW, iz2 = iz * iz, iz3 = iz2 * iz;
      const float zb = zf + B2;
      const float f1 = zb * zb * (1.0f - iW2) - S2 - BS2 * (2.0f * zf + B2) * iz2;
      const float f2 = tau + D - zf - B2 + 0.5f * B2 * iW2 + 0.5f * BS2 * iz2 + gm1g * (zf * iW2 - D * iW);
      const float J11 = 2.0f * zb * (1.0f - iW2) + 2.0f * BS2 * zb * iz3;
      const float J12 = 2.0f * zb * zb * iW3;
      const float J21 = -1.0f - BS2 * iz3 + gm1g * iW2;
      const float J22 = -B2 * iW3 + gm1g * (D * iW2 - 2.0f * zf * iW3);
      const float idet = __fdividef(1.0f, J11 * J22 - J12 * J21);
      const float dz = (f1 * J22 - f2 * J12) * idet;
      const float dW = (J11 * f2 - J21 * f1) * idet;
      if (!isfinite(dz) || !isfinite(dW)) {
        active = false;
      } else {
        float zn = zf - dz, Wn = Wf - dW;
        if (!(zn > 0.0f)) zn = 0.5f * zf;
        if (!(Wn >= 1.0f)) Wn = 0.5f * (Wf + 1.0f);
        const bool conv = fabsf(dz) <= 1e-6f * zf && fabsf(dW) <= 1e-6f * Wf;
        zf = zn;
        Wf = Wn;
        if (conv) {
          active = false;
          converged = true;
        }
      }
    }
  }
  z = f32_to_f64i(zf);
  W = f32_to_f64i(Wf);
  if (converged) {
    // z and W are FP32 values: z^2, W^2 and W^2 - 1 are exact in FP64
    const double W2 = W * W, z2 = z * z, W2z2 = W2 * z2, u2 = W2 - 1.0;
    const double zb = z + in.B2;
    const double F1 = zb * zb * u2 * z2 - in.S2 * W2z2 - in.BS2 * fma(2.0, z, in.B2) * W2;
    const double F2 = (in.tau + in.D - z - in.B2) * W2z2 + 0.5 * in.B2 * z2 + 0.5 * in.BS2 * W2 +
                      p.gm1g * z2 * (z - in.D * W);
    const float r = __fdividef(1.0f, zf * Wf);
    const float iz = Wf * r, iW = zf * r;
    const float iW2 = iW * iW, iW3 = iW2 * iW, iz3 = iz * iz * iz;
    const float v2 = f64_to_f32i(u2) * iW2;
    const float zb32 = zf + B2;
    const float J11 = 2.0f * zb32 * v2 + 2.0f * BS2 * zb32 * iz3;
    const float J12 = 2.0f * zb32 * zb32 * iW3;
    const float J21 = -1.0f - BS2 * iz3 + gm1g * iW2;
    const float J22 = -B2 * iW3 + gm1g * (D * iW2 - 2.0f * zf * iW3);
    const float idet = 1.0f / (J11 * J22 - J12 * J21);
    const float s = iz * iz * iW2;  // 1 / (W^2 z^2)
    // F1 and F2 are of order W^2 z^2 times the predictor's error and would
    // underflow FP32 for small z: they are converted at the scale 2^k of s
    // and multiplied by s's significand, an exact power-of-two shift that
    // leaves f1 and f2 unchanged wherever FP32 F1 and F2 are normal
    const bool sn = s > 0.0f && s <= 3.4028235e38f && s >= 1.17549435e-38f;
    const int ks = sn ? f32_exponent(s) : 0;
    const float sm = sn ? f32_significand(s) : s;
    const float f1 = f64_to_f32i(F1, ks) * sm, f2 = f64_to_f32i(F2, ks) * sm;
    const float dz = (f1 * J22 - f2 * J12) * idet;
    const float dW = (J11 * f2 - J21 * f1) * idet;
    if (fabsf(dz) <= 1e-6f * zf && fabsf(dW) <= 1e-6f * Wf) {
      const double zn = z - f32_to_f64i(dz), Wn = W - f32_to_f64i(dW);
      if (dgt0i(zn) && c2p_root_physical(in, p, zn, Wn)) {
        z = zn;
        W = Wn;
        return 0;
      }
    }
  }
  // from the predictor's last point (an unusable guess fails the FP64
  // Newton's own checks and goes on to Newman-Hamlin and bisection)
  double P0 = (double)Pg;
  if (!(P0 > 0.0) || !isfinite(P0)) P0 = p.gm1g * (in.tau + in.D);
  return c2p_solve(in, p, z, W, P0);
}

// Polytropic EOS (Sec. 2.3, P = K rho^gamma): with rho = D / W,
// h = 1 + gamma/(gamma-1) K rho^(gamma-1) and z = rho h W^2 = D W h, the
// momentum equation f(W) = (z + B^2)^2 (1 - 1/W^2) - (B.S)^2 (2z + B^2)/z^2
// - S^2 is <= 0 at W = 1 and grows without bound (monotonically for
// gamma <= 2).  Newton from the guess W, on a bracket [lo, hi] kept from the
// signs of f; a step that leaves the bracket bisects it (or doubles W while
// no upper end is known).  The first step is accepted below tol_first (a
// guess already good to 1e-6 leaves 1e-12 after one quadratic step), later
// ones below nr_tol.  tau is not used.  Returns 0 (Newton), 1 (a bisection
// step was needed) or 2 (no root: atmosphere); z and W on success.
__device__ __forceinline__ int c2p_polytrope(const C2PIn& in, const DevParams& p, double& z, double& W,
                                             double tol_first) {
  const double D = in.D;
  const double dzk = (2.0 - p.gamma) * p.gfac;
  double lo = 1.0, hi = INFINITY, w = W >= 1.0 ? W : 1.0;
  bool bis = false;
  for (int it = 0; it < p.nr_maxit + 200; ++it) {
    const double iw = 1.0 / w;
    const double kr = poly_k_rho_gm1<double>(p, D * iw);  // K rho^(gamma-1)
    const double zz = D * w * (1.0 + p.gfac * kr);
    const double dz = D * (1.0 + dzk * kr);               // dz/dW
    const double zb = zz + in.B2, iz = 1.0 / zz;
    const double v2 = 1.0 - iw * iw;
    const double f = zb * zb * v2 - in.BS2 * (2.0 * zz + in.B2) * iz * iz - in.S2;
    const double df = 2.0 * zb * (dz * v2 + zb * iw * iw * iw) + 2.0 * in.BS2 * dz * zb * iz * iz * iz;
    if (!isfinite(f) || !isfinite(df)) return 2;
    if (f > 0.0) hi = w; else lo = w;
    double wn = w - f / df;
    if (!(wn >= lo && wn <= hi) || !isfinite(wn)) {
      wn = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * lo;
      bis = true;
    }
    const double tol = it == 0 ? tol_first : p.nr_tol;
    if (fabs(wn - w) <= tol * wn || (isfinite(hi) && hi - lo <= 1e-15 * hi)) {
      W = wn;
      z = D * wn * (1.0 + p.gfac * poly_k_rho_gm1<double>(p, D / wn));
      return bis ? 1 : 0;
    }
    w = wn;
  }
  return 2;
}

// FP32 Newton predictor of the polytropic recovery (mixed path): W to
// about 1e-6 from the guess, for the one FP64 step that follows.  Returns
// false (W unchanged) if it does not get there in 8 steps.
__device__ __forceinline__ bool c2p_polytrope_predict(const C2PIn& in, const DevParams& p, double& W) {
  const float D = f64_to_f32i(in.D), B2 = f64_to_f32i(in.B2), BS2 = f64_to_f32i(in.BS2), S2 = f64_to_f32i(in.S2);
  const float gfac = p.gfacf, dzk = (float)((2.0 - p.gamma) * p.gfac);
  float w = fmaxf(f64_to_f32i(W), 1.0f);
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    const float iw = 1.0f / w;
    const float kr = poly_k_rho_gm1<float>(p, D * iw);
    const float zz = D * w * (1.0f + gfac * kr);
    const float dz = D * (1.0f + dzk * kr);
    const float zb = zz + B2, iz = 1.0f / zz;
    const float v2 = 1.0f - iw * iw;
    const float f = zb * zb * v2 - BS2 * (2.0f * zz + B2) * iz * iz - S2;
    const float df = 2.0f * zb * (dz * v2 + zb * iw * iw * iw) + 2.0f * BS2 * dz * zb * iz * iz * iz;
    const float wn = fmaxf(w - f / df, 1.0f);
    if (!isfinite(wn)) return false;
    if (fabsf(wn - w) <= 1e-6f * wn) {
      W = f32_to_f64i(wn);
      return true;
    }
    w = wn;
  }
  return false;
}

// Recovery of the interior cell c (Sec. 2.3).  The incoming primitives of
// the cell are the Newton initial guess and are overwritten with the result.
// Returns the status: 0 Newton, 1 bisection, 2 atmosphere, 3 pressure floor.
// With PREDICT (mixed path) the guess comes from the FP32 primitives prim32
// (in pairs, [q/2][ncell] float2, q even in .x), an FP32 Newton predictor
// runs before the FP64 Newton, and the result is also stored in prim32.  mcache (nullable) holds, per point, 1/sqrt(gamma)
// and gamma^ij in FP64 (7 components), saving the per-call inverse.
// F32IO (with PREDICT) takes the guess from and writes the result to prim32;
// without it the guess is read from the FP64 primitives.  geom32 (nullable,
// F32IO only) is the FP32 geometry cache, whose gamma_ij and gamma^ij then
// serve the single-precision parts.  Without RESULT64 (F32IO only) the
// primitives are formed in FP32 from the FP64 root (z, W) and only prim32 is
// written: for the intermediate stages of a mixed step, whose primitives
// feed only the FP32 RHS and the next recovery's guess.  POLY: the
// polytropic EOS (p.eos == GRMHD_EOS_POLYTROPE; the launchers dispatch on it).
template <bool PREDICT, bool F32IO = PREDICT, bool RESULT64 = true, bool POLY = false>
__device__ __forceinline__ int con2prim_at(const DevGrid& g, const DevParams& p, const double* __restrict__ cons,
                                           const double* __restrict__ metric, double* __restrict__ prim,
                                           long long c, float* __restrict__ prim32 = nullptr,
                                           const double* __restrict__ mcache = nullptr,
                                           const float* __restrict__ geom32 = nullptr) {
  static_assert(RESULT64 || F32IO, "an FP32-only result needs the FP32 primitives");
  CellMetric m;
  double isg;
  if (mcache && metric) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      m.g[i] = __ldg(metric + (4 + i) * g.ncell + c);
      m.gu[i] = __ldg(mcache + (1 + i) * g.ncell + c);
    }
    isg = __ldg(mcache + c);
  } else {
    cell_metric(metric, g.ncell, c, m);
    isg = 1.0 / m.sqrtg;
  }
  double U[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) U[q] = __ldg(cons + q * g.ncell + c);
  const double D = U[0] * isg, tau = U[4] * isg;
  const double Sl[3] = {U[1] * isg, U[2] * isg, U[3] * isg};
  const double B[3] = {U[5] * isg, U[6] * isg, U[7] * isg};
  double Bl[3], Su[3];
  lower(m.g, B, Bl);
  lower(m.gu, Sl, Su);
  C2PIn in;
  in.D = D;
  in.tau = tau;
  in.S2 = Sl[0] * Su[0] + Sl[1] * Su[1] + Sl[2] * Su[2];
  in.B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const double BS = B[0] * Sl[0] + B[1] * Sl[1] + B[2] * Sl[2];
  in.BS2 = BS * BS;
  // initial guess from the incoming primitives
  double* pc = prim + c;
  double W = 1.0, z = 0.0, P0 = 0.0;
  float Wg = 1.0f, zg = 0.0f, Pgf = 0.0f;  // the FP32 guess (F32IO)
  if (F32IO) {
    // the FP32 primitives in pairs, [q/2][ncell] float2 (q even in .x)
    const float2* pf = reinterpret_cast<const float2*>(prim32) + c;
    const float2 p01 = pf[0], p23 = pf[g.ncell], p45 = pf[2 * g.ncell];
    const float v[3] = {p01.y, p23.x, p23.y};
    float gf[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) gf[i] = geom32 ? __ldg(geom32 + (4 + i) * g.ncell + c) : f64_to_f32i(m.g[i]);
    float vl[3];
    lower(gf, v, vl);
    const float v2g = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
    const float rg = p01.x, Pg = p45.x;
    Wg = (v2g >= 0.0f && v2g < 1.0f) ? rsqrtf(1.0f - v2g) : 1.0f;
    zg = (rg > 0.0f && Pg > 0.0f) ? (rg + p.gfacf * Pg) * Wg * Wg : f64_to_f32i(tau + D + in.B2);
    Pgf = Pg;
  } else {
    const double v[3] = {pc[g.ncell], pc[2 * g.ncell], pc[3 * g.ncell]};
    double vl[3];
    lower(m.g, v, vl);
    const double v2g = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
    const double rg = pc[0], Pg = pc[4 * g.ncell];
    W = (dge0i(v2g) && dlt1i(v2g)) ? 1.0 / sqrt(1.0 - v2g) : 1.0;
    z = (dgt0i(rg) && dgt0i(Pg)) ? (rg + p.gfac * Pg) * W * W : (tau + D + in.B2);
    P0 = Pg;
  }
  int st = 2;
  constexpr bool poly = POLY;
  if constexpr (POLY) {
    if (dgt0i(D)) {
      if (F32IO) W = f32_to_f64i(Wg);
      double tol_first = p.nr_tol;
      if (PREDICT && c2p_polytrope_predict(in, p, W)) tol_first = 1e-6;
      st = c2p_polytrope(in, p, z, W, tol_first);
    }
  } else if (dgt0i(D) && dgt0i(tau + D)) {
    // mixed: the FP32 predictor and one refinement step (c2p_solve_mixed);
    // FP64: the predictor only supplies the starting point, and the FP64
    // Newton still converges to nr_tol, so the root (and the floor decision
    // of a cell whose pressure is round-off) is unchanged
    if (PREDICT && p.precision == GRMHD_MIXED && !(p.flags & GRMHD_NEWMAN_HAMLIN)) {
      if (!F32IO) {
        zg = f64_to_f32i(z);
        Wg = f64_to_f32i(W);
        Pgf = f64_to_f32i(P0);
      }
      st = c2p_solve_mixed(in, p, zg, Wg, Pgf, z, W);
    } else {
      if (F32IO) {
        z = f32_to_f64i(zg);
        W = f32_to_f64i(Wg);
        P0 = f32_to_f64i(Pgf);
      }
      if (!dgt0i(P0) || !dfinitei(P0)) P0 = p.gm1g * (tau + D);
      if (PREDICT) c2p_predict_fp32(in, p, z, W);
      st = c2p_solve(in, p, z, W, P0);
    }
  }
  if constexpr (!RESULT64) {
    // FP32 primitives from the FP64 root: 1/W, 1/z, 1/(z + B^2) from one division
    float outf[8];
    // (the conversions on the integer pipe, fpbits.cuh)
    const float Bf[3] = {f64_to_f32i(B[0]), f64_to_f32i(B[1]), f64_to_f32i(B[2])};
    if (st != 2) {
      const float zf = f64_to_f32i(z), Wf = f64_to_f32i(W), zbf = f64_to_f32i(z + in.B2);
      const float X = 1.0f / (Wf * zf * zbf);
      const float iW = zf * zbf * X, iz = Wf * zbf * X, izb = Wf * zf * X;
      const float rho = f64_to_f32i(D) * iW;
      const float P = poly ? rho * poly_k_rho_gm1<float>(p, rho) : p.gm1gf * (zf * iW * iW - rho);
      const float bsz = f64_to_f32i(BS) * iz;
      float gf[6], guf[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        gf[i] = geom32 ? __ldg(geom32 + (4 + i) * g.ncell + c) : f64_to_f32i(m.g[i]);
        guf[i] = geom32 ? __ldg(geom32 + (17 + i) * g.ncell + c) : f64_to_f32i(m.gu[i]);
      }
      float Blf[3], vlo[3], vu[3];
      lower(gf, Bf, Blf);
#pragma unroll
      for (int i = 0; i < 3; ++i) vlo[i] = (f64_to_f32i(Sl[i]) + bsz * Blf[i]) * izb;
      lower(guf, vlo, vu);
      const float v2 = vu[0] * vlo[0] + vu[1] * vlo[1] + vu[2] * vlo[2];
      if (rho >= p.rho_atmf && v2 < 1.0f && isfinite(P)) {
        outf[0] = rho;
        outf[1] = vu[0];
        outf[2] = vu[1];
        outf[3] = vu[2];
        outf[4] = P;
        if (!(P > 0.0f)) {
          outf[4] = p.p_atmf;
          st = 3;
        }
      } else {
        st = 2;
      }
    }
    if (st == 2) {
      outf[0] = p.rho_atmf;
      outf[1] = outf[2] = outf[3] = 0.0f;
      outf[4] = p.p_atmf;
    }
    outf[5] = Bf[0];
    outf[6] = Bf[1];
    outf[7] = Bf[2];
    float2* po = reinterpret_cast<float2*>(prim32) + c;
#pragma unroll
    for (int h = 0; h < 4; ++h) po[h * g.ncell] = make_float2(outf[2 * h], outf[2 * h + 1]);
    return st;
  }
  double out[8];
  if (st != 2) {
    // 1/W, 1/z and 1/(z + B^2) from one division
    const double zb = z + in.B2;
    const double X = 1.0 / (W * z * zb);
    const double iW = z * zb * X, iz = W * zb * X, izb = W * z * X;
    const double rho = D * iW;
    const double P = poly ? rho * poly_k_rho_gm1<double>(p, rho) : p.gm1g * (z * iW * iW - rho);
    const double bsz = BS * iz;
    double vlo[3], vu[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) vlo[i] = (Sl[i] + bsz * Bl[i]) * izb;
    lower(m.gu, vlo, vu);
    const double v2 = vu[0] * vlo[0] + vu[1] * vlo[1] + vu[2] * vlo[2];
    if (dgeci(rho, p.rho_atm) && dlt1i(v2) && dfinitei(P)) {
      out[0] = rho;
      out[1] = vu[0];
      out[2] = vu[1];
      out[3] = vu[2];
      out[4] = P;
      if (!dgt0i(P)) {  // valid density and velocity, non-positive pressure: floor
        out[4] = p.p_atm;
        st = 3;
      }
    } else {
      st = 2;
    }
  }
  if (st == 2) {
    out[0] = p.rho_atm;
    out[1] = out[2] = out[3] = 0.0;
    out[4] = p.p_atm;
  }
  out[5] = B[0];
  out[6] = B[1];
  out[7] = B[2];
#pragma unroll
  for (int q = 0; q < 8; ++q) pc[q * g.ncell] = out[q];
  if (F32IO) {
    float2* po = reinterpret_cast<float2*>(prim32) + c;
#pragma unroll
    for (int h = 0; h < 4; ++h) po[h * g.ncell] = make_float2(f64_to_f32i(out[2 * h]), f64_to_f32i(out[2 * h + 1]));
  }
  return st;
}

// Ghost point c copies its source: periodic wrap or the nearest interior
// point, per axis (edges and corners included).  Interior points: no-op.
// COHERENT: the sources were written by other CTAs of the same launch, so
// they are read through L2 (ld.global.cg).
template <class F, bool COHERENT = false>
__device__ __forceinline__ void fill_ghost_at(const DevGrid& g, int bc, int nvar, F* __restrict__ f, long long c) {
  int idx[3];
  idx[0] = (int)(c % g.N[0]);
  const long long r = c / g.N[0];
  idx[1] = (int)(r % g.N[1]);
  idx[2] = (int)(r / g.N[1]);
  bool interior = true;
  int src[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int i = idx[d] - g.ng;
    if (i < 0 || i >= g.n[d]) interior = false;
    int s;
    if (bc == GRMHD_BC_PERIODIC) {
      s = i % g.n[d];
      if (s < 0) s += g.n[d];
    } else {
      s = i < 0 ? 0 : (i >= g.n[d] ? g.n[d] - 1 : i);
    }
    src[d] = s + g.ng;
  }
  if (interior) return;
  const long long sc = (long long)src[2] * g.sz + (long long)src[1] * g.sy + src[0];
  for (int q = 0; q < nvar; ++q) f[q * g.ncell + c] = COHERENT ? __ldcg(f + q * g.ncell + sc) : f[q * g.ncell + sc];
}

// Interior cell index of the t-th interior point (x fastest).
__device__ __forceinline__ long long interior_cell(const DevGrid& g, long long t) {
  const int xi = (int)(t % g.n[0]);
  const long long r = t / g.n[0];
  const int yi = (int)(r % g.n[1]);
  const int zi = (int)(r / g.n[1]);
  return (long long)(zi + g.ng) * g.sz + (long long)(yi + g.ng) * g.sy + (xi + g.ng);
}

}  // namespace grmhd
