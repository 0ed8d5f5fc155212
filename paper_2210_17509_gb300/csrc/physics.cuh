// Device physics of the Valencia GRMHD RHS in 3+1 component form, templated
// on the compute type T (double for the FP64 path, float for the mixed path).
//
// Formulas (GRaM-X, arXiv 2210.17509, Sec. 2.2):
//   prim -> cons, Eqs. 6-9, with b^0 = W B^i v_i / alpha and
//   b_i = B_i / W + alpha b^0 v_i (the spatial projection of b^mu = u_nu *F^{mu nu});
//   flux F^d, Eq. 12; signal speeds of the fast-magnetosonic bound
//   a^2 = cs^2 + vA^2 - cs^2 vA^2 (HLLE after Gammie 2003, cited in Sec. 2.3);
//   HLLE combination (Sec. 2.3, step 3).
#pragma once

#include <cuda_runtime.h>

#include "fpbits.cuh"
#include "internal.h"

namespace grmhd {

__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xrsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float xrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double xabs(double x) { return fabs(x); }
__device__ __forceinline__ float xabs(float x) { return fabsf(x); }
__device__ __forceinline__ double xmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float xmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double xmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float xmax(float a, float b) { return fmaxf(a, b); }

// ------------------------------------------------------------ reconstruction
// minmod slope limiter (TVD, Sec. 2.3): 0 across an extremum, otherwise the
// smaller one-sided difference (first argument on a tie).
template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
  if (a * b <= T(0)) return T(0);
  return (xabs(a) <= xabs(b)) ? a : b;
}

// WENO5 (Jiang-Shu indicators, linear weights 1/10, 6/10, 3/10): value at
// the face i+1/2 from the cell values i-2 .. i+2 (FP32, per face; the FP64
// paths use weno5_parts and weno5_cell_parts).  The weights use the textbook
// reciprocals so that the squared products cannot overflow in single
// precision.  Every operation is explicit (fused multiply-adds and
// round-to-nearest products and sums), so that the kernels that inline this
// function, which read their stencils from different memories, compute the
// same bits.
template <class T>
__device__ __forceinline__ T weno5(T um2, T um1, T u0, T up1, T up2, T eps);

template <>
__device__ __forceinline__ float weno5<float>(float um2, float um1, float u0, float up1, float up2, float eps) {
  const float c6 = 1.0f / 6.0f, c1312 = 13.0f / 12.0f;
  const float q0 = __fmul_rn(fmaf(2.0f, um2, fmaf(-7.0f, um1, __fmul_rn(11.0f, u0))), c6);
  const float q1 = __fmul_rn(fmaf(2.0f, up1, fmaf(5.0f, u0, -um1)), c6);
  const float q2 = __fmul_rn(fmaf(5.0f, up1, fmaf(2.0f, u0, -up2)), c6);
  const float t0 = fmaf(-2.0f, um1, __fadd_rn(um2, u0)), s0 = fmaf(3.0f, u0, fmaf(-4.0f, um1, um2));
  const float t1 = fmaf(-2.0f, u0, __fadd_rn(um1, up1)), s1 = __fsub_rn(um1, up1);
  const float t2 = fmaf(-2.0f, up1, __fadd_rn(u0, up2)), s2 = fmaf(3.0f, u0, fmaf(-4.0f, up1, up2));
  const float e0 = __fadd_rn(eps, fmaf(__fmul_rn(c1312, t0), t0, __fmul_rn(__fmul_rn(0.25f, s0), s0)));
  const float e1 = __fadd_rn(eps, fmaf(__fmul_rn(c1312, t1), t1, __fmul_rn(__fmul_rn(0.25f, s1), s1)));
  const float e2 = __fadd_rn(eps, fmaf(__fmul_rn(c1312, t2), t2, __fmul_rn(__fmul_rn(0.25f, s2), s2)));
  const float a0 = __fdividef(0.1f, __fmul_rn(e0, e0)), a1 = __fdividef(0.6f, __fmul_rn(e1, e1)),
              a2 = __fdividef(0.3f, __fmul_rn(e2, e2));
  return __fdividef(fmaf(a0, q0, fmaf(a1, q1, __fmul_rn(a2, q2))), __fadd_rn(__fadd_rn(a0, a1), a2));
}

// weno5<float> of two variables at once, one per lane of a float2, in the
// paired FP32 instructions of this GPU (one fma / add / mul instruction for
// both lanes, half the issue slots of the scalar form).  The operations are
// weno5<float>'s in the same order; every negated operand is moved into a
// constant (round-to-nearest is symmetric in sign: fl(-x) = -fl(x)), and the
// divisions stay per lane, so each lane has the bits of weno5<float>.
__device__ __forceinline__ float2 f2c(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 weno5_x2(float2 um2, float2 um1, float2 u0, float2 up1, float2 up2, float2 eps) {
  const float c6 = 1.0f / 6.0f, c1312 = 13.0f / 12.0f;
  // q0 = (2 um2 - 7 um1 + 11 u0) / 6
  const float2 q0 = __fmul2_rn(__ffma2_rn(f2c(2.0f), um2, __ffma2_rn(f2c(-7.0f), um1, __fmul2_rn(f2c(11.0f), u0))),
                               f2c(c6));
  // q1 = (2 up1 + (5 u0 - um1)) / 6 = (-2 up1 + (um1 - 5 u0)) * (-1/6)
  const float2 q1 = __fmul2_rn(__ffma2_rn(f2c(-2.0f), up1, __ffma2_rn(f2c(-5.0f), u0, um1)), f2c(-c6));
  // q2 = (5 up1 + (2 u0 - up2)) / 6 = (-5 up1 + (up2 - 2 u0)) * (-1/6)
  const float2 q2 = __fmul2_rn(__ffma2_rn(f2c(-5.0f), up1, __ffma2_rn(f2c(-2.0f), u0, up2)), f2c(-c6));
  const float2 t0 = __ffma2_rn(f2c(-2.0f), um1, __fadd2_rn(um2, u0));
  const float2 s0 = __ffma2_rn(f2c(3.0f), u0, __ffma2_rn(f2c(-4.0f), um1, um2));
  const float2 t1 = __ffma2_rn(f2c(-2.0f), u0, __fadd2_rn(um1, up1));
  const float2 s1 = __ffma2_rn(f2c(-1.0f), up1, um1);  // um1 - up1, rounded once
  const float2 t2 = __ffma2_rn(f2c(-2.0f), up1, __fadd2_rn(u0, up2));
  const float2 s2 = __ffma2_rn(f2c(3.0f), u0, __ffma2_rn(f2c(-4.0f), up1, up2));
  const float2 e0 = __fadd2_rn(eps, __ffma2_rn(__fmul2_rn(f2c(c1312), t0), t0, __fmul2_rn(__fmul2_rn(f2c(0.25f), s0), s0)));
  const float2 e1 = __fadd2_rn(eps, __ffma2_rn(__fmul2_rn(f2c(c1312), t1), t1, __fmul2_rn(__fmul2_rn(f2c(0.25f), s1), s1)));
  const float2 e2 = __fadd2_rn(eps, __ffma2_rn(__fmul2_rn(f2c(c1312), t2), t2, __fmul2_rn(__fmul2_rn(f2c(0.25f), s2), s2)));
  const float2 w0 = __fmul2_rn(e0, e0), w1 = __fmul2_rn(e1, e1), w2 = __fmul2_rn(e2, e2);
  const float2 a0 = make_float2(__fdividef(0.1f, w0.x), __fdividef(0.1f, w0.y));
  const float2 a1 = make_float2(__fdividef(0.6f, w1.x), __fdividef(0.6f, w1.y));
  const float2 a2 = make_float2(__fdividef(0.3f, w2.x), __fdividef(0.3f, w2.y));
  const float2 num = __ffma2_rn(a0, q0, __ffma2_rn(a1, q1, __fmul2_rn(a2, q2)));
  const float2 den = __fadd2_rn(__fadd2_rn(a0, a1), a2);
  return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

// Both WENO5 states of the face between cells c-1 and c from the six values
// u[c-3 .. c+2]: the left state from cell c-1, the right state (mirrored
// stencil) from cell c.  In FP64 the two normalisations share one division:
// 1/a and 1/b come from 1/(a b).
template <class T>
__device__ __forceinline__ void weno5_pair(T um3, T um2, T um1, T u0, T up1, T up2, T eps, T& vL, T& vR) {
  vL = weno5<T>(um3, um2, um1, u0, up1, eps);
  vR = weno5<T>(up2, up1, u0, um1, um2, eps);
}

__device__ __forceinline__ void weno5_parts(double um2, double um1, double u0, double up1, double up2, double eps,
                                            double& num, double& den) {
  const double c6 = 1.0 / 6.0, c1312 = 13.0 / 12.0;
  const double q0 = (2.0 * um2 - 7.0 * um1 + 11.0 * u0) * c6;
  const double q1 = (-um1 + 5.0 * u0 + 2.0 * up1) * c6;
  const double q2 = (2.0 * u0 + 5.0 * up1 - up2) * c6;
  const double t0 = um2 - 2.0 * um1 + u0, s0 = um2 - 4.0 * um1 + 3.0 * u0;
  const double t1 = um1 - 2.0 * u0 + up1, s1 = um1 - up1;
  const double t2 = u0 - 2.0 * up1 + up2, s2 = 3.0 * u0 - 4.0 * up1 + up2;
  const double e0 = eps + (c1312 * t0 * t0 + 0.25 * s0 * s0);
  const double e1 = eps + (c1312 * t1 * t1 + 0.25 * s1 * s1);
  const double e2 = eps + (c1312 * t2 * t2 + 0.25 * s2 * s2);
  const double p01 = e0 * e1, p02 = e0 * e2, p12 = e1 * e2;
  const double w0 = 0.1 * p12 * p12, w1 = 0.6 * p02 * p02, w2 = 0.3 * p01 * p01;
  num = w0 * q0 + w1 * q1 + w2 * q2;
  den = w0 + w1 + w2;
}

template <>
__device__ __forceinline__ void weno5_pair<double>(double um3, double um2, double um1, double u0, double up1,
                                                   double up2, double eps, double& vL, double& vR) {
  double nL, dL, nR, dR;
  weno5_parts(um3, um2, um1, u0, up1, eps, nL, dL);
  weno5_parts(up2, up1, u0, um1, um2, eps, nR, dR);
  const double r = 1.0 / (dL * dR);
  vL = nL * (dR * r);
  vR = nR * (dL * r);
}

// Both WENO5 states of one cell i from u[i-2 .. i+2]: "plus" is the value at
// the upper face i+1/2 (the left state of that face), "minus" the value at
// the lower face i-1/2 (the right state, mirrored stencil).  The mirrored
// stencil has the same three smoothness indicators in reverse order, so
// they are formed once.  Two rescalings leave the nonlinear weights
// unchanged: every (eps + beta_k) is multiplied by 12/13, which makes it
// t_k^2 + (3/13) s_k^2 + (12/13) eps (eps13 is that last term), and the
// candidate values are kept as 6 q_k, the factor 6 moving into the
// denominator.
//
// FP64 (the FP64 pipe is what bounds the RHS): everything is formed from the
// four first differences of the stencil, dA = u[i-1] - u[i-2], dB = u[i] -
// u[i-1], dC = u[i+1] - u[i], dD = u[i+2] - u[i+1].  The second differences
// are t0 = dB - dA, t1 = dC - dB, t2 = dD - dC; the one-sided ones s0 = 3 dB
// - dA, s1 = dB + dC (a sign that the square drops), s2 = dD - 3 dC; and
// each candidate is 6 q_k = 6 u[i] + (a two-term combination of differences):
// plus (5 dB - 2 dA, 2 dC + dB, 4 dC - dD), minus (2 dD - 5 dC, -2 dB - dC,
// dA - 4 dB).  As the weights sum to one, a state is u[i] + num / (6 den):
// 46 FP64 operations for both states of a value instead of 52 in terms of
// the values themselves.
// Product form of the weights: d_k / e_k^2 times (e_0 e_1 e_2)^2 are plus
// (P12, 6 P02, 3 P01) and minus (P01, 6 P02, 3 P12) up to a common factor,
// with Pjk = (e_j e_k)^2; the caller forms u[i] + num / (6 den).  Every
// product and sum is written explicitly (rounded products and sums, fused
// multiply-adds), so that every kernel that inlines this forms the same bits.
struct Weno5Cell {
  double dA, dB, dC, dD;   // first differences
  double P01, P12, A, B, C;  // weights (plus: P12, A, B; minus: P01, A, C)
};

// The weights from the first differences (dA .. dD) and the second
// differences t0 = dB - dA, t1 = dC - dB, t2 = dD - dC of the stencil.
__device__ __forceinline__ void weno5_cell_weights_dt(double dA, double dB, double dC, double dD, double t0,
                                                      double t1, double t2, double eps13, Weno5Cell& w) {
  const double k313 = 3.0 / 13.0;
  w.dA = dA;
  w.dB = dB;
  w.dC = dC;
  w.dD = dD;
  const double s0 = fma(3.0, w.dB, -w.dA), s1 = __dadd_rn(w.dB, w.dC), s2 = fma(-3.0, w.dC, w.dD);
  const double e0 = fma(t0, t0, fma(__dmul_rn(k313, s0), s0, eps13));
  const double e1 = fma(t1, t1, fma(__dmul_rn(k313, s1), s1, eps13));
  const double e2 = fma(t2, t2, fma(__dmul_rn(k313, s2), s2, eps13));
  const double p01 = __dmul_rn(e0, e1), p02 = __dmul_rn(e0, e2), p12 = __dmul_rn(e1, e2);
  w.P01 = __dmul_rn(p01, p01);
  w.P12 = __dmul_rn(p12, p12);
  w.A = __dmul_rn(6.0, __dmul_rn(p02, p02));
  w.B = __dmul_rn(3.0, w.P01);
  w.C = __dmul_rn(3.0, w.P12);
}

__device__ __forceinline__ void weno5_cell_weights(double um2, double um1, double u0, double up1, double up2,
                                                   double eps13, Weno5Cell& w) {
  const double dA = __dsub_rn(um1, um2), dB = __dsub_rn(u0, um1), dC = __dsub_rn(up1, u0), dD = __dsub_rn(up2, up1);
  weno5_cell_weights_dt(dA, dB, dC, dD, __dsub_rn(dB, dA), __dsub_rn(dC, dB), __dsub_rn(dD, dC), eps13, w);
}

__device__ __forceinline__ double weno5_cell_num_plus(const Weno5Cell& w) {
  const double q0 = fma(5.0, w.dB, __dmul_rn(-2.0, w.dA));
  const double q1 = fma(2.0, w.dC, w.dB);
  const double q2 = fma(4.0, w.dC, -w.dD);
  return fma(w.P12, q0, fma(w.A, q1, __dmul_rn(w.B, q2)));
}

__device__ __forceinline__ double weno5_cell_num_minus(const Weno5Cell& w) {
  const double q0 = fma(2.0, w.dD, __dmul_rn(-5.0, w.dC));
  const double q1 = fma(-2.0, w.dB, -w.dC);
  const double q2 = fma(-4.0, w.dB, w.dA);
  return fma(w.P01, q0, fma(w.A, q1, __dmul_rn(w.C, q2)));
}

__device__ __forceinline__ void weno5_cell_parts(double um2, double um1, double u0, double up1, double up2,
                                                 double eps13, double& nm, double& dm, double& np, double& dp) {
  Weno5Cell w;
  weno5_cell_weights(um2, um1, u0, up1, up2, eps13, w);
  np = weno5_cell_num_plus(w);
  dp = __dadd_rn(__dadd_rn(w.P12, w.A), w.B);
  nm = weno5_cell_num_minus(w);
  dm = __dadd_rn(__dadd_rn(w.P01, w.A), w.C);
}

// weno5_cell_parts of two neighbouring cells i and i+1 of a line from the
// six values u[i-2 .. i+3]: the two stencils share four values, and with
// them three first differences and two second differences, which are formed
// once (the same operations on the same operands, so each cell has the bits
// of weno5_cell_parts).  Part 1 is skipped (outputs untouched) when !two.
__device__ __forceinline__ void weno5_two_cell_parts(const double u[6], double eps13, bool two, double& nm0,
                                                     double& dm0, double& np0, double& dp0, double& nm1, double& dm1,
                                                     double& np1, double& dp1) {
  const double d0 = __dsub_rn(u[1], u[0]), d1 = __dsub_rn(u[2], u[1]), d2 = __dsub_rn(u[3], u[2]),
               d3 = __dsub_rn(u[4], u[3]);
  const double t0 = __dsub_rn(d1, d0), t1 = __dsub_rn(d2, d1), t2 = __dsub_rn(d3, d2);
  Weno5Cell w;
  weno5_cell_weights_dt(d0, d1, d2, d3, t0, t1, t2, eps13, w);
  np0 = weno5_cell_num_plus(w);
  dp0 = __dadd_rn(__dadd_rn(w.P12, w.A), w.B);
  nm0 = weno5_cell_num_minus(w);
  dm0 = __dadd_rn(__dadd_rn(w.P01, w.A), w.C);
  if (two) {
    const double d4 = __dsub_rn(u[5], u[4]);
    weno5_cell_weights_dt(d1, d2, d3, d4, t1, t2, __dsub_rn(d4, d3), eps13, w);
    np1 = weno5_cell_num_plus(w);
    dp1 = __dadd_rn(__dadd_rn(w.P12, w.A), w.B);
    nm1 = weno5_cell_num_minus(w);
    dm1 = __dadd_rn(__dadd_rn(w.P01, w.A), w.C);
  }
}

// The numerator of one of the two states of weno5_cell_parts (plus: the
// value at the upper face, else at the lower face) and both denominators,
// with the same arithmetic (so that the shared division rounds the same).
__device__ __forceinline__ void weno5_cell_parts_one(double um2, double um1, double u0, double up1, double up2,
                                                     double eps13, bool plus, double& num, double& dm,
                                                     double& dp) {
  Weno5Cell w;
  weno5_cell_weights(um2, um1, u0, up1, up2, eps13, w);
  dp = __dadd_rn(__dadd_rn(w.P12, w.A), w.B);
  dm = __dadd_rn(__dadd_rn(w.P01, w.A), w.C);
  num = plus ? weno5_cell_num_plus(w) : weno5_cell_num_minus(w);
}

// A state from its parts: u[i] + num * (the other denominator's share of the
// one division), the division giving 1 / (6 den_this den_other ...).
__device__ __forceinline__ double weno5_cell_state(double u0, double num, double other_den_times_x) {
  return fma(num, other_den_times_x, u0);
}

// FP32: reciprocal form (the squared products could overflow in single
// precision): weights r_k = 1 / e_k^2, plus (r0, 6 r1, 3 r2), minus
// (r2, 6 r1, 3 r0).
__device__ __forceinline__ void weno5_cell(float um2, float um1, float u0, float up1, float up2, float eps13,
                                           float& vm, float& vp) {
  const float k313 = 3.0f / 13.0f;
  const float t0 = fmaf(-2.0f, um1, um2 + u0), s0 = fmaf(3.0f, u0, fmaf(-4.0f, um1, um2));
  const float t1 = fmaf(-2.0f, u0, um1 + up1), s1 = um1 - up1;
  const float t2 = fmaf(-2.0f, up1, u0 + up2), s2 = fmaf(3.0f, u0, fmaf(-4.0f, up1, up2));
  const float e0 = fmaf(t0, t0, fmaf(k313 * s0, s0, eps13));
  const float e1 = fmaf(t1, t1, fmaf(k313 * s1, s1, eps13));
  const float e2 = fmaf(t2, t2, fmaf(k313 * s2, s2, eps13));
  const float r0 = __fdividef(1.0f, e0 * e0), r1 = 6.0f * __fdividef(1.0f, e1 * e1), r2 = __fdividef(1.0f, e2 * e2);
  const float u11 = 11.0f * u0;
  const float qp0 = fmaf(2.0f, um2, fmaf(-7.0f, um1, u11));
  const float qp1 = fmaf(2.0f, up1, fmaf(5.0f, u0, -um1));
  const float qp2 = fmaf(5.0f, up1, fmaf(2.0f, u0, -up2));
  const float qm0 = fmaf(2.0f, up2, fmaf(-7.0f, up1, u11));
  const float qm1 = fmaf(2.0f, um1, fmaf(5.0f, u0, -up1));
  const float qm2 = fmaf(5.0f, um1, fmaf(2.0f, u0, -um2));
  const float R0 = 3.0f * r0, R2 = 3.0f * r2;
  vp = __fdividef(fmaf(r0, qp0, fmaf(r1, qp1, R2 * qp2)), 6.0f * (r0 + r1 + R2));
  vm = __fdividef(fmaf(r2, qm0, fmaf(r1, qm1, R0 * qm2)), 6.0f * (r2 + r1 + R0));
}

// Both minmod states of one cell from u[i-1 .. i+1].
template <class T>
__device__ __forceinline__ void minmod_cell(T um1, T u0, T up1, T& vm, T& vp) {
  const T h = T(0.5) * minmod<T>(u0 - um1, up1 - u0);
  vp = u0 + h;
  vm = u0 - h;
}

// ---------------------------------------------------------------- geometry
// The factors of the Eq. 13 sources that depend on the metric alone (static
// for a static metric): formed per cell on the fly from the metric, or read
// from the FP64 geometry cache, where they are formed once in FP64 with the
// same operations (source_statics).
template <class T>
struct SrcStatics {
  T ia, ia2;     // 1 / alpha, 1 / alpha^2
  T bia2[3];     // beta^i / alpha^2
  T M[6];        // gamma^ij - beta^i beta^j / alpha^2 (packed like gamma)
  T betal[3];    // beta_i = gamma_ij beta^j
  T asg;         // alpha sqrt(gamma)
  T bb[6];       // beta^i beta^j (packed)
  T bda;         // beta^i d_i alpha
};
constexpr int kSrcStaticsComps = 22;
static_assert(kGeomCacheStat + kSrcStaticsComps == kGeomCacheComps, "geometry cache layout");

template <class T>
__device__ __forceinline__ void source_statics(const T alpha, const T beta[3], const T gm[6], const T sg,
                                               const T gu[6], const T da[3], SrcStatics<T>& st) {
  const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
  st.ia = T(1) / alpha;
  st.ia2 = st.ia * st.ia;
#pragma unroll
  for (int i = 0; i < 3; ++i) st.bia2[i] = beta[i] * st.ia2;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    st.bb[s] = beta[I6[s]] * beta[J6[s]];
    st.M[s] = gu[s] - st.bb[s] * st.ia2;
  }
  st.betal[0] = gm[0] * beta[0] + gm[1] * beta[1] + gm[2] * beta[2];
  st.betal[1] = gm[1] * beta[0] + gm[3] * beta[1] + gm[4] * beta[2];
  st.betal[2] = gm[2] * beta[0] + gm[4] * beta[1] + gm[5] * beta[2];
  st.asg = alpha * sg;
  st.bda = beta[0] * da[0] + beta[1] * da[1] + beta[2] * da[2];
}

// Metric at a face (or a cell) converted to the compute type.
template <class T>
struct Geom {
  T alpha, beta[3];
  T g[6];      // gamma_xx, gamma_xy, gamma_xz, gamma_yy, gamma_yz, gamma_zz
  T sqrtg;     // sqrt(det gamma)
  T gup_dd;    // gamma^{dd} of the face normal
  T ia;        // 1 / alpha (set by the run-time-normal face routines)
};

// Face metric = mean of the two adjacent cell-centre values; sqrt(gamma) and
// gamma^{dd} are always computed in FP64.
template <class T, int DIR>
__device__ __forceinline__ void face_geom(const double* __restrict__ metric, long long ncell, long long c,
                                          long long stride, Geom<T>& m) {
  double a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = 0.5 * (__ldg(metric + q * ncell + c - stride) + __ldg(metric + q * ncell + c));
  const double gxx = a[4], gxy = a[5], gxz = a[6], gyy = a[7], gyz = a[8], gzz = a[9];
  const double cxx = gyy * gzz - gyz * gyz;
  const double cyy = gxx * gzz - gxz * gxz;
  const double czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx - gxy * (gxy * gzz - gyz * gxz) + gxz * (gxy * gyz - gyy * gxz);
  const double cdd = (DIR == 0) ? cxx : ((DIR == 1) ? cyy : czz);
  m.alpha = (T)a[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = (T)a[1 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = (T)a[4 + i];
  m.sqrtg = (T)sqrt(det);
  m.gup_dd = (T)(cdd / det);
}

// Face metric with the face normal given at run time (dir = 0, 1, 2).
template <class T>
__device__ __forceinline__ void face_geom_rt(const double* __restrict__ metric, long long ncell, long long c,
                                             long long stride, int dir, Geom<T>& m) {
  double a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = 0.5 * (__ldg(metric + q * ncell + c - stride) + __ldg(metric + q * ncell + c));
  const double gxx = a[4], gxy = a[5], gxz = a[6], gyy = a[7], gyz = a[8], gzz = a[9];
  const double cxx = gyy * gzz - gyz * gyz;
  const double cyy = gxx * gzz - gxz * gxz;
  const double czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx - gxy * (gxy * gzz - gyz * gxz) + gxz * (gxy * gyz - gyy * gxz);
  const double cdd = (dir == 0) ? cxx : ((dir == 1) ? cyy : czz);
  m.alpha = (T)a[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = (T)a[1 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) m.g[i] = (T)a[4 + i];
  m.sqrtg = (T)sqrt(det);
  m.gup_dd = (T)(cdd / det);
  m.ia = T(1) / m.alpha;
}

template <class T>
__device__ __forceinline__ T sel3(int k, T a, T b, T c) { return k == 0 ? a : (k == 1 ? b : c); }

// Cyclic relabelling of the axes that makes the face normal dir the first
// axis: new axis k is old axis (dir + k) mod 3.  Applied to a primitive
// state and to the face metric, so that one face-state routine (normal = x)
// serves all three directions; unrotate_flux maps the result back.
template <class T>
__device__ __forceinline__ void rotate_state(int dir, const T in[8], T out[8]) {
  out[0] = in[0];
  out[4] = in[4];
  out[1] = sel3(dir, in[1], in[2], in[3]);
  out[2] = sel3(dir, in[2], in[3], in[1]);
  out[3] = sel3(dir, in[3], in[1], in[2]);
  out[5] = sel3(dir, in[5], in[6], in[7]);
  out[6] = sel3(dir, in[6], in[7], in[5]);
  out[7] = sel3(dir, in[7], in[5], in[6]);
}

// A vector in rotated axes (new axis k = old axis (dir + k) mod 3).
template <class T>
__device__ __forceinline__ void rotate_vec(int dir, const T in[3], T out[3]) {
  out[0] = sel3(dir, in[0], in[1], in[2]);
  out[1] = sel3(dir, in[1], in[2], in[0]);
  out[2] = sel3(dir, in[2], in[0], in[1]);
}

template <class T>
__device__ __forceinline__ void unrotate_flux(int dir, const T in[8], T out[8]) {
  out[0] = in[0];
  out[4] = in[4];
  out[1] = sel3(dir, in[1], in[3], in[2]);
  out[2] = sel3(dir, in[2], in[1], in[3]);
  out[3] = sel3(dir, in[3], in[2], in[1]);
  out[5] = sel3(dir, in[5], in[7], in[6]);
  out[6] = sel3(dir, in[6], in[5], in[7]);
  out[7] = sel3(dir, in[7], in[6], in[5]);
}

// Packed symmetric metric [xx, xy, xz, yy, yz, zz] and shift in rotated axes.
template <class T>
__device__ __forceinline__ void rotate_metric(int dir, Geom<T>& m) {
  const T gxx = m.g[0], gxy = m.g[1], gxz = m.g[2], gyy = m.g[3], gyz = m.g[4], gzz = m.g[5];
  m.g[0] = sel3(dir, gxx, gyy, gzz);
  m.g[1] = sel3(dir, gxy, gyz, gxz);
  m.g[2] = sel3(dir, gxz, gxy, gyz);
  m.g[3] = sel3(dir, gyy, gzz, gxx);
  m.g[4] = sel3(dir, gyz, gxz, gxy);
  m.g[5] = sel3(dir, gzz, gxx, gyy);
  const T bx = m.beta[0], by = m.beta[1], bz = m.beta[2];
  m.beta[0] = sel3(dir, bx, by, bz);
  m.beta[1] = sel3(dir, by, bz, bx);
  m.beta[2] = sel3(dir, bz, bx, by);
}

template <class T>
__device__ __forceinline__ void lower(const T g[6], const T v[3], T vl[3]) {
  vl[0] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  vl[1] = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  vl[2] = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
}

// Polytropic EOS (Sec. 2.3): the pressure entry of a state is K rho^gamma
// (states with rho <= 0 are left to the physical-state checks).
// K rho^(gamma - 1) of the polytrope: a plain product for gamma = 2 (the
// paper's TOV polytrope, Sec. 4.4), pow otherwise.
template <class T>
__device__ __forceinline__ T poly_k_rho_gm1(const DevParams& p, T rho) {
  if (p.poly_g2) return (T)p.poly_K * rho;
  if constexpr (sizeof(T) == 4) return (float)p.poly_K * powf(rho, (float)(p.gamma - 1.0));
  else return p.poly_K * pow(rho, p.gamma - 1.0);
}

template <class T>
__device__ __forceinline__ void apply_polytrope_pair(const DevParams& p, T pL[8], T pR[8]) {
  if (pL[0] > T(0)) pL[4] = pL[0] * poly_k_rho_gm1<T>(p, pL[0]);
  if (pR[0] > T(0)) pR[4] = pR[0] * poly_k_rho_gm1<T>(p, pR[0]);
}

// As physical_state, also returning the lowered velocity and v^2.
template <class T, bool CURVED>
__device__ __forceinline__ bool physical_state_v(const T pr[8], const Geom<T>& m, T vl[3], T& v2) {
  const T v[3] = {pr[1], pr[2], pr[3]};
  if (CURVED) {
    lower(m.g, v, vl);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) vl[i] = v[i];
  }
  v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  // FP64: the comparisons on the integer pipe (fpbits.cuh)
  if constexpr (sizeof(T) == 8) return dgt0i(pr[0]) && dgt0i(pr[4]) && dlt1i(v2);
  else return pr[0] > T(0) && pr[4] > T(0) && v2 < T(1);
}

template <class T, bool CURVED>
__device__ __forceinline__ bool physical_state(const T pr[8], const Geom<T>& m) {
  const T v[3] = {pr[1], pr[2], pr[3]};
  T v2;
  if (CURVED) {
    T vl[3];
    lower(m.g, v, vl);
    v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  } else {
    v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  }
  // FP64: the comparisons on the integer pipe (fpbits.cuh)
  if constexpr (sizeof(T) == 8) return dgt0i(pr[0]) && dgt0i(pr[4]) && dlt1i(v2);
  else return pr[0] > T(0) && pr[4] > T(0) && v2 < T(1);
}

// ------------------------------------------------- one side of a Riemann face
template <class T>
struct Side {
  T U[8];
  T F[8];
  T lm, lp;
  T sden;  // speed denominator (SHARED side states only)
};

// Conserved vector (Eqs. 6-9), flux along DIR (Eq. 12) and signal speeds of
// the primitive state pr at a face with metric m.
//
// Signal speeds: with the fast-magnetosonic bound
// a^2 = cs^2 + vA^2 - cs^2 vA^2, cs^2 = Gamma P / (rho h), vA^2 = b^2 / hs,
// hs = rho h + b^2, the bound simplifies to a^2 = Na / hs, Na = Gamma P + b^2,
// and the two roots become
//   lambda_pm = alpha [v^d (hs - Na) pm sqrt(Na (1 - v^2) Q)] / (hs - v^2 Na) - beta^d,
//   Q = gamma^{dd} (hs - v^2 Na) - (v^d)^2 (hs - Na)   (clamped at 0),
// one division per side.  SHARED: the caller passes 1/alpha (ia) and
// finishes the speeds itself -- lm / lp then hold the bracketed numerators
// and sden the denominator -- so that the two sides of a face share one
// division (finish_speeds).
//
// SCALED (with SHARED): U and F come without their common factors sqrt(gamma)
// and alpha (alpha sqrt(gamma) for F), which the two sides of a face share;
// hlle_combine_scaled applies them once.  vl_in / v2_in (nullable): the
// lowered velocity and v^2, when the caller has them already.
template <class T, bool CURVED, int DIR, bool SHARED = false, bool SCALED = false>
__device__ __forceinline__ void side_state(const T pr[8], const Geom<T>& m, T gamma, T gfac, Side<T>& o,
                                           T ia_in = T(0), const T* vl_in = nullptr, T v2_in = T(0)) {
  static_assert(!SCALED || SHARED, "scaled side states finish their speeds with the face");
  const T rho = pr[0], P = pr[4];
  const T v[3] = {pr[1], pr[2], pr[3]};
  const T B[3] = {pr[5], pr[6], pr[7]};
  T vl[3], Bl[3];
  if (CURVED) {
    if (vl_in) {
#pragma unroll
      for (int i = 0; i < 3; ++i) vl[i] = vl_in[i];
    } else {
      lower(m.g, v, vl);
    }
    lower(m.g, B, Bl);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { vl[i] = v[i]; Bl[i] = B[i]; }
  }
  const T v2 = vl_in ? v2_in : v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  const T Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const T B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const T omv2 = T(1) - v2;
  const T W = xrsqrt(omv2);         // Lorentz factor
  const T iW = omv2 * W;            // 1 / W
  const T ab0 = W * Bv;             // alpha b^0
  const T b2 = B2 * omv2 + Bv * Bv; // (B^2 + (alpha b^0)^2) / W^2
  T bl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bl[i] = Bl[i] * iW + ab0 * vl[i];
  const T rhoh = rho + gfac * P;
  const T hs = rhoh + b2;           // rho h*
  const T Ps = P + T(0.5) * b2;     // P*
  const T sg = (CURVED && !SCALED) ? m.sqrtg : T(1);
  const T hW2 = hs * W * W;
  const T D = sg * rho * W;
#pragma unroll
  for (int i = 0; i < 3; ++i) o.U[1 + i] = sg * (hW2 * vl[i] - ab0 * bl[i]);
  const T tau = sg * (hW2 - Ps - ab0 * ab0) - D;
  o.U[0] = D;
  o.U[4] = tau;
  T Bc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) { Bc[i] = sg * B[i]; o.U[5 + i] = Bc[i]; }
  // flux along DIR
  const T alpha = CURVED ? m.alpha : T(1);
  const T af = SCALED ? T(1) : alpha;  // lapse factor of the fluxes
  T vt[3];
  if (CURVED) {
    const T ia = SHARED ? ia_in : T(1) / alpha;
#pragma unroll
    for (int i = 0; i < 3; ++i) vt[i] = v[i] - m.beta[i] * ia;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) vt[i] = v[i];
  }
  const T vtd = vt[DIR];
  const T sgPs = sg * Ps;
  const T BdiW = Bc[DIR] * iW;
  o.F[0] = af * (D * vtd);
#pragma unroll
  for (int j = 0; j < 3; ++j) o.F[1 + j] = af * (o.U[1 + j] * vtd + (j == DIR ? sgPs : T(0)) - bl[j] * BdiW);
  o.F[4] = af * (tau * vtd + sgPs * v[DIR] - ab0 * BdiW);
#pragma unroll
  for (int k = 0; k < 3; ++k) o.F[5 + k] = (k == DIR) ? T(0) : af * (Bc[k] * vtd - Bc[DIR] * vt[k]);
  // signal speeds
  const T Na = gamma * P + b2;
  const T dsp = hs - v2 * Na;  // (1 - v^2 a^2) hs
  const T hmn = hs - Na;       // (1 - a^2) hs
  const T gdd = CURVED ? m.gup_dd : T(1);
  const T vd = v[DIR];
  T Q = gdd * dsp - vd * vd * hmn;
  if constexpr (sizeof(T) == 8) Q = dmax0i(Q);  // the clamp on the integer pipe (fpbits.cuh)
  else Q = xmax(Q, T(0));
  T sq;
  if constexpr (sizeof(T) == 8) sq = sqrt_nr(Na * omv2 * Q);  // fpbits.cuh
  else sq = xsqrt(Na * omv2 * Q);
  const T c0 = vd * hmn;
  if (SHARED) {
    o.lp = c0 + sq;
    o.lm = c0 - sq;
    o.sden = dsp;
  } else {
    const T ide = alpha / dsp;
    const T bd = CURVED ? m.beta[DIR] : T(0);
    o.lp = ide * (c0 + sq) - bd;
    o.lm = ide * (c0 - sq) - bd;
  }
}

// ------------------------------------- both sides of a face, paired (FP32)
// The two sides of a face run the same operations on different states, so
// the FP32 face code forms them together: the left state in the .x lane and
// the right state in the .y lane of paired FP32 instructions (one fma / add
// / mul instruction for both sides), the metric of the face broadcast to both
// lanes.  Square roots, reciprocal square roots and clamps stay per lane.
// The operations are those of side_state<float, CURVED, 0, true, true> and
// physical_state, with every sum and product written explicitly; they
// differ from the scalar forms only in rounding order, and every FP32 kernel
// forms its face fluxes through these, so the tiles, the batched kernels and
// the constrained-transport ring faces stay bit-identical to one another.
// a - b and -a, each rounded once (-1 * b is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(f2c(-1.0f), b, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(f2c(-1.0f), a); }
// lowered vectors of both sides with the face metric
template <bool CURVED>
__device__ __forceinline__ void lower_x2(const Geom<float>& m, const float2 v[3], float2 vl[3]) {
  if (CURVED) {
    const float2 g0 = f2c(m.g[0]), g1 = f2c(m.g[1]), g2 = f2c(m.g[2]), g3 = f2c(m.g[3]), g4 = f2c(m.g[4]),
                 g5 = f2c(m.g[5]);
    vl[0] = __ffma2_rn(g2, v[2], __ffma2_rn(g1, v[1], __fmul2_rn(g0, v[0])));
    vl[1] = __ffma2_rn(g4, v[2], __ffma2_rn(g3, v[1], __fmul2_rn(g1, v[0])));
    vl[2] = __ffma2_rn(g5, v[2], __ffma2_rn(g4, v[1], __fmul2_rn(g2, v[0])));
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) vl[i] = v[i];
  }
}
__device__ __forceinline__ float2 dot_x2(const float2 a[3], const float2 b[3]) {
  return __ffma2_rn(a[2], b[2], __ffma2_rn(a[1], b[1], __fmul2_rn(a[0], b[0])));
}
// physical_state of both face states (unrotated, with the face metric)
template <bool CURVED>
__device__ __forceinline__ void physical_states_x2(const float pL[8], const float pR[8], const Geom<float>& m,
                                                   bool& okL, bool& okR) {
  float2 v[3], vl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = make_float2(pL[1 + i], pR[1 + i]);
  lower_x2<CURVED>(m, v, vl);
  const float2 v2 = dot_x2(v, vl);
  okL = pL[0] > 0.0f && pL[4] > 0.0f && v2.x < 1.0f;
  okR = pR[0] > 0.0f && pR[4] > 0.0f && v2.y < 1.0f;
}
// Side states of a face whose normal is the first axis (rotated states rL,
// rR), SHARED and SCALED as side_state<float, CURVED, 0, true, true> forms
// them: U and F without sqrt(gamma) and alpha, the speed numerators in lp /
// lm and the denominator in sden, for finish_speeds and hlle_combine_scaled.
// ia = 1 / alpha of the face.
template <bool CURVED>
__device__ __forceinline__ void side_states_x2(const float rL[8], const float rR[8], const Geom<float>& m,
                                               float gamma, float gfac, float ia, Side<float>& L, Side<float>& R) {
  const float2 rho = make_float2(rL[0], rR[0]), P = make_float2(rL[4], rR[4]);
  float2 v[3], B[3], vl[3], Bl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = make_float2(rL[1 + i], rR[1 + i]);
    B[i] = make_float2(rL[5 + i], rR[5 + i]);
  }
  lower_x2<CURVED>(m, v, vl);
  lower_x2<CURVED>(m, B, Bl);
  const float2 v2 = dot_x2(v, vl), Bv = dot_x2(B, vl), B2 = dot_x2(B, Bl);
  const float2 omv2 = sub2(f2c(1.0f), v2);
  const float2 W = make_float2(rsqrtf(omv2.x), rsqrtf(omv2.y));
  const float2 iW = __fmul2_rn(omv2, W);
  const float2 ab0 = __fmul2_rn(W, Bv);
  const float2 nab0 = neg2(ab0);
  const float2 b2 = __ffma2_rn(B2, omv2, __fmul2_rn(Bv, Bv));
  float2 bl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bl[i] = __ffma2_rn(Bl[i], iW, __fmul2_rn(ab0, vl[i]));
  const float2 hs = __fadd2_rn(__ffma2_rn(f2c(gfac), P, rho), b2);
  const float2 Ps = __ffma2_rn(f2c(0.5f), b2, P);
  const float2 hW2 = __fmul2_rn(__fmul2_rn(hs, W), W);
  const float2 D = __fmul2_rn(rho, W);
  float2 U[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) U[i] = __ffma2_rn(nab0, bl[i], __fmul2_rn(hW2, vl[i]));
  const float2 tau = sub2(__ffma2_rn(nab0, ab0, sub2(hW2, Ps)), D);
  // v^i - beta^i / alpha, the shift term formed once for both sides
  float2 vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) vt[i] = CURVED ? __fadd2_rn(v[i], f2c(-m.beta[i] * ia)) : v[i];
  const float2 vtd = vt[0];
  const float2 nBdiW = neg2(__fmul2_rn(B[0], iW));
  const float2 nB0 = neg2(B[0]);
  float2 F[8];
  F[0] = __fmul2_rn(D, vtd);
  F[1] = __ffma2_rn(nBdiW, bl[0], __ffma2_rn(U[0], vtd, Ps));
  F[2] = __ffma2_rn(nBdiW, bl[1], __fmul2_rn(U[1], vtd));
  F[3] = __ffma2_rn(nBdiW, bl[2], __fmul2_rn(U[2], vtd));
  F[4] = __ffma2_rn(nBdiW, ab0, __ffma2_rn(Ps, v[0], __fmul2_rn(tau, vtd)));
  F[5] = f2c(0.0f);
  F[6] = __ffma2_rn(nB0, vt[1], __fmul2_rn(B[1], vtd));
  F[7] = __ffma2_rn(nB0, vt[2], __fmul2_rn(B[2], vtd));
  const float2 Na = __ffma2_rn(f2c(gamma), P, b2);
  const float2 dsp = __ffma2_rn(neg2(v2), Na, hs);
  const float2 hmn = sub2(hs, Na);
  const float gdd = CURVED ? m.gup_dd : 1.0f;
  float2 Q = __ffma2_rn(f2c(gdd), dsp, __fmul2_rn(__fmul2_rn(neg2(v[0]), v[0]), hmn));
  Q = make_float2(fmaxf(Q.x, 0.0f), fmaxf(Q.y, 0.0f));
  const float2 a = __fmul2_rn(__fmul2_rn(Na, omv2), Q);
  const float2 sq = make_float2(sqrtf(a.x), sqrtf(a.y));
  const float2 c0 = __fmul2_rn(v[0], hmn);
  const float2 lp = __fadd2_rn(c0, sq), lm = sub2(c0, sq);
  L.U[0] = D.x; R.U[0] = D.y;
  L.U[4] = tau.x; R.U[4] = tau.y;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    L.U[1 + i] = U[i].x; R.U[1 + i] = U[i].y;
    L.U[5 + i] = B[i].x; R.U[5 + i] = B[i].y;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) { L.F[q] = F[q].x; R.F[q] = F[q].y; }
  L.lp = lp.x; R.lp = lp.y;
  L.lm = lm.x; R.lm = lm.y;
  L.sden = dsp.x; R.sden = dsp.y;
}

// Speeds of the two sides of a face from their SHARED side states: one
// division for both denominators.
template <class T, bool CURVED, int DIR>
__device__ __forceinline__ void finish_speeds(const Geom<T>& m, Side<T>& L, Side<T>& R) {
  const T alpha = CURVED ? m.alpha : T(1);
  const T bd = CURVED ? m.beta[DIR] : T(0);
  T X;
  if constexpr (sizeof(T) == 8) X = alpha * rcp_nr(L.sden * R.sden);  // fpbits.cuh
  else X = alpha / (L.sden * R.sden);
  const T iL = R.sden * X, iR = L.sden * X;
  L.lp = iL * L.lp - bd;
  L.lm = iL * L.lm - bd;
  R.lp = iR * R.lp - bd;
  R.lm = iR * R.lm - bd;
}

// HLLE flux (Sec. 2.3) from SCALED side states of a face whose normal is the
// first axis: F = sqrt(gamma) [alpha (xp F~L - xm F~R) + xp xm (U~R - U~L)] /
// (xp - xm), the common factors applied once;
// 1e-300 (double) / 1e-30 (float) guards the degenerate fan xi+ = xi- = 0
// with the mean physical flux.
template <class T>
__device__ __forceinline__ void hlle_combine_scaled(const Side<T>& L, const Side<T>& R, T alpha, T sg, T F[8]) {
  T xm, xp;
  if constexpr (sizeof(T) == 8) {
    // FP64: the bounds and the test on the integer pipe (fpbits.cuh)
    xm = dmin0_2i(L.lm, R.lm);
    xp = dmax0_2i(L.lp, R.lp);
  } else {
    xm = xmin(T(0), xmin(L.lm, R.lm));
    xp = xmax(T(0), xmax(L.lp, R.lp));
  }
  const T den = xp - xm;
  const T tiny = sizeof(T) == 8 ? T(1e-300) : T(1e-30);
  bool degenerate;
  if constexpr (sizeof(T) == 8) degenerate = dltposi(den, tiny);
  else degenerate = den < tiny;
  if (degenerate) {
    const T h = T(0.5) * alpha * sg;
#pragma unroll
    for (int q = 0; q < 8; ++q) F[q] = h * (L.F[q] + R.F[q]);
    return;
  }
  T s;
  if constexpr (sizeof(T) == 8) s = sg * rcp_nr(den);  // fpbits.cuh
  else s = sg / den;
  // the factor s taken into the three coefficients once
  const T as = alpha * s;
  const T axp = as * xp, axm = as * xm, xpm = (xp * xm) * s;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q == 5) {
      // the normal field component (the first axis of the rotated frame) has no flux on either side
      F[q] = xpm * (R.U[q] - L.U[q]);
    } else {
      F[q] = fma(axp, L.F[q], fma(-axm, R.F[q], xpm * (R.U[q] - L.U[q])));
    }
  }
}


}  // namespace grmhd
