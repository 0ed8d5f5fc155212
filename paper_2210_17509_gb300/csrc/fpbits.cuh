// FP64 <-> FP32 conversions on the integer pipe.
//
// On this GPU a conversion instruction between FP64 and FP32 occupies the
// FP64 pipe for as long as an FP64 FMA (about two per SM per clock), and the
// mixed recovery, which hands values back and forth between its FP32
// predictor and its FP64 refinement, is bound by that pipe.  These functions
// do the same conversions on the IEEE-754 bit fields with integer
// instructions, about a dozen each on a pipe with 32 times the rate.
//
// Within the normal FP32 range they give the bits of the hardware
// conversions (round to nearest, ties to even, for FP64 -> FP32; exact for
// FP32 -> FP64).  Outside it: an FP32 result below 2^-126 in magnitude
// flushes to a signed zero (the hardware conversion gives a subnormal), an
// FP32 input below 2^-126 converts to a signed zero, overflow gives an
// infinity and a NaN stays a NaN.
#pragma once

#include <stdint.h>

namespace grmhd {

// FP32 bits of x * 2^k rounded to nearest (ties to even), for the FP64 bits
// (hi, lo) of x; k shifts the exponent (0 for a plain conversion) so that a
// value whose FP32 image would underflow can be carried at a scale where it
// does not, at no extra cost.  The arithmetic is on the two 32-bit words: a
// mask of the sign bit of the 64-bit pattern of a computed FP64 value is
// recognised by the compiler as an FP64 absolute value, which takes an FP64
// instruction.
__host__ __device__ __forceinline__ uint32_t f64_words_to_f32_bits(uint32_t hi, uint32_t lo, int k = 0) {
  const uint32_t sign = hi & 0x80000000u, ha = hi & 0x7fffffffu;
  // round the 52-bit fraction to 23 bits at bit 29 (a carry moves into the exponent)
  const uint32_t l = lo + 0x0fffffffu + ((lo >> 29) & 1u);
  const uint32_t h = ha + (l < lo ? 1u : 0u);
  const int eb = (int)(h >> 20);  // biased FP64 exponent of the rounded value
  const int e = eb + k;
  uint32_t f = ((l >> 29) | (h << 3)) - ((uint32_t)(896 - k) << 23);
  if (e < 897) f = 0u;  // below the normal FP32 range (zero included)
  if (e > 1150 || eb >= 2047) f = (ha > 0x7ff00000u || (ha == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  return sign | f;
}
__host__ __device__ __forceinline__ uint32_t f64_bits_to_f32_bits(uint64_t b, int k = 0) {
  return f64_words_to_f32_bits((uint32_t)(b >> 32), (uint32_t)b, k);
}

// FP64 bits (hi, lo) of the FP32 value with bits u (exact).
__host__ __device__ __forceinline__ void f32_bits_to_f64_words(uint32_t u, uint32_t& hi, uint32_t& lo) {
  const uint32_t a = u & 0x7fffffffu;
  hi = (a >> 3) + (896u << 20);
  lo = a << 29;
  if (a < 0x00800000u) hi = lo = 0u;  // zero and subnormals
  if (a >= 0x7f800000u) hi = 0x7ff00000u | ((a >> 3) & 0x000fffffu);
  hi |= u & 0x80000000u;
}
__host__ __device__ __forceinline__ uint64_t f32_bits_to_f64_bits(uint32_t u) {
  uint32_t hi, lo;
  f32_bits_to_f64_words(u, hi, lo);
  return ((uint64_t)hi << 32) | lo;
}

#ifdef __CUDACC__
// The FP64 value is split into, and assembled from, its two words by PTX
// moves, which keep the bit arithmetic out of the compiler's FP64 pattern
// matching.
__device__ __forceinline__ float f64_to_f32i(double x, int k = 0) {
  uint32_t lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
  return __uint_as_float(f64_words_to_f32_bits(hi, lo, k));
}
__device__ __forceinline__ double f32_to_f64i(float x) {
  uint32_t hi, lo;
  f32_bits_to_f64_words(__float_as_uint(x), hi, lo);
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
  return r;
}
// FP64 comparisons and clamps on the integer pipe.  On this GPU an FP64
// compare or min / max also takes an FP64-pipe slot, so the FP64-bound face
// code makes these decisions on the bit patterns; the results are the IEEE
// ones, NaN operands included.
__device__ __forceinline__ void dwords(double x, uint32_t& hi, uint32_t& lo) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}
__device__ __forceinline__ double dfromwords(uint32_t hi, uint32_t lo) {
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
  return r;
}
// x >= +0 and not a NaN (+0 and +inf included; -0 excluded)
__device__ __forceinline__ bool dwords_nonneg(uint32_t hi, uint32_t lo) {
  return hi < 0x7ff00000u || (hi == 0x7ff00000u && lo == 0u);
}
// x > 0 (IEEE)
__device__ __forceinline__ bool dgt0i(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  return dwords_nonneg(hi, lo) && (hi | lo) != 0u;
}
// x < 1 (IEEE)
__device__ __forceinline__ bool dlt1i(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  const uint32_t ha = hi & 0x7fffffffu;
  const bool nan = ha > 0x7ff00000u || (ha == 0x7ff00000u && lo != 0u);
  return hi < 0x3ff00000u || (hi >= 0x80000000u && !nan);
}
// 0 <= x < c for a positive constant c, i.e. x < c for x >= 0 (IEEE)
__device__ __forceinline__ bool dltposi(double x, double c) {
  uint32_t hi, lo, ch, cl;
  dwords(x, hi, lo);
  dwords(c, ch, cl);
  return hi < ch || (hi == ch && lo < cl);
}
// x finite (IEEE)
__device__ __forceinline__ bool dfinitei(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  return (hi & 0x7ff00000u) != 0x7ff00000u;
}
// x >= 1 (IEEE)
__device__ __forceinline__ bool dge1i(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  return dwords_nonneg(hi, lo) && hi >= 0x3ff00000u;
}
// x >= 0 (IEEE: -0 included)
__device__ __forceinline__ bool dge0i(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  return dwords_nonneg(hi, lo) || (hi == 0x80000000u && lo == 0u);
}
// x > c and x >= c (IEEE) for a bound c >= +0 that is not a NaN
__device__ __forceinline__ bool dgtci(double x, double c) {
  uint32_t hi, lo, ch, cl;
  dwords(x, hi, lo);
  dwords(c, ch, cl);
  return dwords_nonneg(hi, lo) && (hi > ch || (hi == ch && lo > cl));
}
__device__ __forceinline__ bool dgeci(double x, double c) {
  uint32_t hi, lo, ch, cl;
  dwords(x, hi, lo);
  dwords(c, ch, cl);
  return (dwords_nonneg(hi, lo) && (hi > ch || (hi == ch && lo >= cl))) ||
         (hi == 0x80000000u && lo == 0u && (ch | cl) == 0u);
}
// |a| <= c (IEEE) for a bound c >= +0 that is not a NaN
__device__ __forceinline__ bool dabsleci(double a, double c) {
  uint32_t hi, lo, ch, cl;
  dwords(a, hi, lo);
  dwords(c, ch, cl);
  hi &= 0x7fffffffu;
  return dwords_nonneg(hi, lo) && (hi < ch || (hi == ch && lo <= cl));
}
// fmax(x, 0) (+0 for x <= 0 or a NaN)
__device__ __forceinline__ double dmax0i(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  const bool keep = dwords_nonneg(hi, lo);
  return dfromwords(keep ? hi : 0u, keep ? lo : 0u);
}
// fmax(0, fmax(a, b)): the bit patterns of non-negative values order like
// the values; a negative value or a NaN counts as +0.
__device__ __forceinline__ double dmax0_2i(double a, double b) {
  uint32_t ha, la, hb, lb;
  dwords(a, ha, la);
  dwords(b, hb, lb);
  if (!dwords_nonneg(ha, la)) ha = la = 0u;
  if (!dwords_nonneg(hb, lb)) hb = lb = 0u;
  const bool tb = hb > ha || (hb == ha && lb > la);
  return dfromwords(tb ? hb : ha, tb ? lb : la);
}
// fmin(0, fmin(a, b)) = -fmax(0, fmax(-a, -b)), +0 when neither is negative
__device__ __forceinline__ double dmin0_2i(double a, double b) {
  uint32_t ha, la, hb, lb;
  dwords(a, ha, la);
  dwords(b, hb, lb);
  ha ^= 0x80000000u;
  hb ^= 0x80000000u;
  if (!dwords_nonneg(ha, la)) ha = la = 0u;
  if (!dwords_nonneg(hb, lb)) hb = lb = 0u;
  const bool tb = hb > ha || (hb == ha && lb > la);
  const uint32_t h = tb ? hb : ha, l = tb ? lb : la;
  return dfromwords((h | l) != 0u ? h ^ 0x80000000u : 0u, l);
}

// FP64 reciprocal and square root for the FP64-pipe-bound kernels, from the
// hardware's 20-bit approximations (PTX rcp.approx.ftz.f64 and
// rsqrt.approx.ftz.f64, no FP64-pipe instructions) and one Newton-Raphson
// step carried to second order: with e = 1 - x r0 the reciprocal is
// r0 / (1 - e) = r0 (1 + e + e^2 + ...), and with e = 1 - x y0^2 the square
// root is x y0 (1 - e)^(-1/2) = x y0 (1 + e/2 + 3 e^2 / 8 + ...).  The
// neglected terms are of order e^3 ~ 2^-60, so the results are within one
// ulp of the exact value (faithful rounding, not always the correctly
// rounded value) for 3 and 5 FP64 operations, against 5 and 8 for the
// correctly rounded library sequences.  Operands outside the range where the
// approximation and the result are normal (zero, subnormals, results that
// would be subnormal, infinities, NaN, negative square-root operands) take
// the library operation.
__device__ __forceinline__ double rcp_nr(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  if (((hi >> 20) & 0x7ffu) - 1u >= 2044u) return 1.0 / x;  // |x| < 2^-1022 or >= 2^1022, inf, NaN
  double r0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(x));
  const double e = fma(-x, r0, 1.0);
  return fma(fma(e, e, e), r0, r0);
}
__device__ __forceinline__ double sqrt_nr(double x) {
  uint32_t hi, lo;
  dwords(x, hi, lo);
  if ((hi >> 20) - 1u >= 2046u) return sqrt(x);  // negative, zero, subnormal, inf, NaN
  double y0;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
  const double t = x * y0;
  const double e = fma(-t, y0, 1.0);
  return fma(t, fma(0.375, e, 0.5) * e, t);
}

// Unbiased exponent of a positive normal FP32 value, and the value with its
// exponent replaced by 0 (its significand in [1, 2)).
__device__ __forceinline__ int f32_exponent(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127; }
__device__ __forceinline__ float f32_significand(float x) {
  return __uint_as_float((__float_as_uint(x) & 0x807fffffu) | 0x3f800000u);
}
#endif

}  // namespace grmhd
