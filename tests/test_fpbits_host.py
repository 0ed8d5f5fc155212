"""Host check of the integer-pipe FP64 <-> FP32 conversions (csrc/fpbits.cuh).

The mixed recovery converts between its FP32 predictor and its FP64
refinement with integer arithmetic on the IEEE-754 bit fields instead of the
conversion instructions, which occupy the FP64 pipe.  The bit functions are
plain C++, so this test compiles them on the host with g++ and compares them
with the host's own IEEE conversions (round to nearest, ties to even):
- FP64 -> FP32 on random bit patterns, on values spread over the FP32
  exponent range, on exact ties and on values that round up into the next
  binade, with and without an exponent shift k (the result must be the
  conversion of x * 2^k), where the FP32 result is normal, zero, infinite or
  NaN; results in the subnormal FP32 range must flush to zero (or round up to
  the smallest normal);
- FP32 -> FP64 on every 61st bit pattern plus the special values: exact,
  subnormal inputs to signed zero.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2210_17509_gb300", "csrc", "fpbits.cuh")

CHECK = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include "fpbits.cuh"
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
using namespace grmhd;
static uint64_t db(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
static uint32_t fb(float x) { uint32_t b; memcpy(&b, &x, 4); return b; }
static float bf(uint32_t b) { float x; memcpy(&x, &b, 4); return x; }
static double bd(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
int main() {
  std::mt19937_64 rng(7);
  long bad = 0, n = 0;
  auto chk = [&](double x, int k) {
    const float ref = (float)std::ldexp(x, k);
    const uint32_t got = f64_bits_to_f32_bits(db(x), k);
    ++n;
    if (std::isnan(ref)) { bad += !std::isnan(bf(got)); return; }
    if (ref != 0.0f && std::fabs(ref) < FLT_MIN) {
      bad += !((got & 0x7fffffffu) == 0u || std::fabs(bf(got)) == FLT_MIN);
      return;
    }
    if (got != fb(ref)) {
      if (bad < 5) printf("f64->f32 mismatch x=%a k=%d ref=%a got=%a\n", x, k, ref, bf(got));
      ++bad;
    }
  };
  for (long i = 0; i < 2000000; ++i) {
    const uint64_t b = rng();
    double x;
    switch (i % 4) {
      case 0: x = bd(b); break;
      case 1: x = std::ldexp(1.0 + (double)(b >> 12) / 4503599627370496.0, (int)(rng() % 300) - 150);
              if (b & 1) x = -x; break;
      case 2: x = bd((b & ~0x1fffffffull) | 0x10000000ull); break;   // exact ties
      default: x = bd(b | 0x1fffffffull); break;                      // round up into the next value
    }
    int k = (i % 7 == 0) ? (int)(rng() % 61) - 30 : 0;
    if (!std::isfinite(x) || std::fabs(std::ldexp(x, k)) > 1e300 || (x != 0 && std::fabs(std::ldexp(x, k)) < 1e-300))
      k = 0;
    chk(x, k);
  }
  const double sp[] = {0.0, -0.0, 1.0, -1.0, FLT_MAX, -FLT_MAX, 3.4028235677973366e38, 3.4028235677973362e38,
                       FLT_MIN, -FLT_MIN, (double)FLT_MIN * (1 - 1e-9), INFINITY, -INFINITY, NAN, DBL_MAX, DBL_MIN,
                       5e-324, 0.1, 1.0 / 3.0};
  for (double x : sp) chk(x, 0);
  long bad2 = 0;
  auto chk2 = [&](uint32_t u) {
    const float f = bf(u);
    const uint64_t got = f32_bits_to_f64_bits(u);
    if (std::isnan(f)) { bad2 += !std::isnan(bd(got)); return; }
    if (f != 0.0f && std::fabs(f) < FLT_MIN) { bad2 += (got & 0x7fffffffffffffffull) != 0u; return; }
    if (got != db((double)f)) ++bad2;
  };
  for (uint64_t u = 0; u <= 0xffffffffull; u += 61) chk2((uint32_t)u);
  const uint32_t sp2[] = {0u, 0x80000000u, 0x00800000u, 0x80800000u, 0x007fffffu, 0x7f7fffffu, 0x7f800000u,
                          0xff800000u, 0x7fc00000u, 0x3f800000u, 0xffffffffu};
  for (uint32_t u : sp2) chk2(u);
  printf("%ld %ld %ld\n", n, bad, bad2);
  return 0;
}
"""


def test_integer_pipe_conversions_match_ieee(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    n, bad, bad2 = (int(v) for v in out.split()[-3:])
    assert n > 2000000
    assert bad == 0, out
    assert bad2 == 0, out


def test_planted_rounding_error_is_caught(tmp_path):
    # the check must fail on a conversion that truncates instead of rounding
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    hdr = open(HEADER).read()
    planted = hdr.replace("lo + 0x0fffffffu + ((lo >> 29) & 1u)", "lo")
    assert planted != hdr
    (tmp_path / "fpbits.cuh").write_text(planted)
    src = tmp_path / "check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", str(tmp_path), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert int(out.split()[-2]) > 0
