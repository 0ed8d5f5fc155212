"""Device check of the FP64 helpers of csrc/fpbits.cuh against the GPU's own
operations.

The FP64-pipe-bound kernels make their FP64 <-> FP32 conversions, FP64
comparisons and clamps with integer instructions on the bit patterns, and the
face code takes its reciprocals and square roots from the hardware
approximations plus a second-order Newton-Raphson step.  This test compiles a
small CUDA program against the same header, runs it on random and special
operands, and compares:
- the conversions bit for bit with the conversion instructions (normal FP32
  range; subnormal FP32 results must flush to zero),
- the comparisons and clamps with the IEEE operations (NaN, signed zeros and
  infinities included),
- rcp_nr and sqrt_nr with the correctly rounded 1.0 / x and sqrt(x): at most
  one ulp apart, and the library value itself outside the fast range.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_17509_gb300", "csrc")

CHECK = r"""
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "fpbits.cuh"
using namespace grmhd;

// counter-based operand generator (splitmix64)
__device__ __host__ inline uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ double operand(uint64_t i, int kind) {
  const uint64_t b = mix(i * 4 + kind);
  const double specials[12] = {0.0, -0.0, 1.0, -1.0, __longlong_as_double(0x7ff0000000000000ll),
                               __longlong_as_double((long long)0xfff0000000000000ull),
                               __longlong_as_double(0x7ff8000000000000ll),
                               __longlong_as_double((long long)0xfff8000000000000ull), 4.9e-324, 2.2250738585072014e-308,
                               1.7976931348623157e308, 1e-300};
  switch (i % 5) {
    case 0: return specials[(b >> 7) % 12];
    case 1: return __longlong_as_double((long long)b);  // any bit pattern
    case 2: {  // moderate magnitudes of both signs
      const double m = 1.0 + (double)(b >> 12) * 0x1p-52;
      const int e = (int)((b >> 2) % 120) - 60;
      return (b & 1) ? -ldexp(m, e) : ldexp(m, e);
    }
    case 3: {  // around 1 and 0
      const double m = (double)(b >> 11) * 0x1p-53;
      return (b & 1) ? 1.0 - m * 1e-6 : (b & 2 ? m * 1e-6 : 1.0 + m * 1e-6);
    }
    default: {  // wide positive range
      const double m = 1.0 + (double)(b >> 12) * 0x1p-52;
      return ldexp(m, (int)((b >> 2) % 2040) - 1020);
    }
  }
}
__device__ bool same(double a, double b) {
  return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}
// bad[0]: f64->f32  [1]: f32->f64  [2]: comparisons  [3]: clamps
//    [4]: rcp_nr > 1 ulp  [5]: sqrt_nr > 1 ulp  [6]: fast-path values counted
__global__ void check(long long n, unsigned long long* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = operand(i, 0), y = operand(i, 1);
    // conversions
    const float hf = (float)x, mf = f64_to_f32i(x);
    const bool sub = hf != 0.0f && fabsf(hf) < 1.17549435e-38f;
    if (sub ? !(mf == 0.0f || fabsf(mf) == 1.17549435e-38f)
            : !((hf != hf && mf != mf) || __float_as_uint(hf) == __float_as_uint(mf)))
      atomicAdd(bad + 0, 1ull);
    const float xf = __uint_as_float((uint32_t)mix(i * 7 + 3));
    const double hd = (double)xf, md = f32_to_f64i(xf);
    const bool fsub = xf != 0.0f && fabsf(xf) < 1.17549435e-38f;
    if (fsub ? md != 0.0 : !same(hd, md)) atomicAdd(bad + 1, 1ull);
    // comparisons (bounds c >= +0 where the helper asks for one)
    const double c = fabs(y) == fabs(y) ? fabs(y) : 0.5;
    int wrong = 0;
    wrong += dgt0i(x) != (x > 0.0);
    wrong += dlt1i(x) != (x < 1.0);
    wrong += dge1i(x) != (x >= 1.0);
    wrong += dge0i(x) != (x >= 0.0);
    wrong += dfinitei(x) != (bool)isfinite(x);
    wrong += dgtci(x, c) != (x > c);
    wrong += dgeci(x, c) != (x >= c);
    wrong += dabsleci(x, c) != (fabs(x) <= c);
    if (c == c && c >= 0.0) wrong += dltposi(fabs(x), c) != (fabs(x) < c);
    if (wrong) atomicAdd(bad + 2, 1ull);
    // clamps
    int wc = 0;
    wc += !same(dmax0i(x), fmax(x, 0.0) == 0.0 ? 0.0 : fmax(x, 0.0));
    const double mx = fmax(0.0, fmax(x, y)), mn = fmin(0.0, fmin(x, y));
    wc += !same(dmax0_2i(x, y), mx == 0.0 ? 0.0 : mx);
    wc += !(dmin0_2i(x, y) == mn || (dmin0_2i(x, y) == 0.0 && mn == 0.0));
    if (wc) atomicAdd(bad + 3, 1ull);
    // reciprocal and square root: within one ulp of the correctly rounded value
    const double r = rcp_nr(x), rr = 1.0 / x;
    if (!same(r, rr)) {
      const long long d = __double_as_longlong(r) - __double_as_longlong(rr);
      if (d > 1 || d < -1 || (r != r) != (rr != rr)) atomicAdd(bad + 4, 1ull);
    }
    const double s = sqrt_nr(x), sr = sqrt(x);
    if (!same(s, sr)) {
      const long long d = __double_as_longlong(s) - __double_as_longlong(sr);
      if (d > 1 || d < -1 || (s != s) != (sr != sr)) atomicAdd(bad + 5, 1ull);
    }
    if (x > 0.0 && x < 1e300 && x > 1e-300) atomicAdd(bad + 6, 1ull);
  }
}
int main() {
  const long long n = 1ll << 24;
  unsigned long long* bad;
  if (cudaMalloc(&bad, 8 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  cudaMemset(bad, 0, 8 * sizeof(unsigned long long));
  check<<<152 * 8, 256>>>(n, bad);
  unsigned long long h[8];
  cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  printf("%lld %llu %llu %llu %llu %llu %llu %llu %s\n", n, h[0], h[1], h[2], h[3], h[4], h[5], h[6],
         cudaGetErrorString(e));
  cudaFree(bad);
  return e == cudaSuccess ? 0 : 1;
}
"""


@pytest.mark.gpu
def test_fpbits_helpers_match_the_gpu_operations(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split()
    n, conv64, conv32, cmp_, clamp, rcp, sq, fast = (int(v) for v in out[:8])
    assert out[8] == "no", out
    assert n == 1 << 24 and fast > n // 5
    assert conv64 == 0, "f64_to_f32i differs from the conversion instruction"
    assert conv32 == 0, "f32_to_f64i differs from the conversion instruction"
    assert cmp_ == 0, "an integer-pipe comparison differs from the IEEE one"
    assert clamp == 0, "an integer-pipe clamp differs from fmax / fmin"
    assert rcp == 0, "rcp_nr more than one ulp from 1.0 / x"
    assert sq == 0, "sqrt_nr more than one ulp from sqrt(x)"
