"""Device check of the paired FP32 WENO5 (csrc/physics.cuh: weno5_x2).

The mixed RHS reconstructs two variables per paired FP32 instruction; each
lane must have the bits of the scalar weno5<float> (the same operations in the
same order, negated operands moved into constants).  This test compiles a
small CUDA program against the header and compares the two on random
stencils of mixed scales and signs, on smooth and on jumping data, both
states of a face (the mirrored stencil too).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_17509_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

CHECK = r"""
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "physics.cuh"
using namespace grmhd;

__device__ __host__ inline uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ float val(uint64_t i, int k) {
  const uint64_t b = mix(i * 16 + k);
  const float u = (float)(b >> 40) * 0x1p-24f;  // [0, 1)
  switch (i % 4) {
    case 0: return 1.0f + 0.1f * u;                                   // smooth, positive
    case 1: return (b & 1) ? -u : u;                                  // both signs
    case 2: return (k < 3 ? 1.0f : 0.125f) + 1e-3f * u;               // a jump
    default: return ldexpf(1.0f + u, (int)((b >> 8) % 40) - 20);      // scales 1e-6 .. 1e6
  }
}
__global__ void check(long long n, unsigned long long* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float a[6], b[6];
    for (int k = 0; k < 6; ++k) { a[k] = val(2 * i, k); b[k] = val(2 * i + 1, k); }
    const float eps = 1e-6f;
    const float2 e2 = make_float2(eps, eps);
    // left state of a face from u[0..4], right state from the mirrored u[5..1]
    const float2 vL = weno5_x2(make_float2(a[0], b[0]), make_float2(a[1], b[1]), make_float2(a[2], b[2]),
                               make_float2(a[3], b[3]), make_float2(a[4], b[4]), e2);
    const float2 vR = weno5_x2(make_float2(a[5], b[5]), make_float2(a[4], b[4]), make_float2(a[3], b[3]),
                               make_float2(a[2], b[2]), make_float2(a[1], b[1]), e2);
    const float sL0 = weno5<float>(a[0], a[1], a[2], a[3], a[4], eps), sL1 = weno5<float>(b[0], b[1], b[2], b[3], b[4], eps);
    const float sR0 = weno5<float>(a[5], a[4], a[3], a[2], a[1], eps), sR1 = weno5<float>(b[5], b[4], b[3], b[2], b[1], eps);
    const bool same = __float_as_uint(vL.x) == __float_as_uint(sL0) && __float_as_uint(vL.y) == __float_as_uint(sL1) &&
                      __float_as_uint(vR.x) == __float_as_uint(sR0) && __float_as_uint(vR.y) == __float_as_uint(sR1);
    if (!same) atomicAdd(bad, 1ull);
  }
}
int main() {
  const long long n = 1ll << 22;
  unsigned long long* bad;
  if (cudaMalloc(&bad, sizeof(unsigned long long)) != cudaSuccess) return 2;
  cudaMemset(bad, 0, sizeof(unsigned long long));
  check<<<152 * 8, 256>>>(n, bad);
  unsigned long long h = 0;
  cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  printf("%lld %llu %s\n", n, h, cudaGetErrorString(e));
  cudaFree(bad);
  return e == cudaSuccess ? 0 : 1;
}
"""


@pytest.mark.gpu
def test_paired_fp32_weno5_has_the_bits_of_the_scalar_form(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, "-I",
                    INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split()
    assert out[2] == "no", out
    assert int(out[0]) == 1 << 22
    assert int(out[1]) == 0, "weno5_x2 differs from weno5<float> in some lane"
