// FP64 operation costs on this GPU, for ncu: one kernel per operation over
// 2^20 operands (each thread one element, i < n), so that the per-element
// thread-instruction counts of each kernel (DADD, DMUL, DFMA, FP64-pipe and
// XU instructions) are the operation's cost.  The operations: the library's
// correctly rounded division, reciprocal and square root, its rsqrt, the PTX
// approximations rcp.approx.ftz.f64 and rsqrt.approx.ftz.f64, and the
// second-order Newton-Raphson reciprocal and square root of csrc/fpbits.cuh.
// Also prints the largest relative error of the two approximations against
// the library values.
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>

#include "../csrc/fpbits.cuh"

using namespace grmhd;

__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_approx(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

#define OP1(name, expr)                                                   \
  __global__ void name(const double* a, double* y, int n) {               \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;                  \
    if (i < n) {                                                          \
      const double x = a[i];                                              \
      y[i] = (expr);                                                      \
    }                                                                     \
  }
OP1(op_reciprocal, 1.0 / x)
OP1(op_sqrt, sqrt(x))
OP1(op_rsqrt, rsqrt(x))
OP1(op_rcp_approx, rcp_approx(x))
OP1(op_rsqrt_approx, rsqrt_approx(x))
OP1(op_rcp_nr, rcp_nr(x))
OP1(op_sqrt_nr, sqrt_nr(x))

__global__ void op_division(const double* a, const double* b, double* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] / b[i];
}

int main() {
  const int n = 1 << 20;
  double* ha = new double[n];
  double* hb = new double[n];
  double* hy = new double[n];
  double* hz = new double[n];
  unsigned long long s = 88172645463325252ull;
  for (int i = 0; i < n; ++i) {  // operands spread over 1e-10 .. 1e10
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    ha[i] = std::pow(10.0, -10.0 + 20.0 * (double)(s >> 11) / 9007199254740992.0);
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    hb[i] = std::pow(10.0, -5.0 + 10.0 * (double)(s >> 11) / 9007199254740992.0);
  }
  double *a, *b, *y, *z;
  if (cudaMalloc(&a, n * 8) || cudaMalloc(&b, n * 8) || cudaMalloc(&y, n * 8) || cudaMalloc(&z, n * 8)) return 2;
  cudaMemcpy(a, ha, n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(b, hb, n * 8, cudaMemcpyHostToDevice);
  const int B = 256, G = n / B;
  op_division<<<G, B>>>(a, b, y, n);
  op_reciprocal<<<G, B>>>(a, y, n);
  op_sqrt<<<G, B>>>(a, y, n);
  op_rsqrt<<<G, B>>>(a, y, n);
  op_rcp_nr<<<G, B>>>(a, y, n);
  op_sqrt_nr<<<G, B>>>(a, y, n);
  double err[2];
  for (int k = 0; k < 2; ++k) {
    if (k == 0) { op_rcp_approx<<<G, B>>>(a, y, n); op_reciprocal<<<G, B>>>(a, z, n); }
    else { op_rsqrt_approx<<<G, B>>>(a, y, n); op_rsqrt<<<G, B>>>(a, z, n); }
    cudaMemcpy(hy, y, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(hz, z, n * 8, cudaMemcpyDeviceToHost);
    err[k] = 0.0;
    for (int i = 0; i < n; ++i) err[k] = std::fmax(err[k], std::fabs(hy[i] - hz[i]) / std::fabs(hz[i]));
  }
  const cudaError_t e = cudaDeviceSynchronize();
  printf("rcp.approx.ftz.f64 max rel err %.3e (2^%.1f), rsqrt.approx.ftz.f64 max rel err %.3e (2^%.1f): %s\n",
         err[0], std::log2(err[0]), err[1], std::log2(err[1]), cudaGetErrorString(e));
  cudaFree(a); cudaFree(b); cudaFree(y); cudaFree(z);
  delete[] ha; delete[] hb; delete[] hy; delete[] hz;
  return e == cudaSuccess ? 0 : 1;
}
