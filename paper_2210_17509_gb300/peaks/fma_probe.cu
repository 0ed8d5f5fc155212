// Arithmetic-peak probe for the roofline denominators of the FP64 and FP32
// pipes: independent FMA chains (8 per thread, 8 CTAs of 256 threads per SM),
// plus FP64 divide / square-root and FP32 divide throughput, and the rate of
// two instruction kinds that share the FP64 pipe with the arithmetic: FP64
// <-> FP32 conversions and FP64 compares.  Every thread writes one value to
// its own slot of an output buffer sized grid x block.
#include <cstdio>
#include <cuda_runtime.h>
template<class T, int CH>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x[CH];
  #pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
  #pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template<class T>
__global__ void div_loop(T* out, int iters, T a) {
  T x = (T)(threadIdx.x + 1), y = (T)(threadIdx.x + 2), z = (T)3, w = (T)5;
  for (int i = 0; i < iters; ++i) { x = a / x + (T)1; y = a / y + (T)1; z = a / z + (T)1; w = a / w + (T)1; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x + y + z + w;
}
template<class T>
__global__ void sqrt_loop(T* out, int iters, T a) {
  T x = (T)(threadIdx.x + 1), y = (T)(threadIdx.x + 2), z = (T)3, w = (T)5;
  for (int i = 0; i < iters; ++i) { x = sqrt(x) + a; y = sqrt(y) + a; z = sqrt(z) + a; w = sqrt(w) + a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x + y + z + w;
}
// FP64 -> FP32 and FP32 -> FP64 conversions, 8 chains per thread; each chain
// returns to its type through integer operations only.
__global__ void cvt_loop(double* out, int iters, double a) {
  double x[8];
  float f[8];
  #pragma unroll
  for (int c = 0; c < 8; ++c) { x[c] = a + threadIdx.x * 1e-3 + c; f[c] = (float)c + 0.5f; }
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float g = (float)x[c];
      x[c] = __hiloint2double(__float_as_int(g) ^ 0x40000000, i);
      const double y = (double)f[c];
      f[c] = __int_as_float((__double2hiint(y) ^ i) & 0x3fffffff);
    }
  }
  double s = 0;
  #pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c] + f[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// FP64 compares feeding integer counters, 8 chains per thread; the compared
// values change through integer operations only.
__global__ void cmp_loop(double* out, int iters, double b) {
  double x[8];
  int n[8];
  #pragma unroll
  for (int c = 0; c < 8; ++c) { x[c] = threadIdx.x * 1e-3 + c; n[c] = 0; }
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int c = 0; c < 8; ++c) {
      n[c] += x[c] > b ? 1 : 0;
      x[c] = __hiloint2double(__double2hiint(x[c]) ^ (n[c] & 1), i);
    }
  }
  int s = 0;
  #pragma unroll
  for (int c = 0; c < 8; ++c) s += n[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  printf("name=%s sms=%d cc=%d.%d l2=%d smem_optin=%zu regs/sm=%d\n", p.name, p.multiProcessorCount, p.major, p.minor, p.l2CacheSize, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  double* d; float* f;
  cudaMalloc(&d, sizeof(double) * blocks * threads);
  cudaMalloc(&f, sizeof(float) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {
    int it64 = 4096;
    fma_loop<double, 8><<<blocks, threads>>>(d, 64, 0.999, 1e-3);
    cudaEventRecord(e0);
    fma_loop<double, 8><<<blocks, threads>>>(d, it64, 0.999, 1e-3);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * (double)it64 * blocks * threads;
    printf("fp64 fma: %.3f ms  %.3f TFLOP/s\n", ms, flops / ms / 1e9);
    int it32 = 65536;
    fma_loop<float, 8><<<blocks, threads>>>(f, 64, 0.999f, 1e-3f);
    cudaEventRecord(e0);
    fma_loop<float, 8><<<blocks, threads>>>(f, it32, 0.999f, 1e-3f);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    flops = 2.0 * 8 * (double)it32 * blocks * threads;
    printf("fp32 fma: %.3f ms  %.3f TFLOP/s\n", ms, flops / ms / 1e9);
    int itd = 256;
    cudaEventRecord(e0);
    div_loop<double><<<blocks, threads>>>(d, itd, 1.5);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 div: %.3f G div/s\n", 4.0 * itd * blocks * threads / ms / 1e6);
    cudaEventRecord(e0);
    sqrt_loop<double><<<blocks, threads>>>(d, itd, 0.5);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 sqrt: %.3f G sqrt/s\n", 4.0 * itd * blocks * threads / ms / 1e6);
    cudaEventRecord(e0);
    div_loop<float><<<blocks, threads>>>(f, itd * 16, 1.5f);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32 div: %.3f G div/s\n", 4.0 * itd * 16 * blocks * threads / ms / 1e6);
    const int itc = 1024;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    const double per_sm_clk = (double)p.multiProcessorCount * clk_khz * 1e3;  // at the maximum SM clock
    cudaEventRecord(e0);
    cvt_loop<<<blocks, threads>>>(d, itc, 0.25);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = 16.0 * itc * blocks * threads;
    printf("fp64<->fp32 convert: %.3f G/s  %.2f per SM per clock\n", ops / ms / 1e6, ops / (ms * 1e-3) / per_sm_clk);
    cudaEventRecord(e0);
    cmp_loop<<<blocks, threads>>>(d, itc, 1e-3);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    ops = 8.0 * itc * blocks * threads;
    printf("fp64 compare: %.3f G/s  %.2f per SM per clock\n", ops / ms / 1e6, ops / (ms * 1e-3) / per_sm_clk);
  }
  cudaError_t err = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
