// Arithmetic-peak probe for the roofline denominators of the FP64 and FP32
// pipes: independent FMA chains (8 per thread, 8 CTAs of 256 threads per SM),
// plus FP64 divide / square-root and FP32 divide throughput.  Every thread
// writes one value to its own slot of an output buffer sized grid x block.
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
  }
  cudaError_t err = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
