// alu_peak.cu -- measured FP64 and FP32 fused-multiply-add throughput of the current GPU.
// The FP64-ALU roofline of the finite-volume kernels is taken against this number: each thread
// runs independent in-register FMA chains, so the kernel is bound by the FMA pipes alone.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T, int CH>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T, int CH>
double tflops(int blocks, int threads, int iters) {
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_chains<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  fma_chains<T, CH><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 2.0 * CH * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
}

int main() {
  int dev = 0;
  cudaDeviceProp p;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&p, dev);
  printf("device %s, %d SMs\n", p.name, p.multiProcessorCount);
  const int sms = p.multiProcessorCount;
  for (int bpm : {1, 2, 4, 8}) printf("fp64 %d blocks/SM x 256 threads: %.3f TFLOP/s\n", bpm, tflops<double, 8>(sms * bpm, 256, 4096));
  for (int bpm : {2, 4, 8}) printf("fp32 %d blocks/SM x 256 threads: %.3f TFLOP/s\n", bpm, tflops<float, 8>(sms * bpm, 256, 65536));
  const cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
