// alu_peak.cu -- measured arithmetic throughput of the current GPU: FP64 and FP32 fused
// multiply-add (the FP64-ALU roofline of the finite-volume kernels is taken against the FP64
// number), FP64 add and multiply, conversions between FP32 and FP64, and the double-word
// (float-float) multiply-add of hzn_f32x2.cuh.  Each thread runs independent in-register
// chains, so every kernel is bound by the pipe under test alone.
#include <cstdio>
#include <cuda_runtime.h>

#include "../csrc/hzn_f32x2.cuh"

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

// Chains of one operation kind; OP 0: FP64 add, 1: FP64 multiply, 2: double -> float,
// 3: float -> double, 4: double-word multiply-add.  Returns operations per second.
template <int OP, int CH>
__global__ void op_chains(double* out, int iters) {
  double d[CH];
  float f[CH];
  hzn::f32x2 w[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    d[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    f[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    w[c] = hzn::f32x2(f[c], 1e-9f * c);
  }
  const double da = 0.999999, db = 1e-7;
  const hzn::f32x2 wa(0.999999), wb(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (OP == 0) d[c] = d[c] + db;
      if (OP == 1) d[c] = d[c] * da;
      if (OP == 2) {
        // the converted value feeds the next iteration through integer operations only
        const float t = __double2float_rn(d[c]);
        d[c] = __longlong_as_double(__double_as_longlong(d[c]) ^ (long long)(__float_as_int(t) & 1));
      }
      if (OP == 3) {
        const double t = (double)f[c];
        f[c] = __int_as_float(__float_as_int(f[c]) ^ (int)((__double_as_longlong(t) >> 29) & 1));
      }
      if (OP == 4) w[c] = w[c] * wa + wb;
    }
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += d[c] + (double)f[c] + (double)w[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP, int CH>
double ops_per_s(int blocks, int threads, int iters) {
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) op_chains<OP, CH><<<blocks, threads>>>(out, iters);
  cudaEventRecord(e0);
  op_chains<OP, CH><<<blocks, threads>>>(out, iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)CH * iters * blocks * threads / (ms * 1e-3);
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
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  const double per_clk = 1.0 / ((double)sms * khz * 1e3);
  printf("nominal SM clock %.0f MHz; rates below in operations per second and per SM per clock\n", khz * 1e-3);
  for (int bpm : {2, 8}) {
    double r;
    r = ops_per_s<0, 8>(sms * bpm, 256, 4096);
    printf("fp64 add        %d blocks/SM: %.3e /s  %.2f /SM/clk\n", bpm, r, r * per_clk);
    r = ops_per_s<1, 8>(sms * bpm, 256, 4096);
    printf("fp64 mul        %d blocks/SM: %.3e /s  %.2f /SM/clk\n", bpm, r, r * per_clk);
    r = ops_per_s<2, 8>(sms * bpm, 256, 4096);
    printf("cvt f64->f32    %d blocks/SM: %.3e /s  %.2f /SM/clk\n", bpm, r, r * per_clk);
    r = ops_per_s<3, 8>(sms * bpm, 256, 4096);
    printf("cvt f32->f64    %d blocks/SM: %.3e /s  %.2f /SM/clk\n", bpm, r, r * per_clk);
    r = ops_per_s<4, 8>(sms * bpm, 256, 16384);
    printf("f32x2 mul+add   %d blocks/SM: %.3e /s  %.2f /SM/clk (one multiply and one add each)\n", bpm, r, r * per_clk);
  }
  {
    // the substep kernel's occupancy: 2 blocks of 128 threads per SM
    const double r = ops_per_s<4, 4>(sms * 2, 128, 16384);
    printf("f32x2 mul+add   2 blocks/SM x 128 threads, 4 chains: %.3e /s  %.2f /SM/clk\n", r, r * per_clk);
  }
  const cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
