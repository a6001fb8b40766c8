// Self-test entries (see hzn.h): the double-word arithmetic used by the HZ_FP64_DW kernels (the
// same split, operations and half MC slope, applied to caller-given doubles), and the FP64
// reciprocal of the FP64 kernels (rcp_fast).
#include <cuda_runtime.h>

#include "hzn.h"
#include "hzn_kernels.cuh"

namespace {

using hzn::f32x2;

__global__ void k_dw_selftest(const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const f32x2 x = hzn::dw::split(a[i]), y = hzn::dw::split(b[i]);
    const f32x2 ax = fabs(x);
    f32x2 r[HZ_DW_NRESULTS];
    r[0] = x;
    r[1] = y;
    r[2] = x + y;
    r[3] = x - y;
    r[4] = x * y;
    r[5] = x / y;
    r[6] = sqrt(ax);
    r[7] = rsqrt(ax);
    r[8] = hzn::mc_half_slope(x, y);
#pragma unroll
    for (int q = 0; q < HZ_DW_NRESULTS; ++q) {
      out[(2 * q) * n + i] = (double)r[q].hi;
      out[(2 * q + 1) * n + i] = (double)r[q].lo;
    }
  }
}

__global__ void k_rcp_selftest(const double* __restrict__ x, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = hzn::rcp_fast(x[i]);
}

int blocks_of(long long n, int threads) {
  const long long want = (n + threads - 1) / threads;
  return (int)(want < 4096 ? want : 4096);
}

}  // namespace

extern "C" int hz_rcp_selftest(const double* d_x, double* d_out, long long n, void* stream) {
  if (!d_x || !d_out || n < 0) return HZ_ERR_ARG;
  if (n == 0) return HZ_OK;
  k_rcp_selftest<<<blocks_of(n, 256), 256, 0, (cudaStream_t)stream>>>(d_x, d_out, n);
  return hzn::record_cuda_error(cudaGetLastError());
}

extern "C" int hz_dw_selftest(const double* d_a, const double* d_b, double* d_out, long long n,
                              void* stream) {
  if (!d_a || !d_b || !d_out || n < 0) return HZ_ERR_ARG;
  if (n == 0) return HZ_OK;
  const int threads = 256;
  const long long want = (n + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  k_dw_selftest<<<blocks, threads, 0, (cudaStream_t)stream>>>(d_a, d_b, d_out, n);
  return hzn::record_cuda_error(cudaGetLastError());
}
