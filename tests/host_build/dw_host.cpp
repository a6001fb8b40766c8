// Host build of the double-word operations of the pair path (the product's own headers, with
// the stand-in cuda_runtime.h of this folder), mirroring the library's hz_dw_selftest: for each
// i, split a[i] and b[i] and write (hi, lo) of x, y, x + y, x - y, x * y, x / y, sqrt|x|,
// 1/sqrt|x| and the half MC slope of (x, y) to out[(2q) n + i], out[(2q + 1) n + i].
#include "hzn_physics.cuh"

extern "C" void dw_selftest_host(const double* a, const double* b, double* out, long n) {
  using hzn::f32x2;
  for (long i = 0; i < n; ++i) {
    const f32x2 x = hzn::dw::split(a[i]), y = hzn::dw::split(b[i]);
    const f32x2 ax = fabs(x);
    f32x2 r[9];
    r[0] = x;
    r[1] = y;
    r[2] = x + y;
    r[3] = x - y;
    r[4] = x * y;
    r[5] = x / y;
    r[6] = sqrt(ax);
    r[7] = rsqrt(ax);
    r[8] = hzn::mc_half_slope(x, y);
    for (int q = 0; q < 9; ++q) {
      out[(2 * q) * n + i] = (double)r[q].hi;
      out[(2 * q + 1) * n + i] = (double)r[q].lo;
    }
  }
}
