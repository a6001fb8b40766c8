// hzn_ctx.h -- host-side grid context and workspace layout, shared by the C-ABI translation
// units (hzn_api.cu: the forward update; hzn_adjoint.cu: the reverse sweep).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "hzn.h"
#include "hzn_internal.h"

struct hz_ctx {
  hz_grid g;
  hz_options o;
  cudaStream_t st;
  hzn::KParams kp;
  hzn::Variant v;
  char* ws;
  size_t wsbytes;
  hzn::DevScalars* sc;
  void* met;
  double* U0;
  double* U1;
  void* P[2];
  int cur;
  int have_metric, have_prim;
  int zchunks;
};

namespace hzn {

// Workspace layout of one grid: device scalars, metric, two conserved and two primitive
// arrays, and the geometry tables of a DIAG metric (metric layout, FP64).  Grid functions are
// padded: rows of `pitch` elements, fields `fs` elements apart.
struct Layout {
  size_t scal, met, u_bytes, p_bytes, geo, total;
  long long fs, ms;
  int pitch, mpitch, mny;
  long long plane, mplane;
};

Layout layout_of(const hz_grid* g, const hz_options* o);
int check_args(const hz_grid* g, const hz_options* o);
int grid_blocks(long long n, int threads);
int cuda_err(cudaError_t e);

// Caller layout (unpadded, field-major) <-> padded workspace layout.
void launch_pack_in(hz_ctx* c, const double* src, void* dst);
void launch_pack_out(hz_ctx* c, const void* src, bool is_double, double* dst);

// Device clock: mode 0 sets the fixed step dt, mode 1 takes dt = cfl / max speed.
void launch_clock(hz_ctx* c, int mode, double dt, double cfl, double t_end);

// The three substeps of one RK3 step, Pin -> P1 -> P2 -> Pout, conserved state in c->U0/U1.
void launch_rk3(hz_ctx* c, const void* Pin, void* P1, void* P2, void* Pout);

}  // namespace hzn
