// hzn_api.cu -- the C-ABI of libhzn (include/hzn.h): context, workspace layout, copies in and
// out, the time-step clock, and the launch sequence of one RK3 step (three fused substeps,
// §3.2).  The numerical kernels live in hzn_kernels.cuh (instantiated in hzn_k*.cu).

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "hzn.h"
#include "hzn_ctx.h"
#include "hzn_internal.h"

using namespace hzn;

namespace {

constexpr int NF = 9;  // fields of the primitive and conserved vectors

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Caller layout (unpadded, field-major) <-> workspace layout (padded rows), with conversion
// to the storage precision S of the primitive state.
template <typename S>
__global__ void k_pack_in(const KParams kp, const double* __restrict__ src, S* __restrict__ dst,
                          int nfield, int zero_from) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * nfield;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / n);
    const long long r = q % n;
    const int i = (int)(r % kp.nx);
    const int j = (int)((r / kp.nx) % kp.ny);
    const int k = (int)(r / ((long long)kp.nx * kp.ny));
    dst[f * kp.fs + (long long)k * kp.plane + (long long)j * kp.pitch + i] = f >= zero_from ? S(0) : (S)src[q];
  }
}

template <typename S>
__global__ void k_pack_out(const KParams kp, const S* __restrict__ src, double* __restrict__ dst,
                           int nfield, int zero_from) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * nfield;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / n);
    const long long r = q % n;
    const int i = (int)(r % kp.nx);
    const int j = (int)((r / kp.nx) % kp.ny);
    const int k = (int)(r / ((long long)kp.nx * kp.ny));
    dst[q] = f >= zero_from ? 0.0 : (double)src[f * kp.fs + (long long)k * kp.plane + (long long)j * kp.pitch + i];
  }
}

// Metric copy into the padded layout; flags a nonzero shift or off-diagonal gamma_ij.
template <typename S>
__global__ void k_pack_metric(const KParams kp, const double* __restrict__ src, S* __restrict__ dst,
                              DevScalars* sc) {
  const int mx = kp.nx + 2 * kp.gx, my = kp.ny + 2 * kp.gy, mz = kp.nz + 2 * kp.gz;
  const long long n = (long long)mx * my * mz;
  unsigned int general = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * 10;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / n);
    const long long r = q % n;
    const int i = (int)(r % mx);
    const int j = (int)((r / mx) % my);
    const int k = (int)(r / ((long long)mx * my));
    const double v = src[q];
    dst[f * kp.ms + (long long)k * kp.mplane + (long long)j * kp.mpitch + i] = (S)v;
    const bool offdiag = f == 1 || f == 2 || f == 3 || f == 5 || f == 6 || f == 8;
    if (offdiag && v != 0.0) general = 1;
  }
  if (__any_sync(0xffffffffu, general) && (threadIdx.x & 31) == 0) atomicOr(&sc->metric_general, 1u);
}

// Time-step clock: one thread.  mode 0: fixed dt; mode 1: dt = cfl / vmax clipped to t_end.
__global__ void k_clock(DevScalars* sc, int mode, double dt_in, double cfl, double t_end) {
  double dt = dt_in;
  if (mode == 1) {
    const double vmax = __longlong_as_double((long long)sc->vmax_bits);
    dt = vmax > 0.0 ? cfl / vmax : t_end - sc->t;
    if (sc->t + dt > t_end) dt = t_end - sc->t;
    if (dt < 0.0) dt = 0.0;
  }
  sc->dt = dt;
  sc->t += dt;
  sc->steps += 1;
  sc->vmax_bits = 0ull;
}

__global__ void k_reset_scalars(DevScalars* sc) {
  sc->vmax_bits = 0ull;
  sc->fails = 0ull;
  sc->maxit = 0;
  sc->dt = 0.0;
  sc->t = 0.0;
  sc->steps = 0;
}

__global__ void k_reset_vmax(DevScalars* sc) { sc->vmax_bits = 0ull; }

}  // namespace

namespace hzn {

int grid_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

static thread_local int t_last_cuda_error = 0;  // per host thread (hz_last_cuda_error)

int record_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return HZ_OK;
  t_last_cuda_error = (int)e;
  return HZ_ERR_CUDA;
}

int cuda_err(cudaError_t e) { return record_cuda_error(e); }

Layout layout_of(const hz_grid* g, const hz_options* o) {
  Layout L;
  const size_t es = o->precision == HZ_MIXED ? sizeof(float) : sizeof(double);
  const int gx = g->n[0] > 1, gy = g->n[1] > 1, gz = g->n[2] > 1;
  L.pitch = (int)round_up((size_t)g->n[0], 16);
  L.plane = (long long)L.pitch * g->n[1];
  L.fs = (long long)round_up((size_t)(L.plane * g->n[2]), 64);
  L.mpitch = (int)round_up((size_t)(g->n[0] + 2 * gx), 16);
  L.mny = g->n[1] + 2 * gy;
  L.mplane = (long long)L.mpitch * L.mny;
  L.ms = (long long)round_up((size_t)(L.mplane * (g->n[2] + 2 * gz)), 64);
  L.scal = 256;
  L.met = round_up((size_t)L.ms * 10 * es, 256);
  L.u_bytes = (size_t)L.fs * NF * sizeof(double);
  L.p_bytes = round_up((size_t)L.fs * NF * es, 256);
  // geometry tables of a DIAG metric: centre geometry; in FP64 also face geometry and source
  // differences per active axis
  const int ndims = gx + gy + gz;
  const int ngeo = o->precision == HZ_MIXED ? GEO_C : GEO_C + ndims * (GEO_F + GEO_S);
  L.geo = round_up((size_t)L.ms * ngeo * sizeof(double), 256);
  L.total = L.scal + L.met + 2 * L.u_bytes + 2 * L.p_bytes + L.geo;  // U0, U1, P[0], P[1], tables
  return L;
}

int check_args(const hz_grid* g, const hz_options* o) {
  if (!g || !o) return HZ_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 1 || g->n[d] > (1 << 20)) return HZ_ERR_ARG;
    if (g->bc[d] != HZ_BC_OUTFLOW && g->bc[d] != HZ_BC_PERIODIC) return HZ_ERR_ARG;
    if (!(g->dx[d] > 0.0)) return HZ_ERR_ARG;
  }
  // x is always active; inactive axes come last (x, then y, then z)
  if (g->n[0] < 2) return HZ_ERR_UNSUPPORTED;
  if (g->n[1] == 1 && g->n[2] > 1) return HZ_ERR_UNSUPPORTED;
  if ((long long)g->n[0] * g->n[1] * g->n[2] > (1LL << 31)) return HZ_ERR_ARG;
  if (!(o->gamma > 1.0) || o->gamma > 3.0) return HZ_ERR_ARG;
  if (o->precision != HZ_FP64 && o->precision != HZ_MIXED && o->precision != HZ_FP64_DW)
    return HZ_ERR_ARG;
  if (o->precision == HZ_FP64_DW && o->recon != HZ_RECON_MC) return HZ_ERR_UNSUPPORTED;
  if (o->cleaning != 0 && o->cleaning != 1) return HZ_ERR_ARG;
  if (o->cleaning && (!(o->ch > 0.0) || o->ch > 1.0 || !(o->kappa >= 0.0))) return HZ_ERR_ARG;
  if (!(o->rho_floor > 0.0) || !(o->p_floor > 0.0) || !(o->atm_K >= 0.0)) return HZ_ERR_ARG;
  if (!(o->rho_atm >= 0.0)) return HZ_ERR_ARG;
  if (o->c2p_maxit < 1 || o->c2p_maxit > 200) return HZ_ERR_ARG;
  if (!(o->c2p_tol >= 1e-15) || o->c2p_tol > 1e-6) return HZ_ERR_ARG;
  if (o->recon != HZ_RECON_MC && o->recon != HZ_RECON_PPM) return HZ_ERR_ARG;
  if (o->c2p != HZ_C2P_2D && o->c2p != HZ_C2P_1D) return HZ_ERR_ARG;
  // PPM reads three cells on each side: an active axis needs at least three cells
  if (o->recon == HZ_RECON_PPM)
    for (int d = 0; d < 3; ++d)
      if (g->n[d] > 1 && g->n[d] < 3) return HZ_ERR_UNSUPPORTED;
  return HZ_OK;
}

void launch_pack_in(hz_ctx* c, const double* src, void* dst) {
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  const int zero_from = c->o.cleaning ? NF : 8;
  if (c->v.mixed)
    k_pack_in<float><<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, src, (float*)dst, NF, zero_from);
  else
    k_pack_in<double><<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, src, (double*)dst, NF, zero_from);
}

void launch_pack_out(hz_ctx* c, const void* src, bool is_double, double* dst) {
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  const int zero_from = c->o.cleaning ? NF : 8;
  if (is_double)
    k_pack_out<double><<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, (const double*)src, dst, NF, zero_from);
  else
    k_pack_out<float><<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, (const float*)src, dst, NF, zero_from);
}

void launch_clock(hz_ctx* c, int mode, double dt, double cfl, double t_end) {
  k_clock<<<1, 1, 0, c->st>>>(c->sc, mode, dt, cfl, t_end);
}

// The three substeps of one RK3 step with explicit primitive buffers Pin -> P1 -> P2 -> Pout
// (Pin may equal P2, P1 may equal Pout); the conserved state lives in c->U0 / c->U1 and the
// step size in the device clock.
void launch_rk3(hz_ctx* c, const void* Pin, void* P1, void* P2, void* Pout) {
  // Shu-Osher RK3: U1 = U0 + dt L(U0); U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)); U3 = 1/3 U0 + 2/3 (U2 + dt L(U2))
  const StageArgs s1 = {Pin, P1, c->U0, c->U0, c->U1, 0.0, 1.0, 0};
  const StageArgs s2 = {P1, P2, c->U0, c->U1, c->U1, 0.75, 0.25, 0};
  const StageArgs s3 = {P2, Pout, c->U0, c->U1, c->U0, 1.0 / 3.0, 2.0 / 3.0, 1};
  launch_substep(c->v, c->kp, s1, c->met, c->sc, c->zchunks, c->st);
  launch_substep(c->v, c->kp, s2, c->met, c->sc, c->zchunks, c->st);
  launch_substep(c->v, c->kp, s3, c->met, c->sc, c->zchunks, c->st);
}

int run_step(hz_ctx* c, int mode, double dt, double cfl, double t_end) {
  if (!c->have_metric || !c->have_prim) return HZ_ERR_STATE;
  launch_clock(c, mode, dt, cfl, t_end);
  const int a = c->cur, b = 1 - c->cur;
  launch_rk3(c, c->P[a], c->P[b], c->P[a], c->P[b]);
  c->cur = b;
  return cuda_err(cudaGetLastError());
}

// Fill a context for a checked grid and options over a workspace of at least layout_of().total
// bytes, and clear the device scalars on the stream.
int ctx_init(hz_ctx* c, const hz_grid* grid, const hz_options* opts, void* d_workspace,
             size_t bytes, void* stream) {
  const Layout L = layout_of(grid, opts);
  memset(c, 0, sizeof(*c));
  c->g = *grid;
  c->o = *opts;
  c->st = (cudaStream_t)stream;
  c->ws = (char*)d_workspace;
  c->wsbytes = bytes;
  c->sc = (DevScalars*)c->ws;
  c->met = (void*)(c->ws + L.scal);
  char* p = c->ws + L.scal + L.met;
  c->U0 = (double*)p;
  c->U1 = (double*)(p + L.u_bytes);
  c->P[0] = (void*)(p + 2 * L.u_bytes);
  c->P[1] = (void*)(p + 2 * L.u_bytes + L.p_bytes);
  double* geo = (double*)(p + 2 * L.u_bytes + 2 * L.p_bytes);
  c->cur = 0;
  c->v.dims = grid->n[2] > 1 ? 3 : (grid->n[1] > 1 ? 2 : 1);
  c->v.clean = opts->cleaning;
  c->v.mixed = opts->precision == HZ_MIXED;
  c->v.recon = opts->recon;
  c->v.pair = opts->precision == HZ_FP64_DW;
  c->v.diag = 0;

  KParams& kp = c->kp;
  kp.nx = grid->n[0];
  kp.ny = grid->n[1];
  kp.nz = grid->n[2];
  kp.bcx = grid->bc[0];
  kp.bcy = grid->bc[1];
  kp.bcz = grid->bc[2];
  kp.pitch = L.pitch;
  kp.plane = L.plane;
  kp.fs = L.fs;
  kp.mpitch = L.mpitch;
  kp.mny = L.mny;
  kp.mplane = L.mplane;
  kp.ms = L.ms;
  kp.gx = grid->n[0] > 1;
  kp.gy = grid->n[1] > 1;
  kp.gz = grid->n[2] > 1;
  kp.idx = 1.0 / grid->dx[0];
  kp.idy = 1.0 / grid->dx[1];
  kp.idz = 1.0 / grid->dx[2];
  kp.gamma = opts->gamma;
  kp.gfac = opts->gamma / (opts->gamma - 1.0);
  kp.ch = opts->cleaning ? opts->ch : 0.0;
  kp.kappa = opts->cleaning ? opts->kappa : 0.0;
  kp.rho_floor = opts->rho_floor;
  kp.rho_atm = opts->rho_atm;
  kp.p_floor = opts->p_floor;
  const double patm = opts->atm_K > 0.0 ? opts->atm_K * pow(opts->rho_floor, opts->gamma) : opts->p_floor;
  kp.p_atm = patm < opts->p_floor ? opts->p_floor : patm;
  kp.c2p_maxit = opts->c2p_maxit;
  kp.c2p_tol = opts->c2p_tol;
  kp.c2p_step_tol = 0.01 * sqrt(opts->c2p_tol);
  kp.c2p_1d = opts->c2p == HZ_C2P_1D;
  set_float_consts(kp);
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      kp.nsm = nsm;
    else
      kp.nsm = 1;
    kp.dev = dev;
  }
  {
    const int ndims = kp.gx + kp.gy + kp.gz;
    kp.geo_c = geo;
    kp.geo_f = c->v.mixed ? nullptr : geo + GEO_C * L.ms;
    kp.geo_s = c->v.mixed ? nullptr : geo + GEO_C * L.ms + (long long)ndims * GEO_F * L.ms;
  }
  // z chunks: enough blocks for several waves on 152 SMs
  int tx, ty;
  tile_of(c->v.dims, &tx, &ty);
  const int tiles_xy = ((kp.nx + tx - 1) / tx) * ((kp.ny + ty - 1) / ty);
  int chunks = 1;
  if (c->v.dims == 3) {
    const int want = 152 * 2 * 4;
    chunks = (want + tiles_xy - 1) / tiles_xy;
    if (chunks > kp.nz) chunks = kp.nz;
    if (chunks < 1) chunks = 1;
  }
  kp.zlen = (kp.nz + chunks - 1) / chunks;
  c->zchunks = (kp.nz + kp.zlen - 1) / kp.zlen;

  k_reset_scalars<<<1, 1, 0, c->st>>>(c->sc);
  return cuda_err(cudaGetLastError());
}

}  // namespace hzn

extern "C" {

int hz_version(void) { return HZN_VERSION; }

int hz_last_cuda_error(void) { return t_last_cuda_error; }

const char* hz_cuda_error_string(int cuda_code) { return cudaGetErrorString((cudaError_t)cuda_code); }

const char* hz_strerror(int code) {
  switch (code) {
    case HZ_OK: return "ok";
    case HZ_WARN_C2P: return "completed; some cells were reset to atmosphere by the recovery";
    case HZ_ERR_ARG: return "invalid argument";
    case HZ_ERR_CUDA: return "CUDA runtime error";
    case HZ_ERR_STATE: return "call out of order (metric and primitives must be set first)";
    case HZ_ERR_WORKSPACE: return "workspace misaligned or too small";
    case HZ_ERR_UNSUPPORTED: return "option combination not supported";
    case HZ_ERR_TOO_LARGE: return "grid too large for the fixed scratch of hz_step_noalloc";
    default: return "unknown code";
  }
}

int hz_workspace_bytes(const hz_grid* grid, const hz_options* opts, size_t* bytes) {
  if (!bytes) return HZ_ERR_ARG;
  const int e = check_args(grid, opts);
  if (e != HZ_OK) return e;
  *bytes = layout_of(grid, opts).total;
  return HZ_OK;
}

int hz_create(hz_ctx** ctx, const hz_grid* grid, const hz_options* opts, void* d_workspace,
              size_t bytes, void* stream) {
  if (!ctx) return HZ_ERR_ARG;
  *ctx = nullptr;
  int e = check_args(grid, opts);
  if (e != HZ_OK) return e;
  const Layout L = layout_of(grid, opts);
  if (!d_workspace || ((uintptr_t)d_workspace & 255u) != 0 || bytes < L.total) return HZ_ERR_WORKSPACE;
  hz_ctx* c = new (std::nothrow) hz_ctx;
  if (!c) return HZ_ERR_ARG;
  e = ctx_init(c, grid, opts, d_workspace, bytes, stream);
  if (e != HZ_OK) {
    delete c;
    return e;
  }
  *ctx = c;
  return HZ_OK;
}

int hz_destroy(hz_ctx* ctx) {
  delete ctx;
  return HZ_OK;
}

int hz_set_metric(hz_ctx* c, const double* d_metric) {
  if (!c || !d_metric) return HZ_ERR_ARG;
  const long long n = (long long)(c->g.n[0] + 2 * c->kp.gx) * (c->g.n[1] + 2 * c->kp.gy) *
                      (c->g.n[2] + 2 * c->kp.gz);
  cudaError_t e = cudaMemsetAsync(&c->sc->metric_general, 0, sizeof(unsigned int), c->st);
  if (e != cudaSuccess) return cuda_err(e);
  if (c->v.mixed)
    k_pack_metric<float><<<grid_blocks(n * 10, 256), 256, 0, c->st>>>(c->kp, d_metric, (float*)c->met, c->sc);
  else
    k_pack_metric<double><<<grid_blocks(n * 10, 256), 256, 0, c->st>>>(c->kp, d_metric, (double*)c->met, c->sc);
  unsigned int general = 1;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&general, &c->sc->metric_general, sizeof(general), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_err(e);
  c->v.diag = general ? 0 : 1;
  if (c->v.diag) {
    launch_geo_tables(c->v, c->kp, c->met, (double*)c->kp.geo_c, (double*)c->kp.geo_f,
                      (double*)c->kp.geo_s, c->st);
    if (const cudaError_t le = cudaGetLastError(); le != cudaSuccess) return cuda_err(le);
  }
  c->have_metric = 1;
  return HZ_OK;
}

int hz_set_primitives(hz_ctx* c, const double* d_prim) {
  if (!c || !d_prim) return HZ_ERR_ARG;
  if (!c->have_metric) return HZ_ERR_STATE;
  const Layout L = layout_of(&c->g, &c->o);
  c->cur = 0;
  launch_pack_in(c, d_prim, c->P[0]);
  launch_prim2cons(c->v, c->kp, c->P[0], c->met, c->U0, c->st);
  // the second primitive buffer and U1 start as copies so that inactive fields stay defined
  cudaError_t e = cudaMemcpyAsync(c->P[1], c->P[0], L.p_bytes, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->U1, c->U0, L.u_bytes, cudaMemcpyDeviceToDevice, c->st);
  if (e != cudaSuccess) return cuda_err(e);
  k_reset_scalars<<<1, 1, 0, c->st>>>(c->sc);
  launch_max_speed(c->v, c->kp, c->P[0], c->met, c->sc, c->st);
  c->have_prim = 1;
  return cuda_err(cudaGetLastError());
}

int hz_get_primitives(hz_ctx* c, double* d_prim) {
  if (!c || !d_prim) return HZ_ERR_ARG;
  if (!c->have_prim) return HZ_ERR_STATE;
  launch_pack_out(c, c->P[c->cur], !c->v.mixed, d_prim);
  return cuda_err(cudaGetLastError());
}

int hz_get_conserved(hz_ctx* c, double* d_cons) {
  if (!c || !d_cons) return HZ_ERR_ARG;
  if (!c->have_prim) return HZ_ERR_STATE;
  launch_pack_out(c, c->U0, true, d_cons);
  return cuda_err(cudaGetLastError());
}

int hz_step(hz_ctx* c, double dt) {
  if (!c || !(dt > 0.0)) return HZ_ERR_ARG;
  return run_step(c, 0, dt, 0.0, 0.0);
}

int hz_step_cfl(hz_ctx* c, double cfl, double t_end) {
  if (!c || !(cfl > 0.0)) return HZ_ERR_ARG;
  return run_step(c, 1, 0.0, cfl, t_end);
}

int hz_max_speed(hz_ctx* c, double* h_out) {
  if (!c || !h_out) return HZ_ERR_ARG;
  if (!c->have_prim) return HZ_ERR_STATE;
  k_reset_vmax<<<1, 1, 0, c->st>>>(c->sc);
  launch_max_speed(c->v, c->kp, c->P[c->cur], c->met, c->sc, c->st);
  unsigned long long bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, &c->sc->vmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_err(e);
  double v;
  memcpy(&v, &bits, sizeof(v));
  *h_out = v;
  return HZ_OK;
}

int hz_get_stats(hz_ctx* c, hz_stats* h_out) {
  if (!c || !h_out) return HZ_ERR_ARG;
  DevScalars s;
  cudaError_t e = cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_err(e);
  h_out->c2p_failures = (long long)s.fails;
  h_out->c2p_max_iters = s.maxit;
  double v;
  memcpy(&v, &s.vmax_bits, sizeof(v));
  h_out->max_speed = v;
  h_out->t = s.t;
  h_out->dt = s.dt;
  h_out->steps = s.steps;
  return s.fails ? HZ_WARN_C2P : HZ_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// Whole update without any allocation (hz_step_noalloc).  The scratch that hz_create would
// take from the caller's workspace lives in one file-scope device array instead.  Host code
// may not use the array's name as an address: the device address is looked up once per
// device with cudaGetSymbolAddress and passed to the kernels as a pointer.
// ----------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocScratchBytes = HZ_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices];  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device (looked up on first use).
int noalloc_scratch(void** out) {
  int dev = -1;
  if (const cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return cuda_err(e);
  if (dev < 0 || dev >= kNoallocMaxDevices) return HZ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e);
    if (!p) return HZ_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HZ_OK;
}

}  // namespace

extern "C" int hz_step_noalloc(const hz_grid* grid, const hz_options* opts, const double* d_metric,
                               const double* d_prim_in, double* d_prim_out, double dt, int nsteps,
                               void* stream) {
  if (!d_metric || !d_prim_in || !d_prim_out || nsteps < 0 || (nsteps > 0 && !(dt > 0.0)))
    return HZ_ERR_ARG;
  int e = check_args(grid, opts);
  if (e != HZ_OK) return e;
  if (layout_of(grid, opts).total > kNoallocScratchBytes) return HZ_ERR_TOO_LARGE;
  void* scratch = nullptr;
  e = noalloc_scratch(&scratch);
  if (e != HZ_OK) return e;
  hz_ctx c;  // host bookkeeping on the stack: nothing is allocated on the host either
  e = ctx_init(&c, grid, opts, scratch, kNoallocScratchBytes, stream);
  if (e != HZ_OK) return e;
  // every call overwrites the whole state it reads: metric, primitives, conserved state and
  // the counters (cleared by hz_set_primitives) start from this call's inputs
  if ((e = hz_set_metric(&c, d_metric)) != HZ_OK) return e;
  if ((e = hz_set_primitives(&c, d_prim_in)) != HZ_OK) return e;
  for (int s = 0; s < nsteps; ++s)
    if ((e = hz_step(&c, dt)) != HZ_OK) return e;
  if ((e = hz_get_primitives(&c, d_prim_out)) != HZ_OK) return e;
  // wait for the result and report failed recoveries, as hz_get_stats does
  unsigned long long fails = 0;
  cudaError_t ce = cudaMemcpyAsync(&fails, &c.sc->fails, sizeof(fails), cudaMemcpyDeviceToHost, c.st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c.st);
  if (ce != cudaSuccess) return cuda_err(ce);
  return fails ? HZ_WARN_C2P : HZ_OK;
}
