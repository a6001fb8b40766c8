// hzn_adjoint.cu -- reverse (adjoint) sweep of the RK3 finite-volume update, and its C-ABI.
//
// The paper motivates the code by inverse problems on astrophysical sources (§1); it has no
// adjoint.  This file differentiates the discrete update of §2.2/§3.2 exactly: for a loss J of
// the state after n fixed-size steps it returns dJ/dP(0) given dJ/dP(n) (and optionally
// dJ/dU(n)), with every branch decision (MC limiter case, HLLE wave-speed bound, discriminant
// clamp, atmosphere / floor reset) frozen at the forward state.
//
// One substep of the forward update is
//   U' = a U0 + b (U + dt L(P)),   P' = c2p(U')           ((a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3))
// with L the flux divergence plus the metric source.  Its reverse is
//   mu      = lam_U' + (dU/dP at P')^{-T} lam_P'          (implicit-function theorem for the
//                                                           Newton recovery of §2.2: P' solves
//                                                           w(P') = U', so dP'/dU' = (dw/dP)^{-1})
//   lam_U0 += a mu,  lam_U = b mu,  lam_L = b dt mu,
//   lam_P   = (dL/dP)^T lam_L                              (faces: HLLE, flux, conserved vector,
//                                                           wave speeds, MC reconstruction; cells:
//                                                           metric source)
// The flux divergence turns lam_L into per-face flux adjoints (L_c = -(F_{c+1/2} - F_{c-1/2})/dx),
// each face runs the hand-written reverse of its HLLE flux into adjoints of its two
// reconstructed states, and a cell gathers those from the faces whose stencils read it
// (clamped / wrapped ghost reads included), through the frozen MC slope coefficients.
//
// Kernels per reverse substep: k_adj_face (all faces of all active axes) and k_adj_cell (the
// gather of the later substep fused with the implicit-function step of the earlier one).
// Checkpointing (sqrt(n) segments): the forward pass stores (P, U) every K steps; the reverse
// pass recomputes one segment at a time into a tape of the 3K + 1 substep primitive states,
// with the forward kernels, and runs the reverse substeps over it.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "hzn.h"
#include "hzn_ctx.h"
#include "hzn_internal.h"
#include "hzn_physics.cuh"
#include "hzn_adj.h"

namespace hzn {
namespace {

using namespace adj;

constexpr int NF = 9;

inline size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct AdjLayout {
  int K, nseg, ndir;
  int fpitch;
  long long fplane, ffs;
  size_t p_bytes, u_bytes, f_bytes, total;
};

AdjLayout adj_layout(const hz_grid* g, const hz_options* o, int nsteps, int ckpt) {
  const Layout L = layout_of(g, o);
  AdjLayout A;
  int K = ckpt;
  if (K <= 0) {
    K = 1;
    while ((long long)K * K < nsteps) ++K;
  }
  if (K > nsteps) K = nsteps;
  A.K = K;
  A.nseg = (nsteps + K - 1) / K;
  A.ndir = 1 + (g->n[1] > 1) + (g->n[2] > 1);
  const int ay = g->n[1] > 1, az = g->n[2] > 1;
  A.fpitch = (int)rup((size_t)g->n[0] + 1, 16);
  A.fplane = (long long)A.fpitch * (g->n[1] + ay);
  A.ffs = (long long)rup((size_t)(A.fplane * (g->n[2] + az)), 64);
  A.p_bytes = L.p_bytes;
  A.u_bytes = L.u_bytes;
  A.f_bytes = rup((size_t)A.ffs * NF * sizeof(double), 256);
  A.total = (size_t)A.nseg * (A.p_bytes + A.u_bytes)      // checkpoints (P, U)
            + (size_t)(3 * K + 1) * A.p_bytes              // tape of one segment
            + 7 * A.u_bytes                                // lamP, lamU, lamA, lamL, out, U0/U1
            + (size_t)A.ndir * 2 * A.f_bytes;              // face adjoints
  return A;
}

}  // namespace
}  // namespace hzn

using namespace hzn;

struct hz_adjoint {
  hz_ctx* ctx;
  int nsteps;
  double dt;
  AdjLayout A;
  char* ws;
  char* ckP;
  char* ckU;
  char* tape;
  double* rU0;   // conserved states of the recomputation (the context's own stay untouched)
  double* rU1;
  AdjBufs bufs;
  int have_forward;
};

namespace {

inline void* tape_slot(hz_adjoint* a, int s) { return a->tape + (size_t)s * a->A.p_bytes; }

// Threads per block of the reverse kernels: one warp per block while the grid is too small to
// give every SM several blocks of four warps (an FP64-heavy warp keeps an SM's FP64 pipe busy
// on its own), four warps otherwise.
inline int block_threads(long long n) { return n < 152LL * 4 * 128 ? 32 : 128; }

// Recompute the primitive states of every substep of segment q into the tape.
void recompute_segment(hz_adjoint* a, int q, int* nsteps_out) {
  hz_ctx* c = a->ctx;
  const int s0 = q * a->A.K;
  const int ns = (s0 + a->A.K <= a->nsteps) ? a->A.K : a->nsteps - s0;
  double* keep0 = c->U0;
  double* keep1 = c->U1;
  c->U0 = a->rU0;
  c->U1 = a->rU1;
  cudaMemcpyAsync(tape_slot(a, 0), a->ckP + (size_t)q * a->A.p_bytes, a->A.p_bytes,
                  cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->U0, a->ckU + (size_t)q * a->A.u_bytes, a->A.u_bytes, cudaMemcpyDeviceToDevice,
                  c->st);
  launch_clock(c, 0, a->dt, 0.0, 0.0);
  for (int kk = 0; kk < ns; ++kk)
    launch_rk3(c, tape_slot(a, 3 * kk), tape_slot(a, 3 * kk + 1), tape_slot(a, 3 * kk + 2),
               tape_slot(a, 3 * kk + 3));
  c->U0 = keep0;
  c->U1 = keep1;
  *nsteps_out = ns;
}

void launch_cell(hz_adjoint* a, const void* Pb, int stage, int gather) {
  hz_ctx* c = a->ctx;
  AdjShape sh;
  sh.fpitch = a->A.fpitch;
  sh.fplane = a->A.fplane;
  sh.ffs = a->A.ffs;
  sh.dt = a->dt;
  static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
  sh.a = stage < 3 ? ca[stage] : 0.0;
  sh.b = stage < 3 ? cb[stage] : 0.0;
  sh.stage = stage;
  sh.gather = gather;
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  const int threads = block_threads(n);
  const int blocks = grid_blocks(n, threads);
  if (c->v.diag)
    adj_launch_cell<true>(c->o.cleaning, blocks, threads, c->st, c->kp, sh, (const double*)Pb,
                          (const double*)c->met, a->bufs);
  else
    adj_launch_cell<false>(c->o.cleaning, blocks, threads, c->st, c->kp, sh, (const double*)Pb,
                           (const double*)c->met, a->bufs);
}

void launch_face(hz_adjoint* a, const void* Ps) {
  hz_ctx* c = a->ctx;
  AdjShape sh;
  memset(&sh, 0, sizeof(sh));
  sh.fpitch = a->A.fpitch;
  sh.fplane = a->A.fplane;
  sh.ffs = a->A.ffs;
  long long nmax = 0;
  for (int d = 0; d < a->A.ndir; ++d) {
    const long long nf = (long long)(c->g.n[0] + (d == 0)) * (c->g.n[1] + (d == 1)) * (c->g.n[2] + (d == 2));
    if (nf > nmax) nmax = nf;
  }
  const int threads = block_threads(nmax);
  dim3 grid(grid_blocks(nmax, threads), a->A.ndir);
  if (c->v.diag)
    adj_launch_face<true>(c->o.cleaning, grid, threads, c->st, c->kp, sh, (const double*)Ps,
                          (const double*)c->met, a->bufs);
  else
    adj_launch_face<false>(c->o.cleaning, grid, threads, c->st, c->kp, sh, (const double*)Ps,
                           (const double*)c->met, a->bufs);
}

}  // namespace

extern "C" {

int hz_adjoint_workspace_bytes(const hz_grid* grid, const hz_options* opts, int nsteps,
                               int ckpt_every, size_t* bytes) {
  if (!bytes || nsteps < 1) return HZ_ERR_ARG;
  const int e = check_args(grid, opts);
  if (e != HZ_OK) return e;
  if (opts->precision != HZ_FP64 || opts->recon != HZ_RECON_MC) return HZ_ERR_UNSUPPORTED;
  *bytes = adj_layout(grid, opts, nsteps, ckpt_every).total;
  return HZ_OK;
}

int hz_adjoint_create(hz_adjoint** adj, hz_ctx* ctx, int nsteps, double dt, int ckpt_every,
                      void* d_workspace, size_t bytes) {
  if (!adj) return HZ_ERR_ARG;
  *adj = nullptr;
  if (!ctx || nsteps < 1 || !(dt > 0.0)) return HZ_ERR_ARG;
  if (ctx->o.precision != HZ_FP64 || ctx->o.recon != HZ_RECON_MC) return HZ_ERR_UNSUPPORTED;
  if (!ctx->have_metric) return HZ_ERR_STATE;
  const AdjLayout A = adj_layout(&ctx->g, &ctx->o, nsteps, ckpt_every);
  if (!d_workspace || ((uintptr_t)d_workspace & 255u) != 0 || bytes < A.total) return HZ_ERR_WORKSPACE;
  hz_adjoint* a = new (std::nothrow) hz_adjoint;
  if (!a) return HZ_ERR_ARG;
  memset(a, 0, sizeof(*a));
  a->ctx = ctx;
  a->nsteps = nsteps;
  a->dt = dt;
  a->A = A;
  a->ws = (char*)d_workspace;
  char* p = a->ws;
  a->ckP = p;
  p += (size_t)A.nseg * A.p_bytes;
  a->ckU = p;
  p += (size_t)A.nseg * A.u_bytes;
  a->tape = p;
  p += (size_t)(3 * A.K + 1) * A.p_bytes;
  a->bufs.lamP = (double*)p;
  p += A.u_bytes;
  a->bufs.lamU = (double*)p;
  p += A.u_bytes;
  a->bufs.lamA = (double*)p;
  p += A.u_bytes;
  a->bufs.lamL = (double*)p;
  p += A.u_bytes;
  a->bufs.out = (double*)p;
  p += A.u_bytes;
  a->rU0 = (double*)p;
  p += A.u_bytes;
  a->rU1 = (double*)p;
  p += A.u_bytes;
  for (int d = 0; d < 3; ++d) {
    a->bufs.fL[d] = a->bufs.fR[d] = nullptr;
    if (d < A.ndir) {
      a->bufs.fL[d] = (double*)p;
      p += A.f_bytes;
      a->bufs.fR[d] = (double*)p;
      p += A.f_bytes;
    }
  }
  *adj = a;
  return HZ_OK;
}

int hz_adjoint_destroy(hz_adjoint* adj) {
  delete adj;
  return HZ_OK;
}

int hz_adjoint_checkpoint_interval(const hz_adjoint* adj, int* h_every, int* h_segments) {
  if (!adj) return HZ_ERR_ARG;
  if (h_every) *h_every = adj->A.K;
  if (h_segments) *h_segments = adj->A.nseg;
  return HZ_OK;
}

int hz_adjoint_forward(hz_adjoint* a, const double* d_prim_in, double* d_prim_out) {
  if (!a || !d_prim_in) return HZ_ERR_ARG;
  hz_ctx* c = a->ctx;
  int e = hz_set_primitives(c, d_prim_in);
  if (e != HZ_OK) return e;
  for (int s = 0; s < a->nsteps; ++s) {
    if (s % a->A.K == 0) {
      const int q = s / a->A.K;
      cudaMemcpyAsync(a->ckP + (size_t)q * a->A.p_bytes, c->P[c->cur], a->A.p_bytes,
                      cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(a->ckU + (size_t)q * a->A.u_bytes, c->U0, a->A.u_bytes,
                      cudaMemcpyDeviceToDevice, c->st);
    }
    e = hz_step(c, a->dt);
    if (e != HZ_OK) return e;
  }
  if (d_prim_out) {
    e = hz_get_primitives(c, d_prim_out);
    if (e != HZ_OK) return e;
  }
  a->have_forward = 1;
  return cuda_err(cudaGetLastError());
}

int hz_adjoint_backward(hz_adjoint* a, const double* d_gprim_out, const double* d_gcons_out,
                        double* d_gprim_in) {
  if (!a || !d_gprim_out || !d_gprim_in) return HZ_ERR_ARG;
  if (!a->have_forward) return HZ_ERR_STATE;
  hz_ctx* c = a->ctx;
  launch_pack_in(c, d_gprim_out, a->bufs.lamP);
  if (d_gcons_out) launch_pack_in(c, d_gcons_out, a->bufs.lamU);
  else cudaMemsetAsync(a->bufs.lamU, 0, a->A.u_bytes, c->st);
  cudaMemsetAsync(a->bufs.lamA, 0, a->A.u_bytes, c->st);
  cudaMemsetAsync(a->bufs.lamL, 0, a->A.u_bytes, c->st);
  bool first = true;
  for (int q = a->A.nseg - 1; q >= 0; --q) {
    int ns = 0;
    recompute_segment(a, q, &ns);
    for (int kk = ns - 1; kk >= 0; --kk) {
      for (int s = 2; s >= 0; --s) {
        launch_cell(a, tape_slot(a, 3 * kk + s + 1), s, first ? 0 : 1);
        first = false;
        launch_face(a, tape_slot(a, 3 * kk + s));
      }
    }
  }
  launch_cell(a, tape_slot(a, 0), 3, 1);
  launch_pack_out(c, a->bufs.out, true, d_gprim_in);
  return cuda_err(cudaGetLastError());
}

}  // extern "C"
