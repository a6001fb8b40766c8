// hzn_ensemble.cu -- many independent 1-D shock tubes advanced to a common end time in one
// persistent launch (C-ABI hz_ensemble_*).
//
// Each tube is a 1-D problem in Minkowski spacetime with outflow boundaries, its own cell
// count, width and adiabatic index, and its own CFL time step; the scheme is the one of the
// grid path (MC reconstruction, HLLE, RK3, Newton recovery; §2.2, §3.2) in FP64 without
// divergence cleaning.  The paper's fine-grained parallelism (one thread per cell, §3.1) is
// kept inside a tube; across tubes a persistent grid of CTAs pulls tubes from a work queue in
// decreasing order of cost (cells^2), so that long tubes start first.  A CTA owns a whole tube
// and separates the three substeps of each step with block barriers, so no grid-wide
// synchronisation exists.  Every loop is bounded (max_steps per tube).

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "hzn.h"
#include "hzn_kernels.cuh"

using namespace hzn;

namespace {

constexpr int NF = 9;

struct TubeInfo {
  long long off;  // first cell of the tube in the concatenated, padded state arrays
  int n;          // cells
  int pad;
  double idx;     // 1 / dx
  double gamma, gfac;
};

struct TubeResult {
  double t;
  long long steps;
  unsigned long long fails;
  int maxit;
  int pad;
};

struct EnsParams {
  const TubeInfo* tubes;
  const int* order;      // tube indices, most expensive first
  int ntubes;
  long long fs;          // field stride of the state arrays
  double* U0;
  double* U1;
  double* P0;
  double* P1;
  TubeResult* res;
  int* queue;            // next position in order[]
  double t_end, cfl;
  long long max_steps;
  double rho_floor, rho_atm, p_floor, atm_K;
  int c2p_maxit;
  double c2p_tol;
  double c2p_step_tol;
};

// Flat-metric geometry (alpha = 1, beta = 0, gamma_ij = delta_ij).
__device__ __forceinline__ Geom<double> flat_geom() {
  double m[10] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 1.0};
  return make_geom<true>(m);
}

// HLLE flux at face f of a tube (between cells f-1 and f), outflow boundaries; plain loads
// because the primitive buffers are rewritten inside this launch.
__device__ __forceinline__ void tube_face(const double* P, long long fs, int n, int f,
                                          const Geom<double>& G, const Consts<double>& c,
                                          double F[8]) {
  const int i0 = max(f - 2, 0), i1 = max(f - 1, 0), i2 = min(f, n - 1), i3 = min(f + 1, n - 1);
  double PL[9], PR[9];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double* pf = P + q * fs;
    const double a = pf[i0], b = pf[i1], cc = pf[i2], d = pf[i3];
    const double d0 = b - a, d1 = cc - b, d2 = d - cc;
    PL[q] = b + mc_half_slope(d0, d1);
    PR[q] = cc - mc_half_slope(d1, d2);
  }
  PL[8] = PR[8] = 0.0;
  // the grid kernel's HLLE of one face (FP64: both roots as fractions, one division; each
  // state's weighted share added without forming its flux and conserved vectors)
  double F9[9];
  hlle_face_fused<0, false, true>(G, PL, PR, c, 0.0, F9, 1);
#pragma unroll
  for (int q = 0; q < 8; ++q) F[q] = F9[q];
}

__device__ __forceinline__ double cell_speed(const double* P, long long fs, int i, const Geom<double>& G,
                                             const Consts<double>& c, double idx) {
  double Pc[9];
#pragma unroll
  for (int q = 0; q < 8; ++q) Pc[q] = P[q * fs + i];
  Pc[8] = 0.0;
  const State<double> S = make_state<true>(G, Pc, c);
  double lm, lp;
  speeds_of<0, true, double, true>(G, S, cms2_of<double, true>(S, c), lm, lp);
  return fmax(fabs(lm), fabs(lp)) * idx;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_ensemble(const EnsParams ep) {
  constexpr int CH = NT - 1;  // cells per chunk: NT faces
  __shared__ double ff[8][NT];
  __shared__ double red[NT / 32];
  __shared__ int s_q;
  const Geom<double> G = flat_geom();

  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(ep.queue, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= ep.ntubes) break;
    const int tube = ep.order[q];
    const TubeInfo ti = ep.tubes[tube];
    Consts<double> c;
    c.gamma = ti.gamma;
    c.gfac = ti.gfac;
    c.ch = c.ch2 = 0.0;
    const long long fs = ep.fs;
    double* const Pb0 = ep.P0 + ti.off;
    double* const Pb1 = ep.P1 + ti.off;
    double* const U0 = ep.U0 + ti.off;
    double* const U1 = ep.U1 + ti.off;
    const int n = ti.n;
    // atmosphere pressure of this tube's gas
    double p_atm = ep.atm_K > 0.0 ? ep.atm_K * pow(ep.rho_floor, ti.gamma) : ep.p_floor;
    p_atm = p_atm < ep.p_floor ? ep.p_floor : p_atm;

    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) v = fmax(v, cell_speed(Pb0, fs, i, G, c, ti.idx));
    double vmax = block_max<NT>(v, red);
    double t = 0.0;
    long long steps = 0;
    int fails = 0, maxit = 0;
    int cur = 0;
    while (t < ep.t_end && steps < ep.max_steps) {
      double dt = vmax > 0.0 ? ep.cfl / vmax : ep.t_end - t;
      if (t + dt > ep.t_end) dt = ep.t_end - t;
      double vloc = 0.0;
      for (int stage = 0; stage < 3; ++stage) {
        // Shu-Osher RK3 (same buffer rotation as the grid path)
        const int swap = cur ^ (stage == 1 ? 1 : 0);
        const double* Pin = swap ? Pb1 : Pb0;
        double* Pout = swap ? Pb0 : Pb1;
        const double* Uk = stage == 0 ? U0 : U1;
        double* Uout = stage == 2 ? U0 : U1;
        const double a0 = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
        const double ak = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
        for (int c0 = 0; c0 < n; c0 += CH) {
          const int f = c0 + (int)threadIdx.x;
          if (f <= n) {
            double F[8];
            tube_face(Pin, fs, n, f, G, c, F);
#pragma unroll
            for (int qf = 0; qf < 8; ++qf) ff[qf][threadIdx.x] = F[qf];
          }
          __syncthreads();
          const int i = c0 + (int)threadIdx.x;
          if ((int)threadIdx.x < CH && i < n) {
            double U[9], Pg[9], Pn[9];
#pragma unroll
            for (int qf = 0; qf < 8; ++qf) {
              const double L = -(ff[qf][threadIdx.x + 1] - ff[qf][threadIdx.x]) * ti.idx;
              double u = ak * (Uk[qf * fs + i] + dt * L);
              if (a0 != 0.0) u += a0 * U0[qf * fs + i];
              U[qf] = u;
              Pg[qf] = Pin[qf * fs + i];
            }
            U[8] = Pg[8] = 0.0;
            // recovery with atmosphere / floors (same rules as the grid path)
            const bool atm = U[U_D] < ep.rho_atm;
            C2PResult r = {1, 0};
            if (!atm) r = con2prim<false, true>(G, U, Pg, c, ep.c2p_maxit, ep.c2p_step_tol, Pn);
            maxit = max(maxit, r.iters);
            bool reset = false;
            if (atm || !r.ok || Pn[P_RHO] < ep.rho_floor) {
              Pn[P_BX] = U[U_BX];
              Pn[P_BY] = U[U_BY];
              Pn[P_BZ] = U[U_BZ];
              Pn[P_RHO] = ep.rho_floor;
              Pn[P_PRS] = p_atm;
              Pn[P_UX] = Pn[P_UY] = Pn[P_UZ] = 0.0;
              reset = true;
            } else if (Pn[P_PRS] < ep.p_floor) {
              Pn[P_PRS] = ep.p_floor;
              reset = true;
            }
            Pn[P_PSI] = 0.0;
            if (reset) {
              const State<double> S = make_state<true>(G, Pn, c);
              cons_of<false>(G, S, U);
            }
            fails += r.ok ? 0 : 1;
#pragma unroll
            for (int qf = 0; qf < 8; ++qf) {
              Uout[qf * fs + i] = U[qf];
              Pout[qf * fs + i] = Pn[qf];
            }
            if (stage == 2) {
              const State<double> S = make_state<true>(G, Pn, c);
              double lm, lp;
              speeds_of<0, true, double, true>(G, S, cms2_of<double, true>(S, c), lm, lp);
              vloc = fmax(vloc, fmax(fabs(lm), fabs(lp)) * ti.idx);
            }
          }
          __syncthreads();
        }
      }
      cur = 1 - cur;
      vmax = block_max<NT>(vloc, red);
      t += dt;
      ++steps;
    }
    // leave the final primitive state in the first buffer
    if (cur == 1)
      for (int i = threadIdx.x; i < n; i += NT)
#pragma unroll
        for (int qf = 0; qf < 8; ++qf) Pb0[qf * fs + i] = Pb1[qf * fs + i];
    // per-tube statistics
    for (int o = 16; o > 0; o >>= 1) {
      fails += __shfl_xor_sync(0xffffffffu, fails, o);
      maxit = max(maxit, __shfl_xor_sync(0xffffffffu, maxit, o));
    }
    __shared__ int sfail[NT / 32], sit[NT / 32];
    if ((threadIdx.x & 31) == 0) {
      sfail[threadIdx.x >> 5] = fails;
      sit[threadIdx.x >> 5] = maxit;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int nf = 0, mi = 0;
      for (int w = 0; w < NT / 32; ++w) {
        nf += sfail[w];
        mi = max(mi, sit[w]);
      }
      TubeResult rr;
      rr.t = t;
      rr.steps = steps;
      rr.fails = (unsigned long long)nf;
      rr.maxit = mi;
      rr.pad = 0;
      ep.res[tube] = rr;
    }
    __syncthreads();
  }
}

// Conserved state of every tube from its primitive state (flat metric).
__global__ void k_ens_prim2cons(const EnsParams ep, long long total) {
  const Geom<double> G = flat_geom();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    // locate the tube by binary search over offsets is avoided: the pack kernel stores the
    // tube index of every padded cell in P1's last field slot before this runs
    const int tube = (int)ep.P1[8 * ep.fs + q];
    if (tube < 0) continue;
    const TubeInfo ti = ep.tubes[tube];
    Consts<double> c;
    c.gamma = ti.gamma;
    c.gfac = ti.gfac;
    c.ch = c.ch2 = 0.0;
    double P[9], U[9];
#pragma unroll
    for (int f = 0; f < 8; ++f) P[f] = ep.P0[f * ep.fs + q];
    P[8] = 0.0;
    const State<double> S = make_state<true>(G, P, c);
    cons_of<false>(G, S, U);
#pragma unroll
    for (int f = 0; f < 8; ++f) ep.U0[f * ep.fs + q] = U[f];
  }
}

// Caller layout (tubes concatenated without padding, field-major over the concatenation:
// field f of cell c of tube t at [f * Ncat + cat_off[t] + c]) <-> padded state arrays.
__global__ void k_ens_pack(const long long* __restrict__ cat_off, const long long* __restrict__ pad_off,
                           const int* __restrict__ tube_of_cat, long long ncat, long long fs,
                           const double* __restrict__ src, double* __restrict__ dst, int to_internal) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncat * 8;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / ncat);
    const long long r = q % ncat;
    const int t = tube_of_cat[r];
    const long long p = pad_off[t] + (r - cat_off[t]);
    if (to_internal) dst[f * fs + p] = src[f * ncat + r];
    else dst[f * ncat + r] = src[f * fs + p];
  }
}

__global__ void k_fill_int_as_double(double* dst, const int* tube_of_pad, long long npad) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npad;
       q += (long long)gridDim.x * blockDim.x)
    dst[q] = (double)tube_of_pad[q];
}

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct EnsLayout {
  long long npad;        // padded cells (field stride)
  size_t tubes_b, order_b, res_b, q_b, catoff_b, padoff_b, tcat_b, tpad_b, state_b, total;
};

EnsLayout ens_layout(int ntubes, const int* n) {
  EnsLayout L;
  long long npad = 0, ncat = 0;
  for (int t = 0; t < ntubes; ++t) {
    npad += (long long)round_up((size_t)n[t], 32);
    ncat += n[t];
  }
  L.npad = (long long)round_up((size_t)npad, 64);
  L.tubes_b = round_up(sizeof(TubeInfo) * ntubes, 256);
  L.order_b = round_up(sizeof(int) * ntubes, 256);
  L.res_b = round_up(sizeof(TubeResult) * ntubes, 256);
  L.q_b = 256;
  L.catoff_b = round_up(sizeof(long long) * ntubes, 256);
  L.padoff_b = L.catoff_b;
  L.tcat_b = round_up(sizeof(int) * (size_t)ncat, 256);
  L.tpad_b = round_up(sizeof(int) * (size_t)L.npad, 256);
  L.state_b = (size_t)L.npad * NF * sizeof(double);
  L.total = L.tubes_b + L.order_b + L.res_b + L.q_b + L.catoff_b + L.padoff_b + L.tcat_b + L.tpad_b +
            4 * L.state_b;
  return L;
}

int cuda_err(cudaError_t e) { return record_cuda_error(e); }

}  // namespace

struct hz_ensemble {
  int ntubes;
  long long ncat;
  EnsLayout L;
  EnsParams ep;
  cudaStream_t st;
  hz_options o;
  long long* cat_off;    // device
  long long* pad_off;    // device
  int* tube_of_cat;      // device
  int* tube_of_pad;      // device
  int nt, minb;          // launch shape (threads per CTA, CTAs per SM)
  int have_prim;
  std::vector<long long> h_cat_off;
  std::vector<int> h_n;
  cudaGraphExec_t graph;
  double graph_t_end, graph_cfl;
  long long graph_max_steps;
};

namespace {

int ens_launch(hz_ensemble* e, double t_end, double cfl, long long max_steps) {
  e->ep.t_end = t_end;
  e->ep.cfl = cfl;
  e->ep.max_steps = max_steps;
  cudaError_t err = cudaMemsetAsync(e->ep.queue, 0, sizeof(int), e->st);
  if (err != cudaSuccess) return cuda_err(err);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(e->ntubes, nsm * e->minb));
  if (e->nt == 128 && e->minb == 1) k_ensemble<128, 1><<<grid, 128, 0, e->st>>>(e->ep);
  else if (e->nt == 128 && e->minb == 2) k_ensemble<128, 2><<<grid, 128, 0, e->st>>>(e->ep);
  else if (e->nt == 128 && e->minb == 3) k_ensemble<128, 3><<<grid, 128, 0, e->st>>>(e->ep);
  else if (e->nt == 256 && e->minb == 1) k_ensemble<256, 1><<<grid, 256, 0, e->st>>>(e->ep);
  else if (e->nt == 64 && e->minb == 4) k_ensemble<64, 4><<<grid, 64, 0, e->st>>>(e->ep);
  else return HZ_ERR_ARG;
  return cuda_err(cudaGetLastError());
}

}  // namespace

extern "C" {

int hz_ensemble_workspace_bytes(int ntubes, const int* h_n, size_t* bytes) {
  if (ntubes < 1 || !h_n || !bytes) return HZ_ERR_ARG;
  for (int t = 0; t < ntubes; ++t)
    if (h_n[t] < 2 || h_n[t] > (1 << 24)) return HZ_ERR_ARG;
  *bytes = ens_layout(ntubes, h_n).total;
  return HZ_OK;
}

int hz_ensemble_create(hz_ensemble** out, int ntubes, const int* h_n, const double* h_dx,
                       const double* h_gamma, const hz_options* opts, void* d_workspace,
                       size_t bytes, void* stream) {
  if (!out) return HZ_ERR_ARG;
  *out = nullptr;
  if (ntubes < 1 || !h_n || !h_dx || !h_gamma || !opts) return HZ_ERR_ARG;
  for (int t = 0; t < ntubes; ++t) {
    if (h_n[t] < 2 || h_n[t] > (1 << 24)) return HZ_ERR_ARG;
    if (!(h_dx[t] > 0.0) || !(h_gamma[t] > 1.0) || h_gamma[t] > 3.0) return HZ_ERR_ARG;
  }
  if (opts->precision != HZ_FP64 || opts->cleaning || opts->recon != HZ_RECON_MC || opts->c2p != HZ_C2P_2D)
    return HZ_ERR_UNSUPPORTED;
  if (!(opts->rho_floor > 0.0) || !(opts->p_floor > 0.0) || opts->c2p_maxit < 1 ||
      opts->c2p_maxit > 200 || !(opts->c2p_tol >= 1e-15) || opts->c2p_tol > 1e-6)
    return HZ_ERR_ARG;
  const EnsLayout L = ens_layout(ntubes, h_n);
  if (!d_workspace || ((uintptr_t)d_workspace & 255u) != 0 || bytes < L.total) return HZ_ERR_WORKSPACE;
  hz_ensemble* e = new (std::nothrow) hz_ensemble;
  if (!e) return HZ_ERR_ARG;
  e->ntubes = ntubes;
  e->L = L;
  e->st = (cudaStream_t)stream;
  e->o = *opts;
  e->nt = 128;
  e->minb = 2;
  e->have_prim = 0;
  e->graph = nullptr;
  e->h_n.assign(h_n, h_n + ntubes);
  char* p = (char*)d_workspace;
  TubeInfo* d_tubes = (TubeInfo*)p;
  p += L.tubes_b;
  int* d_order = (int*)p;
  p += L.order_b;
  TubeResult* d_res = (TubeResult*)p;
  p += L.res_b;
  int* d_queue = (int*)p;
  p += L.q_b;
  e->cat_off = (long long*)p;
  p += L.catoff_b;
  e->pad_off = (long long*)p;
  p += L.padoff_b;
  e->tube_of_cat = (int*)p;
  p += L.tcat_b;
  e->tube_of_pad = (int*)p;
  p += L.tpad_b;
  double* s = (double*)p;
  e->ep.U0 = s;
  e->ep.U1 = s + (size_t)L.npad * NF;
  e->ep.P0 = s + 2 * (size_t)L.npad * NF;
  e->ep.P1 = s + 3 * (size_t)L.npad * NF;
  e->ep.tubes = d_tubes;
  e->ep.order = d_order;
  e->ep.res = d_res;
  e->ep.queue = d_queue;
  e->ep.ntubes = ntubes;
  e->ep.fs = L.npad;
  e->ep.rho_floor = opts->rho_floor;
  e->ep.rho_atm = opts->rho_atm;
  e->ep.p_floor = opts->p_floor;
  e->ep.c2p_maxit = opts->c2p_maxit;
  e->ep.c2p_tol = opts->c2p_tol;
  e->ep.c2p_step_tol = 0.01 * sqrt(opts->c2p_tol);
  // host tables
  std::vector<TubeInfo> ti(ntubes);
  std::vector<long long> cat(ntubes), pad(ntubes);
  long long nc = 0, np = 0;
  for (int t = 0; t < ntubes; ++t) {
    cat[t] = nc;
    pad[t] = np;
    ti[t].off = np;
    ti[t].n = h_n[t];
    ti[t].pad = 0;
    ti[t].idx = 1.0 / h_dx[t];
    ti[t].gamma = h_gamma[t];
    ti[t].gfac = h_gamma[t] / (h_gamma[t] - 1.0);
    nc += h_n[t];
    np += (long long)round_up((size_t)h_n[t], 32);
  }
  e->ncat = nc;
  e->h_cat_off = cat;
  std::vector<int> order(ntubes);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
  std::vector<int> tcat((size_t)nc), tpad((size_t)L.npad, -1);
  for (int t = 0; t < ntubes; ++t) {
    for (int c = 0; c < h_n[t]; ++c) {
      tcat[(size_t)(cat[t] + c)] = t;
      tpad[(size_t)(pad[t] + c)] = t;
    }
  }
  e->ep.atm_K = opts->atm_K;
  // synchronous uploads of the setup tables (setup is not on the hot path)
  cudaError_t err = cudaMemcpy(d_tubes, ti.data(), sizeof(TubeInfo) * ntubes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(d_order, order.data(), sizeof(int) * ntubes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->cat_off, cat.data(), sizeof(long long) * ntubes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->pad_off, pad.data(), sizeof(long long) * ntubes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->tube_of_cat, tcat.data(), sizeof(int) * (size_t)nc, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->tube_of_pad, tpad.data(), sizeof(int) * (size_t)L.npad, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemset(d_res, 0, sizeof(TubeResult) * ntubes);
  if (err != cudaSuccess) {
    delete e;
    return cuda_err(err);
  }
  *out = e;
  return HZ_OK;
}

int hz_ensemble_destroy(hz_ensemble* e) {
  if (e && e->graph) cudaGraphExecDestroy(e->graph);
  delete e;
  return HZ_OK;
}

int hz_ensemble_set_primitives(hz_ensemble* e, const double* d_prim) {
  if (!e || !d_prim) return HZ_ERR_ARG;
  const long long total = e->L.npad;
  // zero the state (padding cells stay defined), then scatter the tubes
  cudaError_t err = cudaMemsetAsync(e->ep.U0, 0, 4 * e->L.state_b, e->st);
  if (err != cudaSuccess) return cuda_err(err);
  const int nb = (int)std::min<long long>((e->ncat * 8 + 255) / 256, 152 * 16);
  k_ens_pack<<<nb, 256, 0, e->st>>>(e->cat_off, e->pad_off, e->tube_of_cat, e->ncat, e->ep.fs, d_prim, e->ep.P0, 1);
  // tube index of every padded cell, staged in the unused ninth field of P1
  k_fill_int_as_double<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, e->st>>>(
      e->ep.P1 + 8 * e->ep.fs, e->tube_of_pad, total);
  k_ens_prim2cons<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, e->st>>>(e->ep, total);
  err = cudaMemcpyAsync(e->ep.P1, e->ep.P0, e->L.state_b, cudaMemcpyDeviceToDevice, e->st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(e->ep.U1, e->ep.U0, e->L.state_b, cudaMemcpyDeviceToDevice, e->st);
  if (err == cudaSuccess) err = cudaMemsetAsync(e->ep.res, 0, sizeof(TubeResult) * e->ntubes, e->st);
  e->have_prim = 1;
  if (err != cudaSuccess) return cuda_err(err);
  return cuda_err(cudaGetLastError());
}

int hz_ensemble_set_launch(hz_ensemble* e, int threads, int ctas_per_sm) {
  if (!e) return HZ_ERR_ARG;
  const bool ok = (threads == 128 && (ctas_per_sm >= 1 && ctas_per_sm <= 3)) ||
                  (threads == 256 && ctas_per_sm == 1) || (threads == 64 && ctas_per_sm == 4);
  if (!ok) return HZ_ERR_ARG;
  e->nt = threads;
  e->minb = ctas_per_sm;
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  return HZ_OK;
}

int hz_ensemble_run(hz_ensemble* e, double t_end, double cfl, long long max_steps, int use_graph) {
  if (!e || !(t_end >= 0.0) || !(cfl > 0.0) || max_steps < 1) return HZ_ERR_ARG;
  if (!e->have_prim) return HZ_ERR_STATE;
  if (!use_graph) return ens_launch(e, t_end, cfl, max_steps);
  if (e->graph && (e->graph_t_end != t_end || e->graph_cfl != cfl || e->graph_max_steps != max_steps)) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  if (!e->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_err(err);
    const int r = ens_launch(e, t_end, cfl, max_steps);
    err = cudaStreamEndCapture(e->st, &g);
    if (r != HZ_OK || err != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return r != HZ_OK ? r : cuda_err(err);
    }
    err = cudaGraphInstantiate(&e->graph, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      e->graph = nullptr;
      return cuda_err(err);
    }
    e->graph_t_end = t_end;
    e->graph_cfl = cfl;
    e->graph_max_steps = max_steps;
  }
  return cuda_err(cudaGraphLaunch(e->graph, e->st));
}

int hz_ensemble_get_primitives(hz_ensemble* e, double* d_prim) {
  if (!e || !d_prim) return HZ_ERR_ARG;
  if (!e->have_prim) return HZ_ERR_STATE;
  const int nb = (int)std::min<long long>((e->ncat * 8 + 255) / 256, 152 * 16);
  k_ens_pack<<<nb, 256, 0, e->st>>>(e->cat_off, e->pad_off, e->tube_of_cat, e->ncat, e->ep.fs, e->ep.P0, d_prim, 0);
  return cuda_err(cudaGetLastError());
}

int hz_ensemble_results(hz_ensemble* e, double* h_t, long long* h_steps, long long* h_fails) {
  if (!e || !h_t || !h_steps || !h_fails) return HZ_ERR_ARG;
  std::vector<TubeResult> r(e->ntubes);
  cudaError_t err = cudaMemcpyAsync(r.data(), e->ep.res, sizeof(TubeResult) * e->ntubes,
                                    cudaMemcpyDeviceToHost, e->st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(e->st);
  if (err != cudaSuccess) return cuda_err(err);
  long long tot = 0;
  for (int t = 0; t < e->ntubes; ++t) {
    h_t[t] = r[t].t;
    h_steps[t] = r[t].steps;
    h_fails[t] = (long long)r[t].fails;
    tot += h_fails[t];
  }
  return tot ? HZ_WARN_C2P : HZ_OK;
}

// Pick the launch shape that runs a short probe of this ensemble fastest.  The probe advances
// every tube to t_probe; candidates are (threads per CTA, CTAs per SM) in {(64,4), (128,1),
// (128,2), (128,3), (256,1)}.  The state is restored from the primitives given.
int hz_ensemble_autotune(hz_ensemble* e, const double* d_prim, double t_probe, double cfl,
                         int* h_threads, int* h_ctas_per_sm, float* h_ms) {
  if (!e || !d_prim || !h_threads || !h_ctas_per_sm || !(t_probe > 0.0) || !(cfl > 0.0)) return HZ_ERR_ARG;
  const int cand[5][2] = {{64, 4}, {128, 1}, {128, 2}, {128, 3}, {256, 1}};
  cudaEvent_t a, b;
  if (const cudaError_t ea = cudaEventCreate(&a); ea != cudaSuccess) return cuda_err(ea);
  if (const cudaError_t eb = cudaEventCreate(&b); eb != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_err(eb);
  }
  float best = 1e30f;
  int bt = 128, bm = 2;
  for (int k = 0; k < 5; ++k) {
    int r = hz_ensemble_set_launch(e, cand[k][0], cand[k][1]);
    if (r == HZ_OK) r = hz_ensemble_set_primitives(e, d_prim);
    if (r != HZ_OK) break;
    cudaEventRecord(a, e->st);
    r = ens_launch(e, t_probe, cfl, 1LL << 40);
    cudaEventRecord(b, e->st);
    const cudaError_t es = r != HZ_OK ? cudaSuccess : cudaEventSynchronize(b);
    if (r != HZ_OK || es != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return r != HZ_OK ? r : cuda_err(es);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (h_ms) h_ms[k] = ms;
    if (ms < best) {
      best = ms;
      bt = cand[k][0];
      bm = cand[k][1];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *h_threads = bt;
  *h_ctas_per_sm = bm;
  int r = hz_ensemble_set_launch(e, bt, bm);
  if (r == HZ_OK) r = hz_ensemble_set_primitives(e, d_prim);
  return r;
}

}  // extern "C"
