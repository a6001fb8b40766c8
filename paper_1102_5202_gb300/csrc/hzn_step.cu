// hzn_step.cu -- fused finite-volume substep kernels and the C-ABI of libhzn (sm_103a).
//
// One launch performs one Runge-Kutta substep (§3.2) for every cell: MC reconstruction of the
// primitive state to the faces, face metric, HLLE flux (§2.2), flux divergence and metric
// source (§2.1 Eq. 2), the RK stage combination, the Newton recovery of the new primitive
// state (§2.2) and, after the last substep, the maximum characteristic speed for the next
// time step (a warp-shuffle / atomic max).  Paper prior art (§3.3): thread blocks of 32 cells
// along x marching in z, padded rows; here a block owns a TX x TY column tile and a chunk of z,
// keeps the face fluxes of a plane in shared memory, reuses each z-face between two planes,
// and computes every face exactly once per tile.
//
// Grid storage in the workspace: structure of arrays, x fastest, rows padded to 16 elements
// (128 bytes of FP64); the metric carries its ghost layer; primitive boundaries are applied as
// clamped (outflow) or wrapped (periodic) indices, so no primitive ghosts are stored.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#include <new>

#include "hzn.h"
#include "hzn_physics.cuh"

using namespace hzn;

namespace {

constexpr int NF = 9;  // fields of the primitive and conserved vectors

// Device-resident scalars: the time-step clock and the run statistics.
struct DevScalars {
  unsigned long long vmax_bits;  // max speed / dx of the newest state (bits of a positive double)
  unsigned long long fails;      // recovery failures since hz_set_primitives
  int maxit;                     // largest Newton iteration count
  int pad;
  double dt;                     // dt of the step in flight
  double t;                      // simulated time
  long long steps;
};

struct KParams {
  int nx, ny, nz;
  int bcx, bcy, bcz;
  int pitch;             // x pitch of the interior arrays
  long long plane;       // pitch * ny
  long long fs;          // field stride of the interior arrays
  int mpitch, mny;       // metric x pitch, metric y extent
  long long mplane;      // mpitch * mny
  long long ms;          // metric field stride
  int gx, gy, gz;        // metric ghost widths
  double idx, idy, idz;  // 1 / dx
  double gamma, gfac, ch, kappa;
  double rho_floor, rho_atm, p_floor, p_atm;
  int c2p_maxit;
  double c2p_tol;
  int zlen;              // cells of z per block
};

struct StageArgs {
  const double* Pin;
  double* Pout;
  const double* U0;
  const double* Uk;
  double* Uout;
  double a0, ak;         // Uout = a0 U0 + ak (Uk + dt L)
  int last;              // 1 on the last substep: accumulate the CFL maximum
};

__device__ __forceinline__ int bc_index(int q, int n, int periodic) {
  if (periodic) {
    q = q < 0 ? q + n : q;
    q = q >= n ? q - n : q;
    return q;
  }
  return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

__device__ __forceinline__ long long met_off(const KParams& kp, int i, int j, int k) {
  return (long long)(k + kp.gz) * kp.mplane + (long long)(j + kp.gy) * kp.mpitch + (i + kp.gx);
}

__device__ __forceinline__ void load_metric(const KParams& kp, const double* __restrict__ M,
                                            long long off, double m[10]) {
#pragma unroll
  for (int f = 0; f < 10; ++f) m[f] = __ldg(M + f * kp.ms + off);
}

__device__ __forceinline__ Consts<double> consts_of(const KParams& kp) {
  Consts<double> c;
  c.gamma = kp.gamma;
  c.gfac = kp.gfac;
  c.ch2 = kp.ch * kp.ch;
  return c;
}

// HLLE flux of the face at i - 1/2 along D of cell (i, j, k) (the face between cells i-1 and
// i along D), written to out[f * ostride].
template <int D, bool CLEAN>
__device__ __forceinline__ void face_flux(const KParams& kp, const double* __restrict__ P,
                                          const double* __restrict__ M, int i, int j, int k,
                                          double* out, int ostride) {
  constexpr int NV = CLEAN ? 9 : 8;
  // stencil cells s = -2 .. 1 along D
  long long off[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int ii = i, jj = j, kk = k;
    if (D == 0) ii = bc_index(i + s - 2, kp.nx, kp.bcx);
    if (D == 1) jj = bc_index(j + s - 2, kp.ny, kp.bcy);
    if (D == 2) kk = bc_index(k + s - 2, kp.nz, kp.bcz);
    off[s] = (long long)kk * kp.plane + (long long)jj * kp.pitch + ii;
  }
  double PL[9], PR[9];
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    const double* pf = P + f * kp.fs;
    const double a = __ldg(pf + off[0]), b = __ldg(pf + off[1]);
    const double cc = __ldg(pf + off[2]), d = __ldg(pf + off[3]);
    PL[f] = b + 0.5 * mc_slope(b - a, cc - b);
    PR[f] = cc - 0.5 * mc_slope(cc - b, d - cc);
  }
  if (!CLEAN) PL[8] = PR[8] = 0.0;
  // face metric: mean of the two adjacent centre values
  double m[10];
  {
    const long long o1 = met_off(kp, i, j, k);
    const long long o0 = o1 - (D == 0 ? 1 : (D == 1 ? kp.mpitch : kp.mplane));
#pragma unroll
    for (int f = 0; f < 10; ++f) m[f] = 0.5 * (__ldg(M + f * kp.ms + o0) + __ldg(M + f * kp.ms + o1));
  }
  const Geom<double> G = make_geom(m);
  const Consts<double> c = consts_of(kp);
  double FL[9], UL[9], lmL, lpL;
  {
    const State<double> S = make_state(G, PL, c);
    flux_of<D, CLEAN>(G, S, c, FL);
    cons_of<CLEAN>(G, S, UL);
    speeds_of<D>(G, S, cms2_of(S, c), lmL, lpL);
  }
  double FR[9], UR[9], lmR, lpR;
  {
    const State<double> S = make_state(G, PR, c);
    flux_of<D, CLEAN>(G, S, c, FR);
    cons_of<CLEAN>(G, S, UR);
    speeds_of<D>(G, S, cms2_of(S, c), lmR, lpR);
  }
  const double sl = fmin(0.0, fmin(lmL, lmR));
  const double sr = fmax(0.0, fmax(lpL, lpR));
  const double den = sr - sl;
  const double iden = den != 0.0 ? 1.0 / den : 0.0;
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    double v;
    if (den != 0.0) v = (sr * FL[f] - sl * FR[f] + sl * sr * (UR[f] - UL[f])) * iden;
    else v = 0.5 * (FL[f] + FR[f]);
    out[f * ostride] = v;
  }
  if (CLEAN) {
    double cm, cp;
    clean_speeds<D>(G, kp.ch, cm, cp);
    const double csl = fmin(0.0, cm), csr = fmax(0.0, cp);
    const double cden = csr - csl;
    const int fb = U_BX + D;
    if (cden != 0.0) {
      const double ic = 1.0 / cden;
      out[fb * ostride] = (csr * FL[fb] - csl * FR[fb] + csl * csr * (UR[fb] - UL[fb])) * ic;
      out[U_PSI * ostride] = (csr * FL[U_PSI] - csl * FR[U_PSI] + csl * csr * (UR[U_PSI] - UL[U_PSI])) * ic;
    }
  }
}

// Centre 4-metric quantities used by the source: g_tt, beta_i, gamma_ij at one cell.
struct G4 {
  double gtt, blx, bly, blz, gxx, gxy, gxz, gyy, gyz, gzz;
};

__device__ __forceinline__ G4 g4_at(const KParams& kp, const double* __restrict__ M, long long off) {
  double m[10];
  load_metric(kp, M, off, m);
  G4 g;
  g.gxx = m[M_GXX];
  g.gxy = m[M_GXY];
  g.gxz = m[M_GXZ];
  g.gyy = m[M_GYY];
  g.gyz = m[M_GYZ];
  g.gzz = m[M_GZZ];
  g.blx = g.gxx * m[M_BX] + g.gxy * m[M_BY] + g.gxz * m[M_BZ];
  g.bly = g.gxy * m[M_BX] + g.gyy * m[M_BY] + g.gyz * m[M_BZ];
  g.blz = g.gxz * m[M_BX] + g.gyz * m[M_BY] + g.gzz * m[M_BZ];
  g.gtt = -m[M_ALP] * m[M_ALP] + (g.blx * m[M_BX] + g.bly * m[M_BY] + g.blz * m[M_BZ]);
  return g;
}

// Contravariant stress-energy T^{ab} = (w + b^2) u^a u^b + (p + b^2/2) g^{ab} - b^a b^b.
struct Tup {
  double tt, tx, ty, tz, xx, xy, xz, yy, yz, zz;
};

__device__ __forceinline__ Tup tup_of(const Geom<double>& G, const State<double>& S) {
  const double wt = S.w + S.b2, pt = S.p + 0.5 * S.b2;
  const double ia2 = G.ialp * G.ialp;
  Tup T;
  const double u[4] = {S.ut, S.ux, S.uy, S.uz};
  const double b[4] = {S.bt, S.bx, S.by, S.bz};
  const double gut = -ia2;
  const double gtx = G.bx * ia2, gty = G.by * ia2, gtz = G.bz * ia2;
  T.tt = wt * u[0] * u[0] + pt * gut - b[0] * b[0];
  T.tx = wt * u[0] * u[1] + pt * gtx - b[0] * b[1];
  T.ty = wt * u[0] * u[2] + pt * gty - b[0] * b[2];
  T.tz = wt * u[0] * u[3] + pt * gtz - b[0] * b[3];
  T.xx = wt * u[1] * u[1] + pt * (G.ixx - G.bx * G.bx * ia2) - b[1] * b[1];
  T.xy = wt * u[1] * u[2] + pt * (G.ixy - G.bx * G.by * ia2) - b[1] * b[2];
  T.xz = wt * u[1] * u[3] + pt * (G.ixz - G.bx * G.bz * ia2) - b[1] * b[3];
  T.yy = wt * u[2] * u[2] + pt * (G.iyy - G.by * G.by * ia2) - b[2] * b[2];
  T.yz = wt * u[2] * u[3] + pt * (G.iyz - G.by * G.bz * ia2) - b[2] * b[3];
  T.zz = wt * u[3] * u[3] + pt * (G.izz - G.bz * G.bz * ia2) - b[3] * b[3];
  return T;
}

// T^{ab} d g_ab for centred differences between the neighbours gp and gm (unscaled).
__device__ __forceinline__ double tdg(const Tup& T, const G4& gp, const G4& gm) {
  return T.tt * (gp.gtt - gm.gtt) +
         2.0 * (T.tx * (gp.blx - gm.blx) + T.ty * (gp.bly - gm.bly) + T.tz * (gp.blz - gm.blz)) +
         T.xx * (gp.gxx - gm.gxx) + T.yy * (gp.gyy - gm.gyy) + T.zz * (gp.gzz - gm.gzz) +
         2.0 * (T.xy * (gp.gxy - gm.gxy) + T.xz * (gp.gxz - gm.gxz) + T.yz * (gp.gyz - gm.gyz));
}

// max over active axes of max|lambda| / dx at a cell centre (plus the cleaning speed).
template <bool YA, bool ZA, bool CLEAN>
__device__ __forceinline__ double cell_max_speed(const KParams& kp, const Geom<double>& G,
                                                 const double P[9], const Consts<double>& c) {
  const State<double> S = make_state(G, P, c);
  const double c2 = cms2_of(S, c);
  double v = 0.0, lm, lp;
  speeds_of<0>(G, S, c2, lm, lp);
  v = fmax(fabs(lm), fabs(lp)) * kp.idx;
  if (CLEAN) {
    clean_speeds<0>(G, kp.ch, lm, lp);
    v = fmax(v, fmax(fabs(lm), fabs(lp)) * kp.idx);
  }
  if (YA) {
    speeds_of<1>(G, S, c2, lm, lp);
    v = fmax(v, fmax(fabs(lm), fabs(lp)) * kp.idy);
    if (CLEAN) {
      clean_speeds<1>(G, kp.ch, lm, lp);
      v = fmax(v, fmax(fabs(lm), fabs(lp)) * kp.idy);
    }
  }
  if (ZA) {
    speeds_of<2>(G, S, c2, lm, lp);
    v = fmax(v, fmax(fabs(lm), fabs(lp)) * kp.idz);
    if (CLEAN) {
      clean_speeds<2>(G, kp.ch, lm, lp);
      v = fmax(v, fmax(fabs(lm), fabs(lp)) * kp.idz);
    }
  }
  return v;
}

// Block reduction of the CFL maximum, the failure count and the largest iteration count.
template <int NT>
__device__ __forceinline__ void block_stats(DevScalars* sc, double vloc, int nfail, int maxit,
                                            bool want_v) {
  __shared__ double sv[NT / 32];
  __shared__ int sf[NT / 32], si[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    vloc = fmax(vloc, __shfl_xor_sync(0xffffffffu, vloc, o));
    nfail += __shfl_xor_sync(0xffffffffu, nfail, o);
    maxit = max(maxit, __shfl_xor_sync(0xffffffffu, maxit, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sv[w] = vloc;
    sf[w] = nfail;
    si[w] = maxit;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    int nf = 0, mi = 0;
    for (int q = 0; q < NT / 32; ++q) {
      v = fmax(v, sv[q]);
      nf += sf[q];
      mi = max(mi, si[q]);
    }
    if (want_v && v > 0.0) atomicMax(&sc->vmax_bits, (unsigned long long)__double_as_longlong(v));
    if (nf) atomicAdd(&sc->fails, (unsigned long long)nf);
    if (mi) atomicMax(&sc->maxit, mi);
  }
}

// Recovery with atmosphere / floor handling; rewrites U when the cell is reset.
template <bool CLEAN>
__device__ __forceinline__ int recover(const KParams& kp, const Geom<double>& G, double U[9],
                                       const double Pg[9], const Consts<double>& c, double P[9],
                                       int& iters) {
  // atmosphere: a cell whose rest-mass density D / sqrt(gamma) = rho W is below rho_atm is not
  // recovered but set to the atmosphere state (the decision uses the conserved state only)
  const bool atm = U[U_D] < kp.rho_atm * G.sqrtg;
  C2PResult r = {1, 0};
  if (!atm) r = con2prim<CLEAN>(G, U, Pg, c, kp.c2p_maxit, kp.c2p_tol, P);
  iters = r.iters;
  bool reset = false;
  if (atm || !r.ok || P[P_RHO] < kp.rho_floor) {
    const double isg = 1.0 / G.sqrtmg;
    P[P_BX] = U[U_BX] * isg;
    P[P_BY] = U[U_BY] * isg;
    P[P_BZ] = U[U_BZ] * isg;
    P[P_PSI] = CLEAN ? U[U_PSI] / G.sqrtg : 0.0;
    P[P_RHO] = kp.rho_floor;
    P[P_PRS] = kp.p_atm;
    P[P_UX] = P[P_UY] = P[P_UZ] = 0.0;
    reset = true;
  } else if (P[P_PRS] < kp.p_floor) {
    P[P_PRS] = kp.p_floor;
    reset = true;
  }
  if (reset) {
    const State<double> S = make_state(G, P, c);
    cons_of<CLEAN>(G, S, U);
  }
  return r.ok ? 0 : 1;
}

template <int TX, int TY, bool YA, bool ZA, bool CLEAN>
__global__ void __launch_bounds__(TX * TY, 2)
k_substep(const KParams kp, const StageArgs sa, const double* __restrict__ M, DevScalars* sc) {
  constexpr int NT = TX * TY;
  constexpr int NV = CLEAN ? 9 : 8;
  __shared__ double fx[NV][TY][TX + 1];
  __shared__ double fy[YA ? NV : 1][YA ? TY + 1 : 1][TX];
  __shared__ double fz[ZA ? 2 : 1][ZA ? NV : 1][TY][TX];

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const int kz0 = blockIdx.z * kp.zlen;
  const int kz1 = min(kz0 + kp.zlen, kp.nz);
  const bool own = i < kp.nx && j < kp.ny;
  const double dt = sc->dt;
  const Consts<double> c = consts_of(kp);
  const double* __restrict__ P = sa.Pin;

  double vloc = 0.0;
  int nfail = 0, maxit = 0;

  if (ZA && own) face_flux<2, CLEAN>(kp, P, M, i, j, kz0, &fz[kz0 & 1][0][ty][tx], TY * TX);

  for (int k = kz0; k < kz1; ++k) {
    // ---- faces of plane k: each face of the tile once
    if (i <= kp.nx && j < kp.ny) face_flux<0, CLEAN>(kp, P, M, i, j, k, &fx[0][ty][tx], TY * (TX + 1));
    if (YA && i < kp.nx && j <= kp.ny) face_flux<1, CLEAN>(kp, P, M, i, j, k, &fy[0][ty][tx], (TY + 1) * TX);
    if (ZA && own) face_flux<2, CLEAN>(kp, P, M, i, j, k + 1, &fz[(k + 1) & 1][0][ty][tx], TY * TX);
    if (YA) {
      // top row of y-faces of the tile: warp 0; right column of x-faces: warp 1
      if (threadIdx.x < TX) {
        const int ii = i0 + threadIdx.x, jj = j0 + TY;
        if (ii < kp.nx && jj <= kp.ny)
          face_flux<1, CLEAN>(kp, P, M, ii, jj, k, &fy[0][TY][threadIdx.x], (TY + 1) * TX);
      } else if (threadIdx.x >= 32 && threadIdx.x < 32 + TY) {
        const int jj = j0 + (threadIdx.x - 32), ii = i0 + TX;
        if (ii <= kp.nx && jj < kp.ny)
          face_flux<0, CLEAN>(kp, P, M, ii, jj, k, &fx[0][threadIdx.x - 32][TX], TY * (TX + 1));
      }
    } else if (threadIdx.x < TY) {
      const int jj = j0 + threadIdx.x, ii = i0 + TX;
      if (ii <= kp.nx && jj < kp.ny)
        face_flux<0, CLEAN>(kp, P, M, ii, jj, k, &fx[0][threadIdx.x][TX], TY * (TX + 1));
    }
    __syncthreads();

    // ---- cell update of plane k
    if (own) {
      const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
      const long long mo = met_off(kp, i, j, k);
      double L[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        double v = -(fx[f][ty][tx + 1] - fx[f][ty][tx]) * kp.idx;
        if (YA) v -= (fy[f][ty + 1][tx] - fy[f][ty][tx]) * kp.idy;
        if (ZA) v -= (fz[(k + 1) & 1][f][ty][tx] - fz[k & 1][f][ty][tx]) * kp.idz;
        L[f] = v;
      }
      // metric source 1/2 sqrt(-g) T^{ab} d_i g_ab (static metric: no energy source)
      double mc[10];
      load_metric(kp, M, mo, mc);
      const Geom<double> G = make_geom(mc);
      double Pc[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) Pc[f] = __ldg(P + f * kp.fs + off);
      if (!CLEAN) Pc[8] = 0.0;
      {
        const State<double> S = make_state(G, Pc, c);
        const Tup T = tup_of(G, S);
        const double h = 0.5 * G.sqrtmg;
        {
          const G4 gp = g4_at(kp, M, mo + 1), gm = g4_at(kp, M, mo - 1);
          L[U_TX] += h * tdg(T, gp, gm) * (0.5 * kp.idx);
        }
        if (YA) {
          const G4 gp = g4_at(kp, M, mo + kp.mpitch), gm = g4_at(kp, M, mo - kp.mpitch);
          L[U_TY] += h * tdg(T, gp, gm) * (0.5 * kp.idy);
        }
        if (ZA) {
          const G4 gp = g4_at(kp, M, mo + kp.mplane), gm = g4_at(kp, M, mo - kp.mplane);
          L[U_TZ] += h * tdg(T, gp, gm) * (0.5 * kp.idz);
        }
        if (CLEAN) L[U_PSI] += -kp.kappa * G.alp * (G.sqrtg * S.psi);
      }
      // Runge-Kutta stage
      double U[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        const double uk = sa.Uk[f * kp.fs + off];
        U[f] = sa.ak * (uk + dt * L[f]);
        if (sa.a0 != 0.0) U[f] += sa.a0 * sa.U0[f * kp.fs + off];
      }
      if (!CLEAN) U[8] = 0.0;
      // recovery of the new primitive state
      double Pn[9];
      int it;
      nfail += recover<CLEAN>(kp, G, U, Pc, c, Pn, it);
      maxit = max(maxit, it);
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        sa.Uout[f * kp.fs + off] = U[f];
        sa.Pout[f * kp.fs + off] = Pn[f];
      }
      if (sa.last) vloc = fmax(vloc, cell_max_speed<YA, ZA, CLEAN>(kp, G, Pn, c));
    }
    __syncthreads();
  }
  block_stats<NT>(sc, vloc, nfail, maxit, sa.last != 0);
}

// Conserved state from the primitive state, per cell.
template <bool CLEAN>
__global__ void k_prim2cons(const KParams kp, const double* __restrict__ P, const double* __restrict__ M,
                            double* __restrict__ U) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const Consts<double> c = consts_of(kp);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % kp.nx);
    const int j = (int)((q / kp.nx) % kp.ny);
    const int k = (int)(q / ((long long)kp.nx * kp.ny));
    const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    double m[10], Pc[9], Uc[9];
    load_metric(kp, M, met_off(kp, i, j, k), m);
#pragma unroll
    for (int f = 0; f < 9; ++f) Pc[f] = P[f * kp.fs + off];
    if (!CLEAN) Pc[8] = 0.0;
    const Geom<double> G = make_geom(m);
    const State<double> S = make_state(G, Pc, c);
    cons_of<CLEAN>(G, S, Uc);
    if (!CLEAN) Uc[8] = 0.0;
#pragma unroll
    for (int f = 0; f < 9; ++f) U[f * kp.fs + off] = Uc[f];
  }
}

template <bool YA, bool ZA, bool CLEAN>
__global__ void __launch_bounds__(256) k_max_speed(const KParams kp, const double* __restrict__ P,
                                                   const double* __restrict__ M, DevScalars* sc) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const Consts<double> c = consts_of(kp);
  double v = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % kp.nx);
    const int j = (int)((q / kp.nx) % kp.ny);
    const int k = (int)(q / ((long long)kp.nx * kp.ny));
    const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    double m[10], Pc[9];
    load_metric(kp, M, met_off(kp, i, j, k), m);
#pragma unroll
    for (int f = 0; f < 9; ++f) Pc[f] = P[f * kp.fs + off];
    if (!CLEAN) Pc[8] = 0.0;
    const Geom<double> G = make_geom(m);
    v = fmax(v, cell_max_speed<YA, ZA, CLEAN>(kp, G, Pc, c));
  }
  block_stats<256>(sc, v, 0, 0, true);
}

// Copy between the caller's unpadded field-major layout and the padded workspace layout.
__global__ void k_pack(const KParams kp, const double* __restrict__ src, double* __restrict__ dst,
                       int nfield, int to_internal, int zero_from) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * nfield;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / n);
    const long long r = q % n;
    const int i = (int)(r % kp.nx);
    const int j = (int)((r / kp.nx) % kp.ny);
    const int k = (int)(r / ((long long)kp.nx * kp.ny));
    const long long off = f * kp.fs + (long long)k * kp.plane + (long long)j * kp.pitch + i;
    if (to_internal) dst[off] = f >= zero_from ? 0.0 : src[q];
    else dst[q] = f >= zero_from ? 0.0 : src[off];
  }
}

__global__ void k_pack_metric(const KParams kp, const double* __restrict__ src, double* __restrict__ dst) {
  const int mx = kp.nx + 2 * kp.gx, my = kp.ny + 2 * kp.gy, mz = kp.nz + 2 * kp.gz;
  const long long n = (long long)mx * my * mz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * 10;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / n);
    const long long r = q % n;
    const int i = (int)(r % mx);
    const int j = (int)((r / mx) % my);
    const int k = (int)(r / ((long long)mx * my));
    dst[f * kp.ms + (long long)k * kp.mplane + (long long)j * kp.mpitch + i] = src[q];
  }
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

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// ----------------------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------------------
struct hz_ctx {
  hz_grid g;
  hz_options o;
  cudaStream_t st;
  KParams kp;
  char* ws;
  size_t wsbytes;
  DevScalars* sc;
  double* met;
  double* U0;
  double* U1;
  double* P[2];
  int cur;
  int have_metric, have_prim;
  int dims;       // 1, 2 or 3: highest active axis + 1 pattern
  dim3 grid3;
  int block;
};

namespace {

struct Layout {
  size_t scal, met, fs_bytes, total;
  long long fs, ms;
  int pitch, mpitch, mny;
  long long plane, mplane;
};

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
  if (o->precision != HZ_FP64 && o->precision != HZ_MIXED) return HZ_ERR_ARG;
  if (o->precision == HZ_MIXED) return HZ_ERR_UNSUPPORTED;
  if (o->cleaning != 0 && o->cleaning != 1) return HZ_ERR_ARG;
  if (o->cleaning && (!(o->ch > 0.0) || o->ch > 1.0 || !(o->kappa >= 0.0))) return HZ_ERR_ARG;
  if (!(o->rho_floor > 0.0) || !(o->p_floor > 0.0) || !(o->atm_K >= 0.0)) return HZ_ERR_ARG;
  if (!(o->rho_atm >= 0.0)) return HZ_ERR_ARG;
  if (o->c2p_maxit < 1 || o->c2p_maxit > 200) return HZ_ERR_ARG;
  if (!(o->c2p_tol >= 1e-15) || o->c2p_tol > 1e-6) return HZ_ERR_ARG;
  return HZ_OK;
}

Layout layout_of(const hz_grid* g) {
  Layout L;
  const int gx = g->n[0] > 1, gy = g->n[1] > 1, gz = g->n[2] > 1;
  L.pitch = (int)round_up((size_t)g->n[0], 16);
  L.plane = (long long)L.pitch * g->n[1];
  L.fs = (long long)round_up((size_t)(L.plane * g->n[2]), 32);
  L.mpitch = (int)round_up((size_t)(g->n[0] + 2 * gx), 16);
  L.mny = g->n[1] + 2 * gy;
  L.mplane = (long long)L.mpitch * L.mny;
  L.ms = (long long)round_up((size_t)(L.mplane * (g->n[2] + 2 * gz)), 32);
  L.scal = 256;
  L.met = (size_t)L.ms * 10 * sizeof(double);
  L.fs_bytes = (size_t)L.fs * NF * sizeof(double);
  L.total = L.scal + L.met + 4 * L.fs_bytes;  // U0, U1, P[0], P[1]
  return L;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? HZ_OK : HZ_ERR_CUDA; }

int grid_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

template <bool YA, bool ZA>
void launch_max_speed_t(hz_ctx* c, const double* P) {
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  if (c->o.cleaning)
    k_max_speed<YA, ZA, true><<<grid_blocks(n, 256), 256, 0, c->st>>>(c->kp, P, c->met, c->sc);
  else
    k_max_speed<YA, ZA, false><<<grid_blocks(n, 256), 256, 0, c->st>>>(c->kp, P, c->met, c->sc);
}

void launch_max_speed(hz_ctx* c, const double* P) {
  if (c->dims == 1) launch_max_speed_t<false, false>(c, P);
  else if (c->dims == 2) launch_max_speed_t<true, false>(c, P);
  else launch_max_speed_t<true, true>(c, P);
}

template <int TX, int TY, bool YA, bool ZA>
void launch_substep_t(hz_ctx* c, const StageArgs& sa) {
  dim3 grid((c->g.n[0] + TX - 1) / TX, (c->g.n[1] + TY - 1) / TY, c->grid3.z);
  if (c->o.cleaning)
    k_substep<TX, TY, YA, ZA, true><<<grid, TX * TY, 0, c->st>>>(c->kp, sa, c->met, c->sc);
  else
    k_substep<TX, TY, YA, ZA, false><<<grid, TX * TY, 0, c->st>>>(c->kp, sa, c->met, c->sc);
}

void launch_substep(hz_ctx* c, const StageArgs& sa) {
  if (c->dims == 1) launch_substep_t<128, 1, false, false>(c, sa);
  else if (c->dims == 2) launch_substep_t<32, 4, true, false>(c, sa);
  else launch_substep_t<32, 4, true, true>(c, sa);
}

int run_step(hz_ctx* c, int mode, double dt, double cfl, double t_end) {
  if (!c->have_metric || !c->have_prim) return HZ_ERR_STATE;
  k_clock<<<1, 1, 0, c->st>>>(c->sc, mode, dt, cfl, t_end);
  const int a = c->cur, b = 1 - c->cur;
  StageArgs s1 = {c->P[a], c->P[b], c->U0, c->U0, c->U1, 0.0, 1.0, 0};
  StageArgs s2 = {c->P[b], c->P[a], c->U0, c->U1, c->U1, 0.75, 0.25, 0};
  StageArgs s3 = {c->P[a], c->P[b], c->U0, c->U1, c->U0, 1.0 / 3.0, 2.0 / 3.0, 1};
  launch_substep(c, s1);
  launch_substep(c, s2);
  launch_substep(c, s3);
  c->cur = b;
  return cuda_err(cudaGetLastError());
}

// Fill a context for a checked grid and options over a workspace of at least layout_of().total
// bytes, and clear the device scalars on the stream.
int ctx_init(hz_ctx* c, const hz_grid* grid, const hz_options* opts, void* d_workspace,
             size_t bytes, void* stream) {
  const Layout L = layout_of(grid);
  memset(c, 0, sizeof(*c));
  c->g = *grid;
  c->o = *opts;
  c->st = (cudaStream_t)stream;
  c->ws = (char*)d_workspace;
  c->wsbytes = bytes;
  c->sc = (DevScalars*)c->ws;
  c->met = (double*)(c->ws + L.scal);
  char* p = c->ws + L.scal + L.met;
  c->U0 = (double*)p;
  c->U1 = (double*)(p + L.fs_bytes);
  c->P[0] = (double*)(p + 2 * L.fs_bytes);
  c->P[1] = (double*)(p + 3 * L.fs_bytes);
  c->cur = 0;
  c->dims = grid->n[2] > 1 ? 3 : (grid->n[1] > 1 ? 2 : 1);

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
  double patm = opts->atm_K > 0.0 ? opts->atm_K * pow(opts->rho_floor, opts->gamma) : opts->p_floor;
  kp.p_atm = patm < opts->p_floor ? opts->p_floor : patm;
  kp.c2p_maxit = opts->c2p_maxit;
  kp.c2p_tol = opts->c2p_tol;
  // z chunks: enough blocks for several waves on 152 SMs
  int tiles_xy;
  if (c->dims == 1) tiles_xy = (kp.nx + 127) / 128;
  else tiles_xy = ((kp.nx + 31) / 32) * ((kp.ny + 3) / 4);
  int chunks = 1;
  if (c->dims == 3) {
    const int want = 152 * 2 * 4;
    chunks = (want + tiles_xy - 1) / tiles_xy;
    if (chunks > kp.nz) chunks = kp.nz;
    if (chunks < 1) chunks = 1;
  }
  kp.zlen = (kp.nz + chunks - 1) / chunks;
  c->grid3 = dim3(1, 1, (kp.nz + kp.zlen - 1) / kp.zlen);

  k_reset_scalars<<<1, 1, 0, c->st>>>(c->sc);
  return cuda_err(cudaGetLastError());
}

}  // namespace

extern "C" {

int hz_version(void) { return HZN_VERSION; }

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
  *bytes = layout_of(grid).total;
  return HZ_OK;
}

int hz_create(hz_ctx** ctx, const hz_grid* grid, const hz_options* opts, void* d_workspace,
              size_t bytes, void* stream) {
  if (!ctx) return HZ_ERR_ARG;
  *ctx = nullptr;
  int e = check_args(grid, opts);
  if (e != HZ_OK) return e;
  const Layout L = layout_of(grid);
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
  k_pack_metric<<<grid_blocks(n * 10, 256), 256, 0, c->st>>>(c->kp, d_metric, c->met);
  c->have_metric = 1;
  return cuda_err(cudaGetLastError());
}

int hz_set_primitives(hz_ctx* c, const double* d_prim) {
  if (!c || !d_prim) return HZ_ERR_ARG;
  if (!c->have_metric) return HZ_ERR_STATE;
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  c->cur = 0;
  k_pack<<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, d_prim, c->P[0], NF, 1, c->o.cleaning ? NF : 8);
  if (c->o.cleaning)
    k_prim2cons<true><<<grid_blocks(n, 256), 256, 0, c->st>>>(c->kp, c->P[0], c->met, c->U0);
  else
    k_prim2cons<false><<<grid_blocks(n, 256), 256, 0, c->st>>>(c->kp, c->P[0], c->met, c->U0);
  // the second primitive buffer and U1 start as copies so that inactive fields stay defined
  cudaMemcpyAsync(c->P[1], c->P[0], (size_t)c->kp.fs * NF * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->U1, c->U0, (size_t)c->kp.fs * NF * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  k_reset_scalars<<<1, 1, 0, c->st>>>(c->sc);
  launch_max_speed(c, c->P[0]);
  c->have_prim = 1;
  return cuda_err(cudaGetLastError());
}

int hz_get_primitives(hz_ctx* c, double* d_prim) {
  if (!c || !d_prim) return HZ_ERR_ARG;
  if (!c->have_prim) return HZ_ERR_STATE;
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  k_pack<<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, c->P[c->cur], d_prim, NF, 0, c->o.cleaning ? NF : 8);
  return cuda_err(cudaGetLastError());
}

int hz_get_conserved(hz_ctx* c, double* d_cons) {
  if (!c || !d_cons) return HZ_ERR_ARG;
  if (!c->have_prim) return HZ_ERR_STATE;
  const long long n = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  k_pack<<<grid_blocks(n * NF, 256), 256, 0, c->st>>>(c->kp, c->U0, d_cons, NF, 0, c->o.cleaning ? NF : 8);
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
  launch_max_speed(c, c->P[c->cur]);
  unsigned long long bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, &c->sc->vmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return HZ_ERR_CUDA;
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
  if (e != cudaSuccess) return HZ_ERR_CUDA;
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
#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = HZ_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices];  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device (looked up on first use).
int noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HZ_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return HZ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HZ_ERR_CUDA;
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
  if (layout_of(grid).total > kNoallocScratchBytes) return HZ_ERR_TOO_LARGE;
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
  return hz_get_primitives(&c, d_prim_out);
}
