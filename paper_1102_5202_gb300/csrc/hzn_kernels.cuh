// hzn_kernels.cuh -- the fused finite-volume substep kernel and its helpers (templates).
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
// Precision (§3.2 lists SP, DP and DP-only recovery; §6 adjustable flux-difference precision):
//   FP64 path   every step in double;
//   mixed path  primitives and metric stored in float; reconstruction, face fluxes, HLLE and
//               sources in float with the flux divergence accumulated in float; the RK update
//               of the conserved state (stored in double), the recovery and the CFL maximum
//               in double;
//   pair path   the FP64 path's storage, update, recovery and CFL maximum, with
//               reconstruction, face states, fluxes, HLLE, divergence and sources in
//               double-word arithmetic (hzn_f32x2.cuh) on the FP32 pipes.
//
// Grid storage: structure of arrays, x fastest, rows padded to 16 elements; the metric carries
// its ghost layer; primitive boundaries are applied as clamped (outflow) or wrapped (periodic)
// indices, so no primitive ghosts are stored.
#pragma once

#include "hzn_f32x2.cuh"
#include "hzn_internal.h"
#include "hzn_physics.cuh"

namespace hzn {

template <bool MIXED>
struct Prec;
template <>
struct Prec<false> {
  using R = double;  // face / source arithmetic
  using S = double;  // storage of primitives and metric
};
template <>
struct Prec<true> {
  using R = float;
  using S = float;
};

// Arithmetic type of the face, flux and source work: the precision's own, or double-word
// (f32x2) over the FP64 state for the pair path.
template <bool PAIR, bool MIXED>
struct FaceType {
  using R = typename Prec<MIXED>::R;
};
template <>
struct FaceType<true, false> {
  using R = f32x2;
};

template <typename A, typename B>
struct SameType {
  static constexpr bool value = false;
};
template <typename A>
struct SameType<A, A> {
  static constexpr bool value = true;
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

template <typename R>
__device__ __forceinline__ Consts<R> consts_of(const KParams& kp) {
  Consts<R> c;
  if constexpr (SameType<R, float>::value) {
    c.gamma = kp.f_gamma;
    c.gfac = kp.f_gfac;
    c.ch = kp.f_ch;
    c.ch2 = kp.f_ch2;
  } else {
    c.gamma = cvt<R>(kp.gamma);
    c.gfac = cvt<R>(kp.gfac);
    c.ch = cvt<R>(kp.ch);
    c.ch2 = cvt<R>(kp.ch * kp.ch);
  }
  return c;
}

// A KParams constant in the face arithmetic's type: its FP32 copy for float.
template <typename R>
__device__ __forceinline__ R kconst(double d, float f) {
  if constexpr (SameType<R, float>::value) return f;
  else return cvt<R>(d);
}

// The ten metric values at one cell (only alpha and the diagonal for DIAG).
template <bool DIAG, typename R, typename S>
__device__ __forceinline__ void load_metric(const KParams& kp, const S* __restrict__ M, long long off,
                                            R m[10]) {
  if constexpr (DIAG) {
    m[M_ALP] = ldc<R>(M + M_ALP * kp.ms + off);
    m[M_GXX] = ldc<R>(M + M_GXX * kp.ms + off);
    m[M_GYY] = ldc<R>(M + M_GYY * kp.ms + off);
    m[M_GZZ] = ldc<R>(M + M_GZZ * kp.ms + off);
    m[M_BX] = m[M_BY] = m[M_BZ] = m[M_GXY] = m[M_GXZ] = m[M_GYZ] = R(0);
  } else {
#pragma unroll
    for (int f = 0; f < 10; ++f) m[f] = ldc<R>(M + f * kp.ms + off);
  }
}

// The HLLE weights of an FP64 face from its two states' speed quadratics (speed_quadratic: the
// roots are (-b -+ sq) / A' with A' > 0).  The bounds sL = min(0, lambda-), sR = max(0,
// lambda+) are chosen by cross-multiplied comparisons and kept as fractions n / d (n = 0, d = 1
// for a bound clamped at 0); then wL = nR dL / Q, wR = -nL dR / Q and wU = nL nR / Q with
// Q = nR dL - nL dR, so one reciprocal serves the face.  The weights carry sqrt(-g) (the flux
// and conserved vectors are formed without it).
__device__ __forceinline__ void hlle_weights(double sqrtmg, double AL, double BL, double sqL, double AR,
                                             double BR, double sqR, double& wl, double& wr, double& wu) {
  const double nmL = -BL - sqL, nmR = -BR - sqR, npL = -BL + sqL, npR = -BR + sqR;
  const double dL = AL, dR = AR;
  const bool lowL = nmL * dR < nmR * dL;
  double nl = lowL ? nmL : nmR, dl = lowL ? dL : dR;
  if (!(nl < 0.0)) {
    nl = 0.0;
    dl = 1.0;
  }
  const bool highL = npL * dR > npR * dL;
  double nr = highL ? npL : npR, dr = highL ? dL : dR;
  if (!(nr > 0.0)) {
    nr = 0.0;
    dr = 1.0;
  }
  const double q = nr * dl - nl * dr;
  if (q != 0.0) {
    const double iq = sqrtmg * rcp_fast(q);
    wl = nr * dl * iq;
    wr = -nl * dr * iq;
    wu = nl * nr * iq;
  } else {
    wl = wr = 0.5 * sqrtmg;
    wu = 0.0;
  }
}

// One state's share of an FP64 HLLE face flux, added to acc: cf F + cu U with F the state's
// flux vector along D and U its conserved vector (both divided by sqrt(-g), §2.1 Eq. 2), the
// cleaning pair (B^D, Psi) excluded when cleaning is on.  HLLE is linear in F_L, F_R and
// U_R - U_L, so (cf, cu) = (wL, -wU) for the left state and (wR, wU) for the right; F and U
// are never formed: with k = cf u^D + cu u^t, m = (w + b^2) k and n = cf b^D + cu b^t,
//   D:   rho k
//   T_t: m u_t - n b_t + cu (p + b^2/2)
//   T_i: m u_i - n b_i + cf (p + b^2/2) delta_iD
//   B^j: cf (B^j u^D - B^D u^j) / u^t + cu B^j            (B^D: cu B^D without cleaning)
// and, on a general metric with cleaning, cf psi gamma^{Dj} on B^j (j != D).
template <int D, bool CLEAN, bool DIAG, bool FIRST, typename R>
__device__ __forceinline__ void hlle_share(const Geom<R>& G, const State<R>& S, R cf, R cu,
                                           R acc[9]) {
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R bd = sel<D>(S.bx, S.by, S.bz);
  const R Bd = sel<D>(S.Bx, S.By, S.Bz);
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R k = cf * ud + cu * S.ut;
  const R m = wt * k;
  const R n = cf * bd + cu * S.bt;
  const R cfi = cf * S.iut;
  R v[9];
  v[U_D] = S.rho * k;
  v[U_TT] = m * S.l_t - n * S.b_t + cu * pt;
  v[U_TX] = m * S.lx - n * S.b_x + (D == 0 ? cf * pt : R(0));
  v[U_TY] = m * S.ly - n * S.b_y + (D == 1 ? cf * pt : R(0));
  v[U_TZ] = m * S.lz - n * S.b_z + (D == 2 ? cf * pt : R(0));
  v[U_BX] = D == 0 ? cu * S.Bx : cfi * (S.Bx * ud - Bd * S.ux) + cu * S.Bx;
  v[U_BY] = D == 1 ? cu * S.By : cfi * (S.By * ud - Bd * S.uy) + cu * S.By;
  v[U_BZ] = D == 2 ? cu * S.Bz : cfi * (S.Bz * ud - Bd * S.uz) + cu * S.Bz;
  if constexpr (CLEAN && !DIAG) {
    const R cp = cf * S.psi;
    if (D != 0) v[U_BX] += cp * sel<D>(G.ixx, G.ixy, G.ixz);
    if (D != 1) v[U_BY] += cp * sel<D>(G.ixy, G.iyy, G.iyz);
    if (D != 2) v[U_BZ] += cp * sel<D>(G.ixz, G.iyz, G.izz);
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (CLEAN && f == U_BX + D) continue;  // the cleaning pair has its own bounds
    acc[f] = FIRST ? v[f] : acc[f] + v[f];
  }
}

// HLLE flux (§2.2) of an FP64 or FP32 face, written to out[f * ostride]: both states' speeds,
// the HLLE weights, then each state's share (hlle_share).  FP64: the weights from the speed
// quadratics as fractions (hlle_weights); FP32: from the plain roots per state (the
// cross-multiplied comparisons of the fractions would leave the FP32 exponent range in
// near-vacuum cells).  The cleaning pair (B^D, Psi)
// takes HLLE at its own bounds; its flux and conserved components (divided by sqrt(-g)) are
// F_BD = psi gamma^DD, U_BD = B^D, F_Psi = (c_h^2 alpha^2 B^D - beta^D psi) / alpha and
// U_Psi = psi / alpha.  cfac: alpha sqrt(gamma^DD) at the face (DIAG with cleaning).
template <int D, bool CLEAN, bool DIAG, typename R>
__device__ __forceinline__ void hlle_face_fused(const Geom<R>& G, const R PL[9], const R PR[9],
                                                const Consts<R>& c, R cfac, R* out, int ostride) {
  const State<R> SL = make_state<DIAG>(G, PL, c);
  const State<R> SR = make_state<DIAG>(G, PR, c);
  R wl, wr, wu;
  if constexpr (SameType<R, double>::value) {
    double AL, BL, sqL, AR, BR, sqR;
    speed_quadratic<D, DIAG>(G, SL, c, AL, BL, sqL);
    speed_quadratic<D, DIAG>(G, SR, c, AR, BR, sqR);
    hlle_weights(G.sqrtmg, AL, BL, sqL, AR, BR, sqR, wl, wr, wu);
  } else {
    R lmL, lpL, lmR, lpR;
    speeds_of<D, DIAG>(G, SL, cms2_of(SL, c), lmL, lpL);
    speeds_of<D, DIAG>(G, SR, cms2_of(SR, c), lmR, lpR);
    const R sl = fmin(R(0), fmin(lmL, lmR));
    const R sr = fmax(R(0), fmax(lpL, lpR));
    const R den = sr - sl;
    if (den != R(0)) {
      const R iden = fdiv(G.sqrtmg, den);
      wl = sr * iden;
      wr = -sl * iden;
      wu = sl * sr * iden;
    } else {
      wl = wr = R(0.5) * G.sqrtmg;
      wu = R(0);
    }
  }
  R acc[9];
  hlle_share<D, CLEAN, DIAG, true>(G, SL, wl, R(-wu), acc);
  hlle_share<D, CLEAN, DIAG, false>(G, SR, wr, wu, acc);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (CLEAN && f == U_BX + D) continue;
    out[f * ostride] = acc[f];
  }
  if (CLEAN) {
    const int fb = U_BX + D;
    const R BdL = sel<D>(SL.Bx, SL.By, SL.Bz), BdR = sel<D>(SR.Bx, SR.By, SR.Bz);
    const R gdd = sel<D>(G.ixx, G.iyy, G.izz);
    if constexpr (DIAG) {
      // zero shift: bounds -+a, a = c_h alpha sqrt(gamma^DD): weights sqrt(-g)/2 per state and
      // a sqrt(-g)/2 for the jump
      const R hs = R(0.5) * G.sqrtmg, ha = hs * (c.ch * cfac);
      out[fb * ostride] = hs * (gdd * (SL.psi + SR.psi)) - ha * (BdR - BdL);
      out[U_PSI * ostride] = hs * (c.ch2 * G.alp * (BdL + BdR)) - ha * (G.ialp * (SR.psi - SL.psi));
    } else {
      const R bD = sel<D>(G.bx, G.by, G.bz);
      const R FbL = SL.psi * gdd, FbR = SR.psi * gdd;
      const R FpL = G.ialp * (c.ch2 * G.alp * G.alp * BdL - bD * SL.psi);
      const R FpR = G.ialp * (c.ch2 * G.alp * G.alp * BdR - bD * SR.psi);
      R cm, cp;
      clean_speeds<D, DIAG>(G, c.ch, cm, cp);
      const R csl = fmin(R(0), cm), csr = fmax(R(0), cp);
      const R cden = csr - csl;
      if (cden != R(0)) {
        const R ic = fdiv(G.sqrtmg, cden);
        out[fb * ostride] = (csr * FbL - csl * FbR + csl * csr * (BdR - BdL)) * ic;
        out[U_PSI * ostride] = (csr * FpL - csl * FpR + csl * csr * (G.ialp * (SR.psi - SL.psi))) * ic;
      } else {
        out[fb * ostride] = wl * FbL + (wr * FbR + wu * (BdR - BdL));
        out[U_PSI * ostride] = wl * FpL + (wr * FpR + wu * (G.ialp * (SR.psi - SL.psi)));
      }
    }
  }
}

// HLLE flux (§2.2) of one face from its reconstructed left / right primitive states and face
// geometry, written to out[f * ostride].  ROLL: one copy of the state code serves both states
// (a loop the compiler keeps rolled), which halves the code of the double-word path.  cfac:
// alpha sqrt(gamma^DD) at the face (used with cleaning on a DIAG metric).
template <int D, bool CLEAN, bool DIAG, bool ROLL, typename R>
__device__ __forceinline__ void hlle_face(const Geom<R>& G, const R PL[9], const R PR[9],
                                          const Consts<R>& c, R cfac, R* out, int ostride) {
  constexpr int NV = CLEAN ? 9 : 8;
  // wave speeds.  FP64: both states' quadratics, multiplied through by w (w + b^2); their roots
  // enter the HLLE weights as fractions, with one division per face.  FP32 (mixed) and
  // double-word: the plain quadratic per state, since A' scales like w^2 and the cross products
  // underflow the FP32 exponent range in near-vacuum cells.
  constexpr bool SHARED = SameType<R, double>::value && !ROLL;
  R FL[9], UL[9], AL, BL, sqL, lmL, lpL;
  R FR[9], UR[9], AR, BR, sqR, lmR, lpR;
  if constexpr (ROLL) {
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      R Pq[9];
#pragma unroll
      for (int f = 0; f < 9; ++f) Pq[f] = side == 0 ? PL[f] : PR[f];
      const State<R> St = make_state<DIAG>(G, Pq, c);
      R F[9], U[9], lm, lp;
      flux_of<D, CLEAN, DIAG, true>(G, St, c, F);
      cons_of<CLEAN, true>(G, St, U);
      speeds_of<D, DIAG>(G, St, cms2_of(St, c), lm, lp);
      if (side == 0) {
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          FL[f] = F[f];
          UL[f] = U[f];
        }
        lmL = lm;
        lpL = lp;
      } else {
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          FR[f] = F[f];
          UR[f] = U[f];
        }
        lmR = lm;
        lpR = lp;
      }
    }
  } else {
    {
      const State<R> St = make_state<DIAG>(G, PL, c);
      flux_of<D, CLEAN, DIAG, true>(G, St, c, FL);
      cons_of<CLEAN, true>(G, St, UL);
      if constexpr (SHARED) speed_quadratic<D, DIAG>(G, St, c, AL, BL, sqL);
      else speeds_of<D, DIAG>(G, St, cms2_of(St, c), lmL, lpL);
    }
    {
      const State<R> St = make_state<DIAG>(G, PR, c);
      flux_of<D, CLEAN, DIAG, true>(G, St, c, FR);
      cons_of<CLEAN, true>(G, St, UR);
      if constexpr (SHARED) speed_quadratic<D, DIAG>(G, St, c, AR, BR, sqR);
      else speeds_of<D, DIAG>(G, St, cms2_of(St, c), lmR, lpR);
    }
  }
  // HLLE: F = (sR FL - sL FR + sL sR (UR - UL)) / (sR - sL).  FL, FR, UL, UR are the vectors
  // divided by sqrt(-g) (the face's, common to both states), folded back into the weights.
  R wl, wr, wu;
  if constexpr (SHARED) {
    // The roots are (-b -+ sq) / A' with A' > 0.  The bounds sL = min(0, lambda-), sR =
    // max(0, lambda+) are chosen by cross-multiplied comparisons and kept as fractions n / d
    // (n = 0, d = 1 for a bound clamped at 0); then wL = nR dL / Q, wR = -nL dR / Q and
    // wU = nL nR / Q with Q = nR dL - nL dR, so one division serves the face.
    const R nmL = -BL - sqL, nmR = -BR - sqR, npL = -BL + sqL, npR = -BR + sqR;
    const R dL = AL, dR = AR;
    const bool lowL = nmL * dR < nmR * dL;
    R nl = lowL ? nmL : nmR, dl = lowL ? dL : dR;
    if (!(nl < R(0))) {
      nl = R(0);
      dl = R(1);
    }
    const bool highL = npL * dR > npR * dL;
    R nr = highL ? npL : npR, dr = highL ? dL : dR;
    if (!(nr > R(0))) {
      nr = R(0);
      dr = R(1);
    }
    const R q = nr * dl - nl * dr;
    if (q != R(0)) {
      const R iq = G.sqrtmg * rcp_fast(q);
      wl = nr * dl * iq;
      wr = -nl * dr * iq;
      wu = nl * nr * iq;
    } else {
      wl = wr = R(0.5) * G.sqrtmg;
      wu = R(0);
    }
  } else {
    const R sl = fmin(R(0), fmin(lmL, lmR));
    const R sr = fmax(R(0), fmax(lpL, lpR));
    const R den = sr - sl;
    if (den != R(0)) {
      const R iden = fdiv(G.sqrtmg, den);
      wl = sr * iden;
      wr = -sl * iden;
      wu = sl * sr * iden;
    } else {
      wl = wr = R(0.5) * G.sqrtmg;
      wu = R(0);
    }
  }
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    if (CLEAN && (f == U_BX + D || f == U_PSI)) continue;  // the cleaning pair, below
    out[f * ostride] = wl * FL[f] + (wr * FR[f] + wu * (UR[f] - UL[f]));
  }
  if (CLEAN) {
    const int fb = U_BX + D;
    if constexpr (DIAG) {
      // zero shift: the pair's bounds are -+a, a = c_h alpha sqrt(gamma^DD) > 0, so the weights
      // reduce to sqrt(-g) / 2 for each state and a sqrt(-g) / 2 for the jump
      const R hs = R(0.5) * G.sqrtmg, ha = hs * (c.ch * cfac);
      out[fb * ostride] = hs * (FL[fb] + FR[fb]) - ha * (UR[fb] - UL[fb]);
      out[U_PSI * ostride] = hs * (FL[U_PSI] + FR[U_PSI]) - ha * (UR[U_PSI] - UL[U_PSI]);
    } else {
      R cm, cp;
      clean_speeds<D, DIAG>(G, c.ch, cm, cp);
      const R csl = fmin(R(0), cm), csr = fmax(R(0), cp);
      const R cden = csr - csl;
      if (cden != R(0)) {
        const R ic = G.sqrtmg / cden;
        out[fb * ostride] = (csr * FL[fb] - csl * FR[fb] + csl * csr * (UR[fb] - UL[fb])) * ic;
        out[U_PSI * ostride] = (csr * FL[U_PSI] - csl * FR[U_PSI] + csl * csr * (UR[U_PSI] - UL[U_PSI])) * ic;
      } else {
        out[fb * ostride] = wl * FL[fb] + (wr * FR[fb] + wu * (UR[fb] - UL[fb]));
        out[U_PSI * ostride] = wl * FL[U_PSI] + (wr * FR[U_PSI] + wu * (UR[U_PSI] - UL[U_PSI]));
      }
    }
  }
}


// The HLLE flux of the face at i - 1/2 along D of cell (i, j, k) from its reconstructed states
// PL, PR: the face metric (mean of the two adjacent centre values; tabulated for a DIAG metric
// in FP64), then hlle_face_fused.
template <int D, bool CLEAN, bool DIAG, typename R, typename S>
__device__ __forceinline__ void face_riemann(const KParams& kp, const S* __restrict__ M, int i, int j,
                                             int k, R PL[9], R PR[9], R* out, int ostride) {
  if (!CLEAN) PL[8] = PR[8] = R(0);
  Geom<R> G;
  if constexpr (DIAG && !SameType<R, float>::value) {
    G = geo_load<R>(kp.geo_f + D * GEO_F * kp.ms, met_off(kp, i, j, k), kp.ms);
  } else {
    R m[10];
    const long long o1 = met_off(kp, i, j, k);
    const long long o0 = o1 - (D == 0 ? 1 : (D == 1 ? kp.mpitch : kp.mplane));
    R m0[10], m1[10];
    load_metric<DIAG>(kp, M, o0, m0);
    load_metric<DIAG>(kp, M, o1, m1);
#pragma unroll
    for (int f = 0; f < 10; ++f) m[f] = R(0.5) * (m0[f] + m1[f]);
    G = make_geom<DIAG>(m);
  }
  const Consts<R> c = consts_of<R>(kp);
  R cfac = R(0);
  if constexpr (CLEAN && DIAG) {
    if constexpr (!SameType<R, float>::value)
      cfac = ldc<R>(kp.geo_f + (D * GEO_F + GEO_N) * kp.ms + met_off(kp, i, j, k));
    else
      cfac = G.alp * fsqrt(sel<D>(G.ixx, G.iyy, G.izz));
  }
  hlle_face_fused<D, CLEAN, DIAG>(G, PL, PR, c, cfac, out, ostride);
}

// HLLE flux of the face at i - 1/2 along D of cell (i, j, k) (the face between cells i-1 and
// i along D), written to out[f * ostride].
// RECON 0: TVD with the MC limiter (stencil c-2 .. c+1); 1: PPM (stencil c-3 .. c+2).
// ZC (z faces, MC reconstruction): 0 plain; 1 the z-march's first face, which also leaves in zc
// the carry of the next face up; 2 a face whose left state and lower half-stencil come from that
// carry (and which leaves the next one).  For the face k - 1/2 (cells k - 2 .. k + 1) the carry
// is, per field, P_k + sigma_k (the next face's left state), P_{k+1} and P_{k+1} - P_k, so the
// next face needs one load, one difference, one limited slope and two face values: the same
// operations on the same operands as the plain stencil, three FP64 operations and three loads
// fewer per field.  zc: this thread's carry, value q of field f at zc[(3 f + q) zs].
template <int D, bool CLEAN, bool DIAG, int RECON, int ZC = 0, typename R, typename S>
__device__ __forceinline__ void face_flux(const KParams& kp, const S* __restrict__ P,
                                          const S* __restrict__ M, int i, int j, int k, R* out,
                                          int ostride, R* zc = nullptr, int zs = 0) {
  static_assert(ZC == 0 || (D == 2 && RECON == 0), "the carry serves MC z faces");
  constexpr int NV = CLEAN ? 9 : 8;
  constexpr int NS = RECON ? 6 : 4;
  long long off[NS];  // stencil cells s = -NS/2 .. NS/2 - 1 along D
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (ZC == 2 && s < NS - 1) continue;  // only the top cell is new
    int ii = i, jj = j, kk = k;
    if (D == 0) ii = bc_index(i + s - NS / 2, kp.nx, kp.bcx);
    if (D == 1) jj = bc_index(j + s - NS / 2, kp.ny, kp.bcy);
    if (D == 2) kk = bc_index(k + s - NS / 2, kp.nz, kp.bcz);
    off[s] = (long long)kk * kp.plane + (long long)jj * kp.pitch + ii;
  }
  R PL[9], PR[9];
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    const S* pf = P + f * kp.fs;
    if constexpr (ZC == 2) {
      R* cf = zc + 3 * f * zs;
      const R cc = cf[zs], d1 = cf[2 * zs];
      const R d = ldc<R>(pf + off[3]);
      const R d2 = d - cc;
      const R h = mc_half_slope(d1, d2);
      PL[f] = cf[0];
      PR[f] = cc - h;
      cf[0] = cc + h;
      cf[zs] = d;
      cf[2 * zs] = d2;
    } else if constexpr (RECON == 0) {
      const R a = ldc<R>(pf + off[0]), b = ldc<R>(pf + off[1]);
      const R cc = ldc<R>(pf + off[2]), d = ldc<R>(pf + off[3]);
      const R d0 = b - a, d1 = cc - b, d2 = d - cc;
      PL[f] = b + mc_half_slope(d0, d1);
      const R h = mc_half_slope(d1, d2);
      PR[f] = cc - h;
      if constexpr (ZC == 1) {
        R* cf = zc + 3 * f * zs;
        cf[0] = cc + h;
        cf[zs] = d;
        cf[2 * zs] = d2;
      }
    } else {
      ppm_face<R>(ldc<R>(pf + off[0]), ldc<R>(pf + off[1]), ldc<R>(pf + off[2]),
                  ldc<R>(pf + off[3]), ldc<R>(pf + off[4]), ldc<R>(pf + off[5]), PL[f], PR[f]);
    }
  }
  face_riemann<D, CLEAN, DIAG>(kp, M, i, j, k, PL, PR, out, ostride);
}

// HLLE flux of the face at i - 1/2 along D (0 or 1) of cell (i, j, k), its MC stencil read from
// a primitive plane staged in shared memory (stage_plane): sp is the stencil's first cell (i - 2
// along x, j - 2 along y) of field 0, fields sf apart, stencil cells ss apart.  The same
// operations on the same operands as face_flux's MC stencil.
template <int D, bool CLEAN, bool DIAG, typename R, typename S>
__device__ __forceinline__ void face_flux_smem(const KParams& kp, const R* sp, int sf, int ss,
                                               const S* __restrict__ M, int i, int j, int k, R* out,
                                               int ostride) {
  constexpr int NV = CLEAN ? 9 : 8;
  R PL[9], PR[9];
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    const R* q = sp + f * sf;
    const R a = q[0], b = q[ss], cc = q[2 * ss], d = q[3 * ss];
    const R d0 = b - a, d1 = cc - b, d2 = d - cc;
    PL[f] = b + mc_half_slope(d0, d1);
    PR[f] = cc - mc_half_slope(d1, d2);
  }
  face_riemann<D, CLEAN, DIAG>(kp, M, i, j, k, PL, PR, out, ostride);
}

#ifdef __CUDACC__
// Asynchronous 4-byte copy from global to shared memory (cp.async, cached in L1), the commit of
// the copies a thread has issued, and the wait for all of them.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Stage plane k of the FP32 primitive state for the TX x TY tile at (i0, j0): sp[f][ly][lx] with
// SX = TX + 4 columns and SY = TY + 4 rows, local (lx, ly) = global (i0 - 2 + lx, j0 - 2 + ly),
// boundary indices resolved as face_flux resolves them (clamped or wrapped).  Only the cells some
// x or y face of the tile reads are copied (up to the tile's last face + 1 along each axis, which
// for a ragged tile stops inside [-2, n + 1], where bc_index is valid).  Copies are asynchronous;
// the caller waits (cp_async_wait_all) and synchronises the block before reading.
template <int TX, int TY, int NV>
__device__ __forceinline__ void stage_plane(const KParams& kp, const float* __restrict__ P, float* sp,
                                            int i0, int j0, int k) {
  constexpr int SX = TX + 4, SY = TY + 4, SF = SX * SY;
  const int nxl = min(TX, kp.nx - i0) + 4, nyl = min(TY, kp.ny - j0) + 4;
  const float* pk = P + (long long)k * kp.plane;
  for (int e = threadIdx.x; e < SF; e += TX * TY) {
    const int ly = e / SX, lx = e - ly * SX;
    if (lx < nxl && ly < nyl) {
      const int ii = bc_index(i0 - 2 + lx, kp.nx, kp.bcx), jj = bc_index(j0 - 2 + ly, kp.ny, kp.bcy);
      const float* src = pk + (long long)jj * kp.pitch + ii;
#pragma unroll
      for (int f = 0; f < NV; ++f) cp_async4(sp + f * SF + e, src + f * kp.fs);
    }
  }
  cp_async_commit();
}
#endif  // __CUDACC__

// One face of the double-word path with its direction D given at run time (one copy of the
// face code for all three directions): the stencil runs along D, and vectors and the metric are
// rotated cyclically (component (D + a) mod 3 becomes component a) so that the face normal is x;
// the x-direction HLLE code forms the flux, which is rotated back.
template <bool CLEAN, bool DIAG>
__device__ __forceinline__ void face_flux_dw(const KParams& kp, const double* __restrict__ P,
                                             const double* __restrict__ M, int D, int i, int j, int k,
                                             f32x2* out, int ostride) {
  using R = f32x2;
  constexpr int NV = CLEAN ? 9 : 8;
  const int c0 = D, c1 = D == 2 ? 0 : D + 1, c2 = D == 0 ? 2 : D - 1;  // rotated axes
  const int id = D == 0 ? i : (D == 1 ? j : k);
  const int nd = D == 0 ? kp.nx : (D == 1 ? kp.ny : kp.nz);
  const int bcd = D == 0 ? kp.bcx : (D == 1 ? kp.bcy : kp.bcz);
  const long long base = (long long)k * kp.plane + (long long)j * kp.pitch + i;
  const long long step = D == 0 ? 1 : (D == 1 ? kp.pitch : kp.plane);
  long long off[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) off[s] = base + (long long)(bc_index(id + s - 2, nd, bcd) - id) * step;
  R PL[9], PR[9];
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    const double* pf = P + f * kp.fs;
    const R a = ldc<R>(pf + off[0]), b = ldc<R>(pf + off[1]);
    const R cc = ldc<R>(pf + off[2]), d = ldc<R>(pf + off[3]);
    const R d0 = b - a, d1 = cc - b, d2 = d - cc;
    PL[f] = b + mc_half_slope(d0, d1);
    PR[f] = cc - mc_half_slope(d1, d2);
  }
  if (!CLEAN) PL[8] = PR[8] = R(0);
  auto pick = [](int cmp, R x, R y, R z) { return cmp == 0 ? x : (cmp == 1 ? y : z); };
  // rotate the velocity and field components of both states
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int o = q == 0 ? P_UX : P_BX;
    R L0 = PL[o], L1 = PL[o + 1], L2 = PL[o + 2], R0 = PR[o], R1 = PR[o + 1], R2 = PR[o + 2];
    PL[o] = pick(c0, L0, L1, L2);
    PL[o + 1] = pick(c1, L0, L1, L2);
    PL[o + 2] = pick(c2, L0, L1, L2);
    PR[o] = pick(c0, R0, R1, R2);
    PR[o + 1] = pick(c1, R0, R1, R2);
    PR[o + 2] = pick(c2, R0, R1, R2);
  }
  // face metric in the rotated frame
  Geom<R> G;
  const long long mo = met_off(kp, i, j, k);
  if constexpr (DIAG) {
    G = geo_load<R>(kp.geo_f + D * GEO_F * kp.ms, mo, kp.ms);
    const R g0 = G.gxx, g1 = G.gyy, g2 = G.gzz, h0 = G.ixx, h1 = G.iyy, h2 = G.izz;
    G.gxx = pick(c0, g0, g1, g2);
    G.gyy = pick(c1, g0, g1, g2);
    G.gzz = pick(c2, g0, g1, g2);
    G.ixx = pick(c0, h0, h1, h2);
    G.iyy = pick(c1, h0, h1, h2);
    G.izz = pick(c2, h0, h1, h2);
  } else {
    const long long mstep = D == 0 ? 1 : (D == 1 ? kp.mpitch : kp.mplane);
    R m0[10], m1[10], m[10], r[10];
    load_metric<false>(kp, M, mo - mstep, m0);
    load_metric<false>(kp, M, mo, m1);
#pragma unroll
    for (int f = 0; f < 10; ++f) m[f] = R(0.5) * (m0[f] + m1[f]);
    // gamma_ab as a 3 x 3 table by index, then permuted
    const R gm[3][3] = {{m[M_GXX], m[M_GXY], m[M_GXZ]}, {m[M_GXY], m[M_GYY], m[M_GYZ]},
                        {m[M_GXZ], m[M_GYZ], m[M_GZZ]}};
    auto gsel = [&](int a, int b) {
      const R* row0 = gm[0];
      const R* row1 = gm[1];
      const R* row2 = gm[2];
      const R x = pick(b, row0[0], row0[1], row0[2]);
      const R y = pick(b, row1[0], row1[1], row1[2]);
      const R z = pick(b, row2[0], row2[1], row2[2]);
      return pick(a, x, y, z);
    };
    r[M_ALP] = m[M_ALP];
    r[M_BX] = pick(c0, m[M_BX], m[M_BY], m[M_BZ]);
    r[M_BY] = pick(c1, m[M_BX], m[M_BY], m[M_BZ]);
    r[M_BZ] = pick(c2, m[M_BX], m[M_BY], m[M_BZ]);
    r[M_GXX] = gsel(c0, c0);
    r[M_GXY] = gsel(c0, c1);
    r[M_GXZ] = gsel(c0, c2);
    r[M_GYY] = gsel(c1, c1);
    r[M_GYZ] = gsel(c1, c2);
    r[M_GZZ] = gsel(c2, c2);
    G = make_geom<false>(r);
  }
  const Consts<R> c = consts_of<R>(kp);
  R cfac = R(0);
  if constexpr (CLEAN && DIAG) cfac = ldc<R>(kp.geo_f + (D * GEO_F + GEO_N) * kp.ms + mo);
  R F[9];
  hlle_face<0, CLEAN, DIAG, true>(G, PL, PR, c, cfac, F, 1);
  // rotate back: rotated component a is original component (D + a) mod 3
  R T[3] = {F[U_TX], F[U_TY], F[U_TZ]}, B[3] = {F[U_BX], F[U_BY], F[U_BZ]};
  auto back = [&](int orig, const R v[3]) {
    // the rotated index a with (D + a) mod 3 == orig
    const int a2 = orig - D;
    const int aa = a2 < 0 ? a2 + 3 : a2;
    return pick(aa, v[0], v[1], v[2]);
  };
  F[U_TX] = back(0, T);
  F[U_TY] = back(1, T);
  F[U_TZ] = back(2, T);
  F[U_BX] = back(0, B);
  F[U_BY] = back(1, B);
  F[U_BZ] = back(2, B);
#pragma unroll
  for (int f = 0; f < NV; ++f) out[f * ostride] = F[f];
}

template <bool DIAG, typename R, typename S>
__device__ __forceinline__ G4<R> g4_at(const KParams& kp, const S* __restrict__ M, long long off) {
  R m[10];
  load_metric<DIAG>(kp, M, off, m);
  G4<R> g;
  g.gxx = m[M_GXX];
  g.gyy = m[M_GYY];
  g.gzz = m[M_GZZ];
  if constexpr (DIAG) {
    g.gxy = g.gxz = g.gyz = g.blx = g.bly = g.blz = R(0);
    g.gtt = -m[M_ALP] * m[M_ALP];
  } else {
    g.gxy = m[M_GXY];
    g.gxz = m[M_GXZ];
    g.gyz = m[M_GYZ];
    g.blx = g.gxx * m[M_BX] + g.gxy * m[M_BY] + g.gxz * m[M_BZ];
    g.bly = g.gxy * m[M_BX] + g.gyy * m[M_BY] + g.gyz * m[M_BZ];
    g.blz = g.gxz * m[M_BX] + g.gyz * m[M_BY] + g.gzz * m[M_BZ];
    g.gtt = -m[M_ALP] * m[M_ALP] + (g.blx * m[M_BX] + g.bly * m[M_BY] + g.blz * m[M_BZ]);
  }
  return g;
}

// The cell's CFL rate: the sum over active axes of max|lambda| / dx (each axis's bound widened
// to the cleaning speed when on); dt = CFL / (max over cells).  The RK stages update all axes at
// once, so the Courant numbers of the axes add up for a mode along a diagonal; in 1-D this is
// the per-axis maximum.
template <bool YA, bool ZA, bool CLEAN, bool DIAG, typename R>
__device__ __forceinline__ double cell_max_speed(const KParams& kp, const Geom<R>& G, const R P[9],
                                                 const Consts<R>& c) {
  // FP64: quotients and square roots through rcp_fast and the reciprocal square root
  constexpr bool FAST = SameType<R, double>::value;
  const State<R> S = make_state<DIAG>(G, P, c);
  const R c2 = cms2_of<R, FAST>(S, c);
  R lm, lp;
  speeds_of<0, DIAG, R, FAST>(G, S, c2, lm, lp);
  double a = (double)fmax(fabs(lm), fabs(lp));
  if (CLEAN) {
    clean_speeds<0, DIAG>(G, c.ch, lm, lp);
    a = fmax(a, (double)fmax(fabs(lm), fabs(lp)));
  }
  double v = a * kp.idx;
  if (YA) {
    speeds_of<1, DIAG, R, FAST>(G, S, c2, lm, lp);
    a = (double)fmax(fabs(lm), fabs(lp));
    if (CLEAN) {
      clean_speeds<1, DIAG>(G, c.ch, lm, lp);
      a = fmax(a, (double)fmax(fabs(lm), fabs(lp)));
    }
    v += a * kp.idy;
  }
  if (ZA) {
    speeds_of<2, DIAG, R, FAST>(G, S, c2, lm, lp);
    a = (double)fmax(fabs(lm), fabs(lp));
    if (CLEAN) {
      clean_speeds<2, DIAG>(G, c.ch, lm, lp);
      a = fmax(a, (double)fmax(fabs(lm), fabs(lp)));
    }
    v += a * kp.idz;
  }
  return v;
}

// The CFL rate of a cell just set to the atmosphere (u~ = 0) on a zero-shift diagonal metric, in
// closed form: along every axis the dispersion relation has A = 1/alpha^2, B = 0 and
// C = -c^2 gamma^dd, so lambda = -+ c alpha sqrt(gamma^dd), with c^2 = c_s^2 + v_A^2 - c_s^2 v_A^2
// = (gamma p + b^2) / (w + b^2) for that state; with cleaning each axis's bound is
// max(c, c_h) alpha sqrt(gamma^dd).  cfl_geo: sum_d alpha sqrt(gamma^dd) / dx_d (centre table).
template <bool CLEAN>
__device__ __forceinline__ double atm_cfl_rate(const KParams& kp, double b2, double cfl_geo) {
  const double gp = kp.gamma * kp.p_atm;
  const double w = fma(kp.gfac, kp.p_atm, kp.rho_floor);
  const double c2 = (gp + b2) * rcp_fast(w + b2);
  double c = c2 * rsqrt(c2);
  if (CLEAN) c = fmax(c, kp.ch);
  return c * cfl_geo;
}

// The same for any state at rest (density rho, pressure p, b^2 = alpha^2 gamma_ij B^i B^j; a
// state with c^2 = 0 has rate c_h, or 0 without cleaning).
template <bool CLEAN>
__device__ __forceinline__ double rest_cfl_rate(const KParams& kp, double rho, double p, double b2,
                                                double cfl_geo) {
  const double gp = kp.gamma * p;
  const double w = fma(kp.gfac, p, rho);
  const double c2 = (gp + b2) * rcp_fast(w + b2);
  double c = c2 > 0.0 ? c2 * rsqrt(c2) : 0.0;
  if (CLEAN) c = fmax(c, kp.ch);
  return c * cfl_geo;
}

// Which warps of a TX x TY tile compute its extra faces on plane k: the top row of y faces (one
// full warp pass, warp wy) and the right column of x faces (TY lanes of warp wx).  A warp's FP64
// instruction holds the FP64 pipe for the same time whatever its active lanes, so each job costs
// its warp a full face pass; ROTATE moves both jobs one warp along per plane, so that over NW
// planes every warp carries the same number of passes.
template <int NW, bool ROTATE>
__host__ __device__ __forceinline__ void extra_warps(int k, int& wy, int& wx) {
  static_assert((NW & (NW - 1)) == 0, "a power of two warps");
  if constexpr (NW < 2) {  // one warp (1-D tiles): no extra faces of this kind
    wy = wx = 0;
  } else {
    wy = ROTATE ? (k & (NW - 1)) : 0;
    wx = ROTATE ? ((k + NW / 2) & (NW - 1)) : 1;
  }
}

#ifdef __CUDACC__  // device-only: block reduction, kernels, launchers (the helpers build for the host too)
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
#endif  // __CUDACC__

// Reset of a cell the recovery does not accept (§3.2 names no rule; the atmosphere and floors of
// the method's readings).  to_atm: the atmosphere state; else the recovered state with its
// pressure raised to p_floor.  Rewrites P and U.  atm_b2: when not null and the cell is set to
// the atmosphere, receives that state's b^2.
template <bool CLEAN, bool DIAG, typename TP>
__device__ __forceinline__ void reset_cell(const KParams& kp, const Geom<double>& G, double U[9],
                                           const Consts<double>& c, TP P[9], bool to_atm,
                                           double* atm_b2) {
  if (to_atm) {
    // The atmosphere state: rho_floor, p_atm, u~ = 0, the cell's B and psi.  Its conserved
    // vector in closed form: u~ = 0 gives W = 1, u^t = 1/alpha, u_i = 0 and b^t = 0, hence
    // b^i = alpha B^i and b^2 = gamma_ij Bn^i Bn^j with the Eulerian field Bn^i = alpha B^i =
    // U_B^i / sqrt(gamma), and U = (sqrt(gamma) rho, -sqrt(-g) (rho + p / (gamma - 1) + b^2/2),
    // 0, 0, 0, U_B, U_Psi): the value make_state + cons_of give for that state (§2.1).
    const double isg = rcp_fast(G.sqrtg);
    const double bnx = U[U_BX] * isg, bny = U[U_BY] * isg, bnz = U[U_BZ] * isg;
    double b2;
    if constexpr (DIAG) {
      b2 = G.gxx * bnx * bnx + G.gyy * bny * bny + G.gzz * bnz * bnz;
    } else {
      b2 = (G.gxx * bnx + 2.0 * (G.gxy * bny + G.gxz * bnz)) * bnx +
           (G.gyy * bny + 2.0 * G.gyz * bnz) * bny + G.gzz * bnz * bnz;
    }
    P[P_BX] = store_as<TP>(bnx * G.ialp);
    P[P_BY] = store_as<TP>(bny * G.ialp);
    P[P_BZ] = store_as<TP>(bnz * G.ialp);
    P[P_PSI] = CLEAN ? store_as<TP>(U[U_PSI] * isg) : TP(0);
    P[P_RHO] = kconst<TP>(kp.rho_floor, kp.f_rho_floor);
    P[P_PRS] = kconst<TP>(kp.p_atm, kp.f_p_atm);
    P[P_UX] = P[P_UY] = P[P_UZ] = TP(0);
    // rest-mass plus internal energy density of the atmosphere: rho + p / (gamma - 1), with
    // 1 / (gamma - 1) = gamma / (gamma - 1) - 1
    const double e_atm = fma(kp.p_atm, kp.gfac - 1.0, kp.rho_floor);
    U[U_D] = G.sqrtg * kp.rho_floor;
    U[U_TT] = -G.sqrtmg * fma(0.5, b2, e_atm);
    U[U_TX] = U[U_TY] = U[U_TZ] = 0.0;
    if (atm_b2) *atm_b2 = b2;
  } else {
    P[P_PRS] = (TP)kp.p_floor;
    double Pd[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) Pd[f] = (double)P[f];
    const State<double> S = make_state<DIAG>(G, Pd, c);
    cons_of<CLEAN>(G, S, U);
  }
}

// Recovery with atmosphere / floor handling; rewrites U when the cell is reset.  TG, TP: the
// element types of the guess and of the result (float for the mixed path, whose primitive
// state is stored in FP32; a pressure-floor reset recomputes U from that stored state).
// atm_b2: when not null and the cell is set to the atmosphere, receives that state's b^2.
template <bool CLEAN, bool DIAG, bool ONE_FINISH = false, typename TG = double, typename TP = double>
__device__ __forceinline__ int recover(const KParams& kp, const Geom<double>& G, double U[9],
                                       const TG Pg[9], const Consts<double>& c, TP P[9],
                                       int& iters, double* atm_b2 = nullptr) {
  // atmosphere: a cell whose rest-mass density D / sqrt(gamma) = rho W is below rho_atm is not
  // recovered but set to the atmosphere state (the decision uses the conserved state only)
  const bool atm = U[U_D] < kp.rho_atm * G.sqrtg;
  C2PResult r = {1, 0};
  if (!atm)
    r = con2prim<CLEAN, DIAG, ONE_FINISH, TG, TP>(G, U, Pg, c, kp.c2p_maxit, kp.c2p_step_tol, P, kp.c2p_1d);
  iters = r.iters;
  if (atm || !r.ok || (double)P[P_RHO] < kp.rho_floor)
    reset_cell<CLEAN, DIAG>(kp, G, U, c, P, true, atm_b2);
  else if ((double)P[P_PRS] < kp.p_floor)
    reset_cell<CLEAN, DIAG>(kp, G, U, c, P, false, nullptr);
  return r.ok ? 0 : 1;
}

#ifdef __CUDACC__
// Inputs of an out-of-line recovery (con2prim_call).
template <typename TG>
struct C2PArgs {
  Geom<double> G;
  Consts<double> c;
  double U[9];
  TG Pg[9];
  double step_tol;
  int maxit, one_d;
};

// con2prim as a function of its own (not inlined): a kernel whose cells mostly skip the Newton
// iteration (atmosphere) then reserves no registers for it, and the iteration's live values are
// saved and restored only on the path that calls it.
template <bool CLEAN, bool DIAG, bool ONE_FINISH, typename TG, typename TP>
static __device__ __noinline__ C2PResult con2prim_call(const C2PArgs<TG>* a, TP* P) {
  return con2prim<CLEAN, DIAG, ONE_FINISH, TG, TP>(a->G, a->U, a->Pg, a->c, a->maxit, a->step_tol, P, a->one_d);
}

// recover() for a kernel that stores the conserved vector itself: U is written to Uout (field
// stride fs) before the Newton iteration, which runs out of line (con2prim_call), and again,
// reloaded and rewritten, only for a cell that is then reset.  Same results as recover()
// followed by the store of U.
template <bool CLEAN, bool DIAG, bool ONE_FINISH, typename TG, typename TP>
__device__ __forceinline__ int recover_stored(const KParams& kp, const Geom<double>& G, double U[9],
                                              double* Uout, long long fs, const TG Pg[9],
                                              const Consts<double>& c, TP P[9], int& iters,
                                              double* atm_b2 = nullptr) {
  constexpr int NV = CLEAN ? 9 : 8;
  const bool atm = U[U_D] < kp.rho_atm * G.sqrtg;
  C2PResult r = {1, 0};
  bool to_atm = atm;
  if (!atm) {
#pragma unroll
    for (int f = 0; f < NV; ++f) Uout[f * fs] = U[f];
    {
      C2PArgs<TG> a;
      a.G = G;
      a.c = c;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        a.U[f] = U[f];
        a.Pg[f] = Pg[f];
      }
      a.step_tol = kp.c2p_step_tol;
      a.maxit = kp.c2p_maxit;
      a.one_d = kp.c2p_1d;
      TP Pr[9];
      r = con2prim_call<CLEAN, DIAG, ONE_FINISH, TG, TP>(&a, Pr);
#pragma unroll
      for (int f = 0; f < 9; ++f) P[f] = Pr[f];
    }
    to_atm = !r.ok || (double)P[P_RHO] < kp.rho_floor;
    if (!to_atm && !((double)P[P_PRS] < kp.p_floor)) {
      iters = r.iters;
      return 0;
    }
    // a reset after the iteration: the conserved vector back from memory (an opaque load, so
    // that the compiler does not keep it in registers through the iteration)
#pragma unroll
    for (int f = 0; f < NV; ++f)
      asm volatile("ld.global.f64 %0, [%1];" : "=d"(U[f]) : "l"(Uout + f * fs) : "memory");
  }
  iters = r.iters;
  reset_cell<CLEAN, DIAG>(kp, G, U, c, P, to_atm, to_atm ? atm_b2 : nullptr);
#pragma unroll
  for (int f = 0; f < NV; ++f) Uout[f * fs] = U[f];
  return r.ok ? 0 : 1;
}
#endif  // __CUDACC__

#ifdef __CUDACC__
// PAIR (FP64 state only): reconstruction, face states, fluxes, HLLE, divergence and sources in
// double-word arithmetic (f32x2, on the FP32 pipes); the RK update, the recovery and the CFL
// maximum in FP64 as on the FP64 path.
template <int TX, int TY, bool YA, bool ZA, bool CLEAN, bool DIAG, bool MIXED, int RECON,
          bool PAIR = false>
__global__ void __launch_bounds__(TX * TY, MIXED ? 4 : 2)
k_substep(const KParams kp, const StageArgs sa, const typename Prec<MIXED>::S* __restrict__ M,
          DevScalars* sc) {
  static_assert(!(PAIR && MIXED), "the double-word faces run over the FP64 state");
  using R = typename FaceType<PAIR, MIXED>::R;
  using RN = typename Prec<MIXED>::R;  // type of the recovered state
  using S = typename Prec<MIXED>::S;
  constexpr int NT = TX * TY;
  constexpr int NV = CLEAN ? 9 : 8;
  __shared__ R fx[NV][TY][TX + 1];
  __shared__ R fy[YA ? NV : 1][YA ? TY + 1 : 1][TX];
  __shared__ R fz[ZA ? 2 : 1][ZA ? NV : 1][TY][TX];
  // 3-D kernels that read their faces from global memory: the tile's right column of x faces
  // (TY per plane) is computed for XB planes at once, one lane per face, every XB planes of a z
  // segment, and kept here (a warp's FP64 instruction costs the same pipe time with TY active
  // lanes as with 32, so one batched pass replaces XB passes).  The staged mixed kernel, which
  // is bound by latency rather than by a pipe, keeps one pass per plane (batched: -1.8 %).
  constexpr bool XBATCH = ZA && YA && !PAIR && !(MIXED && RECON == 0);
  constexpr int XB = 32 / TY;
  static_assert(32 % TY == 0, "whole planes of x faces per warp");
  __shared__ R fxr[XBATCH ? XB : 1][XBATCH ? TY : 1][XBATCH ? NV : 1];
  // z-face reconstruction carry (face_flux ZC), three values per field and thread, in dynamic
  // shared memory (it does not fit the 48 KB of static shared memory beside the face fluxes)
  constexpr bool ZCARRY = ZA && !PAIR && RECON == 0;
  extern __shared__ __align__(16) unsigned char hz_dyn_smem[];
  R* const zc = reinterpret_cast<R*>(hz_dyn_smem) + threadIdx.x;
  // Mixed 3-D MC kernels: the primitive plane that the x and y faces read (the tile with a
  // two-cell halo) is staged in shared memory by asynchronous copies (stage_plane), behind the
  // carry; the copies of plane k + 1 are issued before the cell update of plane k and overlap it.
  constexpr bool STAGE = MIXED && YA && ZA && RECON == 0 && !PAIR;
  constexpr int SX = TX + 4, SF = (TX + 4) * (TY + 4);
  constexpr bool ROTATE = true;
  R* const sp = reinterpret_cast<R*>(hz_dyn_smem + (ZCARRY ? 3 * NV * NT * sizeof(R) : 0));

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const double dt = sc->dt;
  const bool first_stage = sa.a0 == 0.0 && sa.ak == 1.0;  // U = Uk + dt L
  const Consts<R> c = consts_of<R>(kp);
  const Consts<double> cd = consts_of<double>(kp);
  const R ridx = kconst<R>(kp.idx, kp.f_idx), ridy = kconst<R>(kp.idy, kp.f_idy);
  const R ridz = kconst<R>(kp.idz, kp.f_idz);
  const R rhdx = kconst<R>(0.5 * kp.idx, 0.5f * kp.f_idx), rhdy = kconst<R>(0.5 * kp.idy, 0.5f * kp.f_idy);
  const R rhdz = kconst<R>(0.5 * kp.idz, 0.5f * kp.f_idz);
  const R rkappa = kconst<R>(kp.kappa, kp.f_kappa);
  const S* __restrict__ P = (const S*)sa.Pin;
  S* __restrict__ Pout = (S*)sa.Pout;

  double vloc = 0.0;
  int nfail = 0, maxit = 0;

  // FP64 kernels (bound by the FP64 pipe): a persistent grid; the plane-tiles (tile column, z)
  // in column order are split into gridDim.x equal contiguous ranges, one per block, so that no
  // partial last wave idles SMs; a range is one or more z segments of columns, each marched
  // upwards from its first z face.  Mixed and double-word kernels (bound by latency): one block
  // per tile column and z chunk (grid ntx x nty x chunks), whose launch order keeps the blocks
  // running together on neighbouring tiles at the same heights, which share their halos in L2.
  constexpr bool PERSIST = !MIXED && !PAIR;
  const int ntx = (kp.nx + TX - 1) / TX, nty = (kp.ny + TY - 1) / TY;
  const long long total = (long long)ntx * nty * kp.nz;
  long long q = PERSIST ? total * blockIdx.x / gridDim.x : 0;
  const long long q1 = PERSIST ? total * (blockIdx.x + 1) / gridDim.x : 1;
  while (q < q1) {
  long long col;
  int kz0, kz1;
  if constexpr (PERSIST) {
    col = q / kp.nz;
    kz0 = (int)(q - col * kp.nz);
    kz1 = (int)min((long long)kp.nz, kz0 + (q1 - q));
    q += kz1 - kz0;
  } else {
    col = (long long)blockIdx.y * ntx + blockIdx.x;
    kz0 = blockIdx.z * kp.zlen;
    kz1 = min(kz0 + kp.zlen, kp.nz);
    q = q1;
  }
  const int i0 = (int)(col % ntx) * TX, j0 = (int)(col / ntx) * TY;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < kp.nx && j < kp.ny;

  if constexpr (STAGE) stage_plane<TX, TY, NV>(kp, P, sp, i0, j0, kz0);
  if constexpr (!PAIR) {
    if (ZA && own) {
      if constexpr (ZCARRY)
        face_flux<2, CLEAN, DIAG, RECON, 1>(kp, P, M, i, j, kz0, &fz[kz0 & 1][0][ty][tx], TY * TX, zc, NT);
      else
        face_flux<2, CLEAN, DIAG, RECON>(kp, P, M, i, j, kz0, &fz[kz0 & 1][0][ty][tx], TY * TX);
    }
  }
  if constexpr (STAGE) {
    cp_async_wait_all();
    __syncthreads();
  }

  for (int k = kz0; k < kz1; ++k) {
    // ---- faces of plane k: each face of the tile once
    if constexpr (PAIR) {
      // one copy of the double-word face code, run in passes: x faces, y faces, the upper z
      // face, the tile's extra row / column, and (first plane only) the lower z face
#pragma unroll 1
      for (int pass = 0; pass < 5; ++pass) {
        int D = -1, ii = i, jj = j, kk = k, os = 0;
        R* o = nullptr;
        if (pass == 0) {
          if (i <= kp.nx && j < kp.ny) {
            D = 0;
            o = &fx[0][ty][tx];
            os = TY * (TX + 1);
          }
        } else if (pass == 1) {
          if (YA && i < kp.nx && j <= kp.ny) {
            D = 1;
            o = &fy[0][ty][tx];
            os = (TY + 1) * TX;
          }
        } else if (pass == 2) {
          if (ZA && own) {
            D = 2;
            kk = k + 1;
            o = &fz[(k + 1) & 1][0][ty][tx];
            os = TY * TX;
          }
        } else if (pass == 3) {
          if (YA && threadIdx.x < TX) {
            ii = i0 + threadIdx.x;
            jj = j0 + TY;
            if (ii < kp.nx && jj <= kp.ny) {
              D = 1;
              o = &fy[0][TY][threadIdx.x];
              os = (TY + 1) * TX;
            }
          } else if (YA ? (threadIdx.x >= 32 && threadIdx.x < 32 + TY) : threadIdx.x < TY) {
            const int t = YA ? threadIdx.x - 32 : threadIdx.x;
            jj = j0 + t;
            ii = i0 + TX;
            if (ii <= kp.nx && jj < kp.ny) {
              D = 0;
              o = &fx[0][t][TX];
              os = TY * (TX + 1);
            }
          }
        } else {
          if (ZA && own && k == kz0) {
            D = 2;
            o = &fz[kz0 & 1][0][ty][tx];
            os = TY * TX;
          }
        }
        if (D >= 0) face_flux_dw<CLEAN, DIAG>(kp, P, M, D, ii, jj, kk, o, os);
      }
    } else if constexpr (STAGE) {
      // x and y faces from the staged plane; z faces as below
      if (i <= kp.nx && j < kp.ny)
        face_flux_smem<0, CLEAN, DIAG>(kp, sp + (ty + 2) * SX + tx, SF, 1, M, i, j, k, &fx[0][ty][tx], TY * (TX + 1));
      if (i < kp.nx && j <= kp.ny)
        face_flux_smem<1, CLEAN, DIAG>(kp, sp + ty * SX + tx + 2, SF, SX, M, i, j, k, &fy[0][ty][tx], (TY + 1) * TX);
      if (own) {
        if constexpr (ZCARRY)
          face_flux<2, CLEAN, DIAG, RECON, 2>(kp, P, M, i, j, k + 1, &fz[(k + 1) & 1][0][ty][tx], TY * TX, zc, NT);
        else
          face_flux<2, CLEAN, DIAG, RECON>(kp, P, M, i, j, k + 1, &fz[(k + 1) & 1][0][ty][tx], TY * TX);
      }
      // the tile's extra faces, on warps that change with the plane (extra_warps)
      int wy, wx;
      extra_warps<NT / 32, ROTATE>(k, wy, wx);
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (wid == wy) {
        const int ii = i0 + lane, jj = j0 + TY;
        if (ii < kp.nx && jj <= kp.ny)
          face_flux_smem<1, CLEAN, DIAG>(kp, sp + TY * SX + lane + 2, SF, SX, M, ii, jj, k,
                                         &fy[0][TY][lane], (TY + 1) * TX);
      } else if (wid == wx && lane < TY) {
        const int t = lane, jj = j0 + t, ii = i0 + TX;
        if (ii <= kp.nx && jj < kp.ny)
          face_flux_smem<0, CLEAN, DIAG>(kp, sp + (t + 2) * SX + TX, SF, 1, M, ii, jj, k, &fx[0][t][TX],
                                         TY * (TX + 1));
      }
    } else {
    if (i <= kp.nx && j < kp.ny) face_flux<0, CLEAN, DIAG, RECON>(kp, P, M, i, j, k, &fx[0][ty][tx], TY * (TX + 1));
    if (YA && i < kp.nx && j <= kp.ny) face_flux<1, CLEAN, DIAG, RECON>(kp, P, M, i, j, k, &fy[0][ty][tx], (TY + 1) * TX);
    if (ZA && own) {
      if constexpr (ZCARRY)
        face_flux<2, CLEAN, DIAG, RECON, 2>(kp, P, M, i, j, k + 1, &fz[(k + 1) & 1][0][ty][tx], TY * TX, zc, NT);
      else
        face_flux<2, CLEAN, DIAG, RECON>(kp, P, M, i, j, k + 1, &fz[(k + 1) & 1][0][ty][tx], TY * TX);
    }
    if (YA) {
      // the tile's extra faces (top row of y faces, right column of x faces), on warps that
      // change with the plane (extra_warps)
      int wy, wx;
      extra_warps<NT / 32, ROTATE>(k, wy, wx);
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (wid == wy) {
        const int ii = i0 + lane, jj = j0 + TY;
        if (ii < kp.nx && jj <= kp.ny)
          face_flux<1, CLEAN, DIAG, RECON>(kp, P, M, ii, jj, k, &fy[0][TY][lane], (TY + 1) * TX);
      } else if (wid == wx) {
        if constexpr (XBATCH) {
          if ((k - kz0) % XB == 0) {  // the right x faces of planes k .. k + XB - 1
            const int kk = k + lane / TY, jj = j0 + lane % TY, ii = i0 + TX;
            if (kk < kz1 && ii <= kp.nx && jj < kp.ny)
              face_flux<0, CLEAN, DIAG, RECON>(kp, P, M, ii, jj, kk, &fxr[lane / TY][lane % TY][0], 1);
          }
        } else if (lane < TY) {
          const int jj = j0 + lane, ii = i0 + TX;
          if (ii <= kp.nx && jj < kp.ny)
            face_flux<0, CLEAN, DIAG, RECON>(kp, P, M, ii, jj, k, &fx[0][lane][TX], TY * (TX + 1));
        }
      }
    } else if (threadIdx.x < TY) {
      const int jj = j0 + threadIdx.x, ii = i0 + TX;
      if (ii <= kp.nx && jj < kp.ny)
        face_flux<0, CLEAN, DIAG, RECON>(kp, P, M, ii, jj, k, &fx[0][threadIdx.x][TX], TY * (TX + 1));
    }
    }
    // the cell's own primitive state from the staged plane, before the next plane replaces it
    R Pcs[9];
    if constexpr (STAGE) {
      if (own) {
#pragma unroll
        for (int f = 0; f < NV; ++f) Pcs[f] = sp[f * SF + (ty + 2) * SX + tx + 2];
      }
    }
    __syncthreads();
    if constexpr (STAGE) {
      if (k + 1 < kz1) stage_plane<TX, TY, NV>(kp, P, sp, i0, j0, k + 1);
    }

    // ---- cell update of plane k
    if (own) {
      const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
      const long long mo = met_off(kp, i, j, k);
      R L[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        R fr = fx[f][ty][tx + 1];
        if constexpr (XBATCH) {
          if (tx == TX - 1) fr = fxr[(k - kz0) % XB][ty][f];
        }
        R v = -(fr - fx[f][ty][tx]) * ridx;
        if (YA) v -= (fy[f][ty + 1][tx] - fy[f][ty][tx]) * ridy;
        if (ZA) v -= (fz[(k + 1) & 1][f][ty][tx] - fz[k & 1][f][ty][tx]) * ridz;
        L[f] = v;
      }
      // metric source 1/2 sqrt(-g) T^{ab} d_i g_ab (static metric: no energy source)
      Geom<R> G;
      if constexpr (DIAG && !MIXED) {
        G = geo_load<R>(kp.geo_c, mo, kp.ms);
      } else {
        R mc[10];
        load_metric<DIAG>(kp, M, mo, mc);
        G = make_geom<DIAG>(mc);
      }
      R Pc[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        if constexpr (STAGE) Pc[f] = Pcs[f];
        else Pc[f] = ldc<R>(P + f * kp.fs + off);
      }
      if (!CLEAN) Pc[8] = R(0);
      {
        const State<R> St = make_state<DIAG>(G, Pc, c);
        const Tup<R> T = tup_of<DIAG>(G, St);
        const R h = R(0.5) * G.sqrtmg;
        if constexpr (DIAG && !MIXED) {
          // tabulated differences of g_tt, g_xx, g_yy, g_zz between the two neighbours
          const double* gs = kp.geo_s;
          const long long ms = kp.ms;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            if ((d == 1 && !YA) || (d == 2 && !ZA)) continue;
            const double* g = gs + d * GEO_S * ms + mo;
            const R s = T.tt * ldc<R>(g) + T.xx * ldc<R>(g + ms) + T.yy * ldc<R>(g + 2 * ms) +
                        T.zz * ldc<R>(g + 3 * ms);
            L[U_TX + d] += h * s * (d == 0 ? rhdx : (d == 1 ? rhdy : rhdz));
          }
        } else {
          {
            const G4<R> gp = g4_at<DIAG, R>(kp, M, mo + 1), gm = g4_at<DIAG, R>(kp, M, mo - 1);
            L[U_TX] += h * tdg<DIAG>(T, gp, gm) * rhdx;
          }
          if (YA) {
            const G4<R> gp = g4_at<DIAG, R>(kp, M, mo + kp.mpitch), gm = g4_at<DIAG, R>(kp, M, mo - kp.mpitch);
            L[U_TY] += h * tdg<DIAG>(T, gp, gm) * rhdy;
          }
          if (ZA) {
            const G4<R> gp = g4_at<DIAG, R>(kp, M, mo + kp.mplane), gm = g4_at<DIAG, R>(kp, M, mo - kp.mplane);
            L[U_TZ] += h * tdg<DIAG>(T, gp, gm) * rhdz;
          }
        }
        if (CLEAN) L[U_PSI] += -rkappa * G.alp * (G.sqrtg * St.psi);
      }
      // Runge-Kutta stage (FP64)
      double U[9];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        const double uk = sa.Uk[f * kp.fs + off];
        double u;
        if (first_stage) u = uk + dt * to_dbl(L[f]);
        else u = sa.ak * (uk + dt * to_dbl(L[f])) + sa.a0 * sa.U0[f * kp.fs + off];
        U[f] = u;
      }
      if (!CLEAN) U[8] = 0.0;
      // recovery of the new primitive state (FP64 Newton; the mixed path forms its guess and
      // the FP32-stored part of its result in FP32)
      int it;
      RN Pn[9];
      if constexpr (PAIR) {
        // FP64 recovery from the stored FP64 guess, FP64 CFL maximum
        Geom<double> Gd;
        if constexpr (DIAG) {
          Gd = geo_load<double>(kp.geo_c, mo, kp.ms);
        } else {
          double md[10];
          load_metric<DIAG>(kp, M, mo, md);
          Gd = make_geom<DIAG>(md);
        }
        double Pg[9];
#pragma unroll
        for (int f = 0; f < NV; ++f) Pg[f] = __ldg(P + f * kp.fs + off);
        if (!CLEAN) Pg[8] = 0.0;
        double ab2 = -1.0;
        nfail += recover<CLEAN, DIAG>(kp, Gd, U, Pg, cd, Pn, it, DIAG ? &ab2 : nullptr);
        if (sa.last) {
          if (DIAG && ab2 >= 0.0)
            vloc = fmax(vloc, atm_cfl_rate<CLEAN>(kp, ab2, __ldg(kp.geo_c + GEO_N * kp.ms + mo)));
          else
            vloc = fmax(vloc, cell_max_speed<YA, ZA, CLEAN, DIAG>(kp, Gd, Pn, cd));
        }
      } else if constexpr (MIXED) {
        Geom<double> Gd;
        if constexpr (DIAG) {
          Gd = geo_load<double>(kp.geo_c, mo, kp.ms);
        } else {
          double md[10];
          load_metric<DIAG>(kp, M, mo, md);
          Gd = make_geom<DIAG>(md);
        }
        // the conserved vector is stored by the recovery (recover_stored), and the FP32 centre
        // geometry of the CFL speeds is formed again after it: neither is held in registers
        // through the Newton iteration
        nfail += recover_stored<CLEAN, DIAG, true>(kp, Gd, U, sa.Uout + off, kp.fs, Pc, cd, Pn, it);
        if (sa.last) {
          R mc[10];
#pragma unroll
          for (int f = 0; f < 10; ++f) mc[f] = R(0);
          if constexpr (DIAG) {
            const S* mp = M + mo;
            asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(mc[M_ALP]) : "l"(mp + M_ALP * kp.ms));
            asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(mc[M_GXX]) : "l"(mp + M_GXX * kp.ms));
            asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(mc[M_GYY]) : "l"(mp + M_GYY * kp.ms));
            asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(mc[M_GZZ]) : "l"(mp + M_GZZ * kp.ms));
          } else {
#pragma unroll
            for (int f = 0; f < 10; ++f)
              asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(mc[f]) : "l"(M + mo + f * kp.ms));
          }
          const Geom<R> Gc = make_geom<DIAG>(mc);
          vloc = fmax(vloc, cell_max_speed<YA, ZA, CLEAN, DIAG>(kp, Gc, Pn, c));
        }
      } else {
        double ab2 = -1.0;
        nfail += recover<CLEAN, DIAG>(kp, G, U, Pc, cd, Pn, it, DIAG ? &ab2 : nullptr);
        if (sa.last) {
          if (DIAG && ab2 >= 0.0)
            vloc = fmax(vloc, atm_cfl_rate<CLEAN>(kp, ab2, __ldg(kp.geo_c + GEO_N * kp.ms + mo)));
          else
            vloc = fmax(vloc, cell_max_speed<YA, ZA, CLEAN, DIAG>(kp, G, Pn, c));
        }
      }
      maxit = max(maxit, it);
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        if constexpr (!MIXED) sa.Uout[f * kp.fs + off] = U[f];  // mixed: stored by recover_stored
        Pout[f * kp.fs + off] = (S)Pn[f];
      }
    }
    if constexpr (STAGE) cp_async_wait_all();  // plane k + 1 staged before the barrier
    __syncthreads();
  }
  }  // z segments of this block
  block_stats<NT>(sc, vloc, nfail, maxit, sa.last != 0);
}

// Conserved state from the primitive state, per cell (FP64 arithmetic on the stored values).
template <bool CLEAN, bool DIAG, bool MIXED>
__global__ void k_prim2cons(const KParams kp, const typename Prec<MIXED>::S* __restrict__ P,
                            const typename Prec<MIXED>::S* __restrict__ M, double* __restrict__ U) {
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const Consts<double> c = consts_of<double>(kp);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % kp.nx);
    const int j = (int)((q / kp.nx) % kp.ny);
    const int k = (int)(q / ((long long)kp.nx * kp.ny));
    const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    double m[10], Pc[9], Uc[9];
    load_metric<DIAG>(kp, M, met_off(kp, i, j, k), m);
#pragma unroll
    for (int f = 0; f < 9; ++f) Pc[f] = (double)P[f * kp.fs + off];
    if (!CLEAN) Pc[8] = 0.0;
    const Geom<double> G = make_geom<DIAG>(m);
    const State<double> S = make_state<DIAG>(G, Pc, c);
    cons_of<CLEAN>(G, S, Uc);
    if (!CLEAN) Uc[8] = 0.0;
#pragma unroll
    for (int f = 0; f < 9; ++f) U[f * kp.fs + off] = Uc[f];
  }
}

template <bool YA, bool ZA, bool CLEAN, bool DIAG, bool MIXED>
__global__ void __launch_bounds__(256) k_max_speed(const KParams kp, const typename Prec<MIXED>::S* __restrict__ P,
                                                   const typename Prec<MIXED>::S* __restrict__ M,
                                                   DevScalars* sc) {
  using R = typename Prec<MIXED>::R;
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const Consts<R> c = consts_of<R>(kp);
  double v = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % kp.nx);
    const int j = (int)((q / kp.nx) % kp.ny);
    const int k = (int)(q / ((long long)kp.nx * kp.ny));
    const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    R m[10], Pc[9];
    load_metric<DIAG>(kp, M, met_off(kp, i, j, k), m);
#pragma unroll
    for (int f = 0; f < 9; ++f) Pc[f] = (R)P[f * kp.fs + off];
    if (!CLEAN) Pc[8] = R(0);
    const Geom<R> G = make_geom<DIAG>(m);
    if constexpr (DIAG && !MIXED) {
      // a cell at rest (the atmosphere, most of a star's grid): the closed form
      if (Pc[P_UX] == 0.0 && Pc[P_UY] == 0.0 && Pc[P_UZ] == 0.0) {
        const double b2 = G.alp * G.alp *
                          (G.gxx * Pc[P_BX] * Pc[P_BX] + G.gyy * Pc[P_BY] * Pc[P_BY] + G.gzz * Pc[P_BZ] * Pc[P_BZ]);
        v = fmax(v, rest_cfl_rate<CLEAN>(kp, Pc[P_RHO], Pc[P_PRS], b2,
                                         __ldg(kp.geo_c + GEO_N * kp.ms + met_off(kp, i, j, k))));
        continue;
      }
    }
    v = fmax(v, cell_max_speed<YA, ZA, CLEAN, DIAG>(kp, G, Pc, c));
  }
  block_stats<256>(sc, v, 0, 0, true);
}

inline int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// One substep launch.  FP64 kernels run on a persistent grid: as many blocks as are resident at
// once (blocks per SM from the occupancy calculator, once per instantiation, times the SMs),
// each taking an equal share of the plane-tiles, at least one.  Mixed
// and double-word kernels: one block per tile column and z chunk.  dyn: the dynamic shared
// memory (the z-face carry of the MC kernels).
template <int TX, int TY, bool YA, bool ZA, bool CLEAN, bool DIAG, bool MIXED, int RECON, bool PAIR>
void launch_substep_one(const KParams& kp, const StageArgs& sa, const typename Prec<MIXED>::S* M,
                        DevScalars* sc, size_t dyn, int zchunks, cudaStream_t st) {
  auto kern = k_substep<TX, TY, YA, ZA, CLEAN, DIAG, MIXED, RECON, PAIR>;
  // once per instantiation and device (function attributes are per device): the dynamic shared
  // memory opt-in and the resident blocks per SM.  The context's device is the current one.
  constexpr int kMaxDev = 64;
  static int per_sm_of[kMaxDev] = {};
  const int dv = kp.dev >= 0 && kp.dev < kMaxDev ? kp.dev : 0;
  int& per_sm = per_sm_of[dv];
  if (per_sm == 0) {
    if (dyn) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TX * TY, dyn) != cudaSuccess || nb < 1)
      nb = 1;
    per_sm = nb;
  }
  if constexpr (MIXED || PAIR) {  // one block per tile column and z chunk (see k_substep)
    const dim3 grid((kp.nx + TX - 1) / TX, (kp.ny + TY - 1) / TY, zchunks);
    kern<<<grid, TX * TY, dyn, st>>>(kp, sa, M, sc);
    return;
  }
  const long long total = (long long)((kp.nx + TX - 1) / TX) * ((kp.ny + TY - 1) / TY) * kp.nz;
  long long g = (long long)per_sm * (kp.nsm > 0 ? kp.nsm : 1);
  // at least one plane-tile per block: a grid with fewer plane-tiles than resident blocks
  // spreads over as many blocks as it has plane-tiles (in 3-D a z segment's first face then
  // costs a full stencil more per plane, which is cheaper than marching 8 planes in series)
  if (g > total) g = total;
  if (g < 1) g = 1;
  kern<<<(unsigned)g, TX * TY, dyn, st>>>(kp, sa, M, sc);
}

// Launchers for one (precision, dimensionality); dispatch on cleaning and metric class.
template <bool YA, bool ZA, bool MIXED, int RECON, bool PAIR = false>
void launch_substep_t(const Variant& v, const KParams& kp, const StageArgs& sa, const void* Mv,
                      DevScalars* sc, int zchunks, cudaStream_t st) {
  // 1-D: one warp of cells per block, so that a short tube spreads over many SMs (each FP64
  // warp instruction occupies an SM's FP64 pipe for 16 cycles; several warps of one block on
  // one SM would serialise)
  constexpr int TX = 32;
  constexpr int TY = (!YA && !ZA) ? 1 : 4;
  using S = typename Prec<MIXED>::S;
  using R = typename FaceType<PAIR, MIXED>::R;
  const S* M = (const S*)Mv;
  // dynamic shared memory: the z-face reconstruction carry of the MC kernels (k_substep)
  constexpr bool ZCARRY = ZA && !PAIR && RECON == 0;
  // and, for the mixed 3-D MC kernels, the staged primitive plane
  constexpr bool STAGE = MIXED && YA && ZA && RECON == 0 && !PAIR;
  const size_t dyn = (ZCARRY ? (size_t)3 * (v.clean ? 9 : 8) * TX * TY * sizeof(R) : 0) +
                     (STAGE ? (size_t)(v.clean ? 9 : 8) * (TX + 4) * (TY + 4) * sizeof(float) : 0);
  if (v.clean) {
    if (v.diag) launch_substep_one<TX, TY, YA, ZA, true, true, MIXED, RECON, PAIR>(kp, sa, M, sc, dyn, zchunks, st);
    else launch_substep_one<TX, TY, YA, ZA, true, false, MIXED, RECON, PAIR>(kp, sa, M, sc, dyn, zchunks, st);
  } else {
    if (v.diag) launch_substep_one<TX, TY, YA, ZA, false, true, MIXED, RECON, PAIR>(kp, sa, M, sc, dyn, zchunks, st);
    else launch_substep_one<TX, TY, YA, ZA, false, false, MIXED, RECON, PAIR>(kp, sa, M, sc, dyn, zchunks, st);
  }
}

// Geometry tables of a DIAG metric (see KParams): one thread per point of the padded metric
// layout; the same arithmetic as the kernels' own make_geom of the centre and face metrics.
template <typename S>
__global__ void k_geo_tables(const KParams kp, const S* __restrict__ M, double* __restrict__ gc,
                             double* __restrict__ gf, double* __restrict__ gs, int faces) {
  const int ya = kp.gy, za = kp.gz;
  const long long n = (long long)(kp.nx + 1) * (kp.ny + ya) * (kp.nz + za);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (kp.nx + 1));
    const int j = (int)((q / (kp.nx + 1)) % (kp.ny + ya));
    const int k = (int)(q / ((long long)(kp.nx + 1) * (kp.ny + ya)));
    const long long mo = met_off(kp, i, j, k);
    const bool cell = i < kp.nx && j < kp.ny && k < kp.nz;
    if (cell) {
      double m[10];
      load_metric<true>(kp, M, mo, m);
      const Geom<double> Gc = make_geom<true>(m);
      geo_store(gc, mo, kp.ms, Gc);
      // CFL rate of a state at rest per unit signal speed: sum_d alpha sqrt(gamma^dd) / dx_d
      double r = Gc.alp * sqrt(Gc.ixx) * kp.idx;
      if (ya) r += Gc.alp * sqrt(Gc.iyy) * kp.idy;
      if (za) r += Gc.alp * sqrt(Gc.izz) * kp.idz;
      gc[GEO_N * kp.ms + mo] = r;
    }
    if (!faces) continue;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if ((d == 1 && !ya) || (d == 2 && !za)) continue;
      // face i - 1/2 along d: needs the index along d in [0, n_d], the others inside
      const bool fin = (d == 0 ? i <= kp.nx : i < kp.nx) && (d == 1 ? j <= kp.ny : j < kp.ny) &&
                       (d == 2 ? k <= kp.nz : k < kp.nz);
      const long long st = d == 0 ? 1 : (d == 1 ? kp.mpitch : kp.mplane);
      if (fin) {
        double m0[10], m1[10], m[10];
        load_metric<true>(kp, M, mo - st, m0);
        load_metric<true>(kp, M, mo, m1);
#pragma unroll
        for (int f = 0; f < 10; ++f) m[f] = 0.5 * (m0[f] + m1[f]);
        const Geom<double> Gf = make_geom<true>(m);
        geo_store(gf + d * GEO_F * kp.ms, mo, kp.ms, Gf);
        gf[(d * GEO_F + GEO_N) * kp.ms + mo] = Gf.alp * sqrt(d == 0 ? Gf.ixx : (d == 1 ? Gf.iyy : Gf.izz));
      }
      if (cell) {
        const G4<double> gp = g4_at<true, double>(kp, M, mo + st), gm = g4_at<true, double>(kp, M, mo - st);
        double* g = gs + d * GEO_S * kp.ms + mo;
        g[0] = gp.gtt - gm.gtt;
        g[kp.ms] = gp.gxx - gm.gxx;
        g[2 * kp.ms] = gp.gyy - gm.gyy;
        g[3 * kp.ms] = gp.gzz - gm.gzz;
      }
    }
  }
}

template <bool YA, bool ZA, bool MIXED>
void launch_max_speed_t(const Variant& v, const KParams& kp, const void* Pv, const void* Mv,
                        DevScalars* sc, cudaStream_t st) {
  using S = typename Prec<MIXED>::S;
  const S* P = (const S*)Pv;
  const S* M = (const S*)Mv;
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const int nb = blocks_for(n, 256);
  if (v.clean) {
    if (v.diag) k_max_speed<YA, ZA, true, true, MIXED><<<nb, 256, 0, st>>>(kp, P, M, sc);
    else k_max_speed<YA, ZA, true, false, MIXED><<<nb, 256, 0, st>>>(kp, P, M, sc);
  } else {
    if (v.diag) k_max_speed<YA, ZA, false, true, MIXED><<<nb, 256, 0, st>>>(kp, P, M, sc);
    else k_max_speed<YA, ZA, false, false, MIXED><<<nb, 256, 0, st>>>(kp, P, M, sc);
  }
}

template <bool MIXED>
void launch_prim2cons_t(const Variant& v, const KParams& kp, const void* Pv, const void* Mv,
                        double* U, cudaStream_t st) {
  using S = typename Prec<MIXED>::S;
  const S* P = (const S*)Pv;
  const S* M = (const S*)Mv;
  const long long n = (long long)kp.nx * kp.ny * kp.nz;
  const int nb = blocks_for(n, 256);
  if (v.clean) {
    if (v.diag) k_prim2cons<true, true, MIXED><<<nb, 256, 0, st>>>(kp, P, M, U);
    else k_prim2cons<true, false, MIXED><<<nb, 256, 0, st>>>(kp, P, M, U);
  } else {
    if (v.diag) k_prim2cons<false, true, MIXED><<<nb, 256, 0, st>>>(kp, P, M, U);
    else k_prim2cons<false, false, MIXED><<<nb, 256, 0, st>>>(kp, P, M, U);
  }
}

#endif  // __CUDACC__

}  // namespace hzn
