// hzn_adjoint.cuh -- reverse-mode (adjoint) physics of one face and one cell, device side.
//
// Hand-written reverses of the state algebra, conserved vector, flux vector and
// fast-magnetosonic speeds of hzn_physics.cuh (§2.1 Eq. 2, §2.2), of the HLLE flux of one face
// with its frozen wave-speed bounds, of the MC slope with its frozen case (§3.2), of the metric
// source, and the implicit-function adjoint of the primitive recovery (§2.2).  The metric is
// held fixed (it is not differentiated).  Every function computes a vector-Jacobian product:
// given the adjoint ("bar") of its outputs it adds the adjoint of its inputs.  The two kernels
// of a reverse substep (k_adj_face, k_adj_cell) and their host launchers close the file; each
// metric class (diagonal, general) is instantiated in its own unit (hzn_adj_diag.cu,
// hzn_adj_general.cu).
#pragma once

#include "hzn_adj.h"
#include "hzn_internal.h"
#include "hzn_physics.cuh"

namespace hzn {
namespace adj {

// Boundary index of a stencil position q (any integer): wrapped (periodic) or clamped (outflow).
__device__ __forceinline__ int bc_idx(int q, int n, int periodic) {
  if (periodic) {
    q %= n;
    return q < 0 ? q + n : q;
  }
  return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

// Reverse-mode adjoints ("bars") of the quantities of State.
struct SBar {
  double rho, p, w, b2, psi;
  double W, ut, iut;
  double ux, uy, uz;        // u^i
  double lx, ly, lz, l_t;   // u_i, u_t
  double bt, bx, by, bz;    // b^mu
  double b_t, b_x, b_y, b_z;
  double Bx, By, Bz;
};

__device__ __forceinline__ void zero(SBar& s) {
  s.rho = s.p = s.w = s.b2 = s.psi = 0.0;
  s.W = s.ut = s.iut = 0.0;
  s.ux = s.uy = s.uz = 0.0;
  s.lx = s.ly = s.lz = s.l_t = 0.0;
  s.bt = s.bx = s.by = s.bz = 0.0;
  s.b_t = s.b_x = s.b_y = s.b_z = 0.0;
  s.Bx = s.By = s.Bz = 0.0;
}

template <int D>
__device__ __forceinline__ double& selr(double& x, double& y, double& z) {
  return D == 0 ? x : (D == 1 ? y : z);
}

// Reverse of make_state (metric held fixed): adds dJ/dP to Pb.  DIAG: zero shift and diagonal
// gamma_ij, whose identically zero terms are dropped (as make_state<true> drops them).
template <bool DIAG>
__device__ __forceinline__ void state_rev(const Geom<double>& G, const State<double>& S,
                                          const double P[9], double gfac, SBar& s, double Pb[9]) {
  // b^2 = b^t b_t + b^i b_i
  s.bt += s.b2 * S.b_t;
  s.b_t += s.b2 * S.bt;
  s.bx += s.b2 * S.b_x;
  s.by += s.b2 * S.b_y;
  s.bz += s.b2 * S.b_z;
  s.b_x += s.b2 * S.bx;
  s.b_y += s.b2 * S.by;
  s.b_z += s.b2 * S.bz;
  // b_t = g_tt b^t + beta_i b^i ; b_i = beta_i b^t + gamma_ij b^j
  s.bt += G.gtt * s.b_t;
  if constexpr (DIAG) {
    s.bx += G.gxx * s.b_x;
    s.by += G.gyy * s.b_y;
    s.bz += G.gzz * s.b_z;
  } else {
    s.bx += G.blx * s.b_t;
    s.by += G.bly * s.b_t;
    s.bz += G.blz * s.b_t;
    s.bt += G.blx * s.b_x + G.bly * s.b_y + G.blz * s.b_z;
    s.bx += G.gxx * s.b_x + G.gxy * s.b_y + G.gxz * s.b_z;
    s.by += G.gxy * s.b_x + G.gyy * s.b_y + G.gyz * s.b_z;
    s.bz += G.gxz * s.b_x + G.gyz * s.b_y + G.gzz * s.b_z;
  }
  // b^i = (B^i + b^t u^i) / u^t ; B^i + b^t u^i = b^i u^t
  s.Bx += S.iut * s.bx;
  s.By += S.iut * s.by;
  s.Bz += S.iut * s.bz;
  s.bt += S.iut * (S.ux * s.bx + S.uy * s.by + S.uz * s.bz);
  s.ux += S.bt * S.iut * s.bx;
  s.uy += S.bt * S.iut * s.by;
  s.uz += S.bt * S.iut * s.bz;
  s.iut += S.ut * (S.bx * s.bx + S.by * s.by + S.bz * s.bz);
  // b^t = B^i u_i
  s.Bx += S.lx * s.bt;
  s.By += S.ly * s.bt;
  s.Bz += S.lz * s.bt;
  s.lx += S.Bx * s.bt;
  s.ly += S.By * s.bt;
  s.lz += S.Bz * s.bt;
  // u^i = u~^i - u^t beta^i
  Pb[P_UX] += s.ux;
  Pb[P_UY] += s.uy;
  Pb[P_UZ] += s.uz;
  // u_t = -alpha W + beta^i u_i
  s.W -= G.alp * s.l_t;
  if constexpr (!DIAG) {
    s.ut -= G.bx * s.ux + G.by * s.uy + G.bz * s.uz;
    s.lx += G.bx * s.l_t;
    s.ly += G.by * s.l_t;
    s.lz += G.bz * s.l_t;
  }
  // u^t = W / alpha, 1/u^t = alpha / W
  const double iW = rcp_fast(S.W);
  s.W += s.ut * G.ialp - s.iut * S.iut * iW;
  // W = sqrt(q), q = 1 + u_i u~^i
  const double qb = 0.5 * s.W * iW;
  s.lx += P[P_UX] * qb;
  s.ly += P[P_UY] * qb;
  s.lz += P[P_UZ] * qb;
  Pb[P_UX] += S.lx * qb;
  Pb[P_UY] += S.ly * qb;
  Pb[P_UZ] += S.lz * qb;
  // u_i = gamma_ij u~^j
  if constexpr (DIAG) {
    Pb[P_UX] += G.gxx * s.lx;
    Pb[P_UY] += G.gyy * s.ly;
    Pb[P_UZ] += G.gzz * s.lz;
  } else {
    Pb[P_UX] += G.gxx * s.lx + G.gxy * s.ly + G.gxz * s.lz;
    Pb[P_UY] += G.gxy * s.lx + G.gyy * s.ly + G.gyz * s.lz;
    Pb[P_UZ] += G.gxz * s.lx + G.gyz * s.ly + G.gzz * s.lz;
  }
  // w = rho + gamma/(gamma-1) p
  Pb[P_RHO] += s.rho + s.w;
  Pb[P_PRS] += s.p + gfac * s.w;
  Pb[P_BX] += s.Bx;
  Pb[P_BY] += s.By;
  Pb[P_BZ] += s.Bz;
  Pb[P_PSI] += s.psi;
}

// Reverse of cons_of: conserved-vector adjoint Ub into the state bars.
template <bool CLEAN>
__device__ __forceinline__ void cons_rev(const Geom<double>& G, const State<double>& S,
                                         const double Ub[9], SBar& s) {
  const double sg = G.sqrtmg;
  const double wt = S.w + S.b2;
  s.rho += sg * S.ut * Ub[U_D];
  s.ut += sg * S.rho * Ub[U_D];
  const double u0 = sg * Ub[U_TT], ux = sg * Ub[U_TX], uy = sg * Ub[U_TY], uz = sg * Ub[U_TZ];
  const double lsum = u0 * S.l_t + ux * S.lx + uy * S.ly + uz * S.lz;
  const double bsum = u0 * S.b_t + ux * S.b_x + uy * S.b_y + uz * S.b_z;
  const double wtb = S.ut * lsum;
  s.ut += wt * lsum;
  const double a = wt * S.ut;
  s.l_t += a * u0;
  s.lx += a * ux;
  s.ly += a * uy;
  s.lz += a * uz;
  s.bt -= bsum;
  s.b_t -= S.bt * u0;
  s.b_x -= S.bt * ux;
  s.b_y -= S.bt * uy;
  s.b_z -= S.bt * uz;
  const double ptb = u0;
  s.Bx += sg * Ub[U_BX];
  s.By += sg * Ub[U_BY];
  s.Bz += sg * Ub[U_BZ];
  if (CLEAN) s.psi += G.sqrtg * Ub[U_PSI];
  s.w += wtb;
  s.b2 += wtb + 0.5 * ptb;
  s.p += ptb;
}

// Reverse of flux_of along D: flux adjoint Fb into the state bars.
template <int D, bool CLEAN, bool DIAG>
__device__ __forceinline__ void flux_rev(const Geom<double>& G, const State<double>& S,
                                         const Consts<double>& c, const double Fb[9], SBar& s) {
  const double sg = G.sqrtmg;
  const double wt = S.w + S.b2;
  const double ud = sel<D>(S.ux, S.uy, S.uz), bd = sel<D>(S.bx, S.by, S.bz);
  double udb = 0.0, bdb = 0.0;
  // sqrt(-g) rho u^D
  s.rho += sg * ud * Fb[U_D];
  udb += sg * S.rho * Fb[U_D];
  // sqrt(-g) (w_t u^D u_nu - b^D b_nu + delta^D_nu p_t)
  const double f0 = sg * Fb[U_TT], fx = sg * Fb[U_TX], fy = sg * Fb[U_TY], fz = sg * Fb[U_TZ];
  const double lsum = f0 * S.l_t + fx * S.lx + fy * S.ly + fz * S.lz;
  const double bsum = f0 * S.b_t + fx * S.b_x + fy * S.b_y + fz * S.b_z;
  const double wtb = ud * lsum;
  udb += wt * lsum;
  const double a = wt * ud;
  s.l_t += a * f0;
  s.lx += a * fx;
  s.ly += a * fy;
  s.lz += a * fz;
  bdb -= bsum;
  s.b_t -= bd * f0;
  s.b_x -= bd * fx;
  s.b_y -= bd * fy;
  s.b_z -= bd * fz;
  const double ptb = sel<D>(fx, fy, fz);
  // induction: sqrt(-g) (B^j u^D - B^D u^j) / u^t for j != D
  const double Bd = sel<D>(S.Bx, S.By, S.Bz);
  const double gx = D == 0 ? 0.0 : sg * Fb[U_BX];
  const double gy = D == 1 ? 0.0 : sg * Fb[U_BY];
  const double gz = D == 2 ? 0.0 : sg * Fb[U_BZ];
  s.iut += gx * (S.Bx * ud - Bd * S.ux) + gy * (S.By * ud - Bd * S.uy) + gz * (S.Bz * ud - Bd * S.uz);
  const double ti = S.iut;
  s.Bx += gx * ti * ud;
  s.By += gy * ti * ud;
  s.Bz += gz * ti * ud;
  udb += ti * (gx * S.Bx + gy * S.By + gz * S.Bz);
  double Bdb = -ti * (gx * S.ux + gy * S.uy + gz * S.uz);
  s.ux -= gx * ti * Bd;
  s.uy -= gy * ti * Bd;
  s.uz -= gz * ti * Bd;
  if (CLEAN) {
    // sqrt(-g) gamma^{Dj} psi on B^j; sqrt(gamma)(c_h^2 alpha^2 B^D - beta^D psi) on Psi
    if constexpr (DIAG) {
      s.psi += sg * sel<D>(G.ixx, G.iyy, G.izz) * Fb[U_BX + D];
    } else {
      s.psi += sg * (sel<D>(G.ixx, G.ixy, G.ixz) * Fb[U_BX] + sel<D>(G.ixy, G.iyy, G.iyz) * Fb[U_BY] +
                     sel<D>(G.ixz, G.iyz, G.izz) * Fb[U_BZ]) -
               G.sqrtg * sel<D>(G.bx, G.by, G.bz) * Fb[U_PSI];
    }
    Bdb += G.sqrtg * c.ch2 * G.alp * G.alp * Fb[U_PSI];
  }
  selr<D>(s.ux, s.uy, s.uz) += udb;
  selr<D>(s.bx, s.by, s.bz) += bdb;
  selr<D>(s.Bx, s.By, s.Bz) += Bdb;
  s.w += wtb;
  s.b2 += wtb + 0.5 * ptb;
  s.p += ptb;
}

// Reverse of cms2_of + speeds_of along D: adjoints lmb, lpb of the two roots into the bars.
template <int D, bool DIAG>
__device__ __forceinline__ void speeds_rev(const Geom<double>& G, const State<double>& S,
                                           const Consts<double>& c, double lmb, double lpb,
                                           SBar& s) {
  if (lmb == 0.0 && lpb == 0.0) return;
  const double gp = c.gamma * S.p;
  const double wt = S.w + S.b2;
  const double N = gp * wt + S.b2 * (S.w - gp), Dd = S.w * wt;
  const double iDd = rcp_fast(Dd);
  const double c2 = N * iDd;
  const double ia2 = G.ialp * G.ialp;
  const double ud = sel<D>(S.ux, S.uy, S.uz);
  const double oc = 1.0 - c2;
  const double bd = DIAG ? 0.0 : sel<D>(G.bx, G.by, G.bz);
  const double gtd = DIAG ? 0.0 : bd * ia2;
  const double gdd = DIAG ? sel<D>(G.ixx, G.iyy, G.izz) : sel<D>(G.ixx, G.iyy, G.izz) - bd * bd * ia2;
  const double A = oc * S.ut * S.ut + c2 * ia2;
  const double B = -2.0 * (oc * S.ut * ud - c2 * gtd);
  const double C = oc * ud * ud - c2 * gdd;
  const double disc = B * B - 4.0 * A * C;
  const double rsq = disc > 0.0 ? rsqrt(disc) : 0.0;
  const double sq = disc * rsq;
  const double i2a = 0.5 * rcp_fast(A);
  const double lp = (-B + sq) * i2a, lm = (-B - sq) * i2a;
  double Ab = -(lpb * lp + lmb * lm) * (i2a + i2a);  // / A
  double Bb = -i2a * (lpb + lmb);
  double Cb = 0.0;
  if (disc > 0.0) {
    const double discb = i2a * (lpb - lmb) * 0.5 * rsq;
    Bb += 2.0 * B * discb;
    Ab -= 4.0 * C * discb;
    Cb -= 4.0 * A * discb;
  }
  double ocb = Ab * S.ut * S.ut - 2.0 * Bb * S.ut * ud + Cb * ud * ud;
  const double utb = 2.0 * Ab * oc * S.ut - 2.0 * Bb * oc * ud;
  const double udb = -2.0 * Bb * oc * S.ut + 2.0 * Cb * oc * ud;
  double c2b = Ab * ia2 + 2.0 * Bb * gtd - Cb * gdd - ocb;
  const double Nb = c2b * iDd, Ddb = -c2b * c2 * iDd;
  const double gpb = Nb * (wt - S.b2);
  const double wtb = Nb * gp + Ddb * S.w;
  s.b2 += Nb * (S.w - gp) + wtb;
  s.w += Nb * S.b2 + Ddb * wt + wtb;
  s.p += c.gamma * gpb;
  s.ut += utb;
  selr<D>(s.ux, s.uy, s.uz) += udb;
}

// Frozen MC case of the slope sigma = cm dm + cp dp (sigma = 2 dm, 2 dp or (dm + dp)/2, or 0
// when dm and dp do not share a strict sign); ties go to the earlier argument of
// min(2|dm|, 2|dp|, |dm + dp|/2), as in the plain FP64 formulation of §3.2.
__device__ __forceinline__ void mc_coef(double dm, double dp, double& cm, double& cp) {
  cm = cp = 0.0;
  if (dm == 0.0 || dp == 0.0 || ((dm > 0.0) != (dp > 0.0))) return;
  const double x1 = 2.0 * fabs(dm), x2 = 2.0 * fabs(dp), x3 = 0.5 * fabs(dm + dp);
  int which = x2 < x1 ? 2 : 1;
  const double m = which == 2 ? x2 : x1;
  if (x3 < m) which = 3;
  if (which == 1) cm = 2.0;
  else if (which == 2) cp = 2.0;
  else cm = cp = 0.5;
}

// Face reverse along D at the face i - 1/2 of cell (i, j, k): recompute the face state, then
// push the face-flux adjoint Fb back to the reconstructed left / right primitive states.
template <int D, bool CLEAN, bool DIAG>
__device__ void face_rev(const KParams& kp, const double* __restrict__ P, const double* __restrict__ M,
                         int i, int j, int k, const double Fb[9], double PLb[9], double PRb[9]) {
  constexpr int NV = CLEAN ? 9 : 8;
  long long off[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int ii = i, jj = j, kk = k;
    if (D == 0) ii = bc_idx(i + s - 2, kp.nx, kp.bcx);
    if (D == 1) jj = bc_idx(j + s - 2, kp.ny, kp.bcy);
    if (D == 2) kk = bc_idx(k + s - 2, kp.nz, kp.bcz);
    off[s] = (long long)kk * kp.plane + (long long)jj * kp.pitch + ii;
  }
  double PL[9], PR[9];
#pragma unroll
  for (int f = 0; f < NV; ++f) {
    const double* pf = P + f * kp.fs;
    const double a = pf[off[0]], b = pf[off[1]], cc = pf[off[2]], d = pf[off[3]];
    PL[f] = b + mc_half_slope(b - a, cc - b);
    PR[f] = cc - mc_half_slope(cc - b, d - cc);
  }
  if (!CLEAN) PL[8] = PR[8] = 0.0;
  const long long o1 = (long long)(k + kp.gz) * kp.mplane + (long long)(j + kp.gy) * kp.mpitch + (i + kp.gx);
  Geom<double> G;
  if constexpr (DIAG) {
    // face geometry of the diagonal metric from its table
    G = geo_load<double>(kp.geo_f + D * GEO_F * kp.ms, o1, kp.ms);
  } else {
    double m[10];
    const long long o0 = o1 - (D == 0 ? 1 : (D == 1 ? kp.mpitch : kp.mplane));
#pragma unroll
    for (int f = 0; f < 10; ++f) m[f] = 0.5 * (M[f * kp.ms + o0] + M[f * kp.ms + o1]);
    G = make_geom<false>(m);
  }
  Consts<double> c;
  c.gamma = kp.gamma;
  c.gfac = kp.gfac;
  c.ch = kp.ch;
  c.ch2 = kp.ch * kp.ch;
  const State<double> SL = make_state<DIAG>(G, PL, c), SR = make_state<DIAG>(G, PR, c);
  double FL[9], UL[9], FR[9], UR[9], lmL, lpL, lmR, lpR;
  flux_of<D, CLEAN, DIAG>(G, SL, c, FL);
  cons_of<CLEAN>(G, SL, UL);
  speeds_of<D, DIAG>(G, SL, cms2_of(SL, c), lmL, lpL);
  flux_of<D, CLEAN, DIAG>(G, SR, c, FR);
  cons_of<CLEAN>(G, SR, UR);
  speeds_of<D, DIAG>(G, SR, cms2_of(SR, c), lmR, lpR);
  if (!CLEAN) FL[8] = FR[8] = UL[8] = UR[8] = 0.0;
  // frozen wave-speed bounds: sL = min(0, lmL, lmR), sR = max(0, lpL, lpR)
  const bool mr = lmR < lmL;
  const double mi = mr ? lmR : lmL;
  const bool sl_on = mi < 0.0;
  const double sl = sl_on ? mi : 0.0;
  const bool pr = lpL < lpR;
  const double pi = pr ? lpR : lpL;
  const bool sr_on = 0.0 < pi;
  const double sr = sr_on ? pi : 0.0;
  const double den = sr - sl;
  const double iden = den != 0.0 ? rcp_fast(den) : 0.0;
  double FLb[9], FRb[9], ULb[9], URb[9];
  double slb = 0.0, srb = 0.0;
  const int fb = U_BX + D;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    FLb[q] = FRb[q] = ULb[q] = URb[q] = 0.0;
    if (q >= NV) continue;
    if (CLEAN && (q == fb || q == U_PSI)) continue;
    const double g = Fb[q];
    if (den != 0.0) {
      const double dU = UR[q] - UL[q];
      const double F = (sr * FL[q] - sl * FR[q] + sl * sr * dU) * iden;
      FLb[q] = sr * iden * g;
      FRb[q] = -sl * iden * g;
      URb[q] = sl * sr * iden * g;
      ULb[q] = -URb[q];
      srb += g * (FL[q] + sl * dU - F) * iden;
      slb += g * (-FR[q] + sr * dU + F) * iden;
    } else {
      FLb[q] = FRb[q] = 0.5 * g;
    }
  }
  if (CLEAN) {
    // the pair (B^D, Psi) with the metric-only cleaning speeds
    double cm, cp;
    clean_speeds<D, DIAG>(G, c.ch, cm, cp);
    const double csl = fmin(0.0, cm), csr = fmax(0.0, cp);
    const double cden = csr - csl;
    const double ic = rcp_fast(cden);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int q = t == 0 ? fb : U_PSI;
      const double g = Fb[q];
      FLb[q] = csr * ic * g;
      FRb[q] = -csl * ic * g;
      URb[q] = csl * csr * ic * g;
      ULb[q] = -URb[q];
    }
  }
  const double lmLb = (sl_on && !mr) ? slb : 0.0, lmRb = (sl_on && mr) ? slb : 0.0;
  const double lpLb = (sr_on && !pr) ? srb : 0.0, lpRb = (sr_on && pr) ? srb : 0.0;
#pragma unroll
  for (int f = 0; f < 9; ++f) PLb[f] = PRb[f] = 0.0;
  {
    SBar s;
    zero(s);
    flux_rev<D, CLEAN, DIAG>(G, SL, c, FLb, s);
    cons_rev<CLEAN>(G, SL, ULb, s);
    speeds_rev<D, DIAG>(G, SL, c, lmLb, lpLb, s);
    state_rev<DIAG>(G, SL, PL, c.gfac, s, PLb);
  }
  {
    SBar s;
    zero(s);
    flux_rev<D, CLEAN, DIAG>(G, SR, c, FRb, s);
    cons_rev<CLEAN>(G, SR, URb, s);
    speeds_rev<D, DIAG>(G, SR, c, lmRb, lpRb, s);
    state_rev<DIAG>(G, SR, PR, c.gfac, s, PRb);
  }
  if (!CLEAN) PLb[8] = PRb[8] = 0.0;
}

// Reverse of the metric source 1/2 sqrt(-g) T^{ab} d_i g_ab (centred differences) and of the
// cleaning damping -kappa alpha sqrt(gamma) psi at one cell, given lam_L there.
template <bool CLEAN, bool DIAG>
__device__ __forceinline__ void source_rev(const KParams& kp, const double* __restrict__ M, long long mo,
                           const Geom<double>& G, const State<double>& S, const double Pc[9],
                           const double Lb[9], const Consts<double>& c, double Pb[9]) {
  // Mb[10] = sum_i lam_L[T_i] h (0.5/dx_i) (g(+i) - g(-i)), components tt, tx, ty, tz (beta_i),
  // xx, xy, xz, yy, yz, zz; off-diagonal components enter T^{ab} d g_ab twice.
  double Mb[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) Mb[q] = 0.0;
  const double h = 0.5 * G.sqrtmg;
  bool any = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int act = d == 0 ? 1 : (d == 1 ? kp.gy : kp.gz);
    if (!act) continue;
    const double wgt = Lb[U_TX + d] * h * 0.5 * (d == 0 ? kp.idx : (d == 1 ? kp.idy : kp.idz));
    if (wgt == 0.0) continue;
    if constexpr (DIAG) {
      // tabulated differences of g_tt, g_xx, g_yy, g_zz (the only nonzero components)
      const double* g = kp.geo_s + d * GEO_S * kp.ms + mo;
      const double dtt = g[0], dxx = g[kp.ms], dyy = g[2 * kp.ms], dzz = g[3 * kp.ms];
      if (dtt != 0.0 || dxx != 0.0 || dyy != 0.0 || dzz != 0.0) any = true;
      Mb[0] += wgt * dtt;
      Mb[4] += wgt * dxx;
      Mb[7] += wgt * dyy;
      Mb[9] += wgt * dzz;
      continue;
    }
    const long long st = d == 0 ? 1 : (d == 1 ? kp.mpitch : kp.mplane);
    double gp[10], gm[10];
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      gp[f] = M[f * kp.ms + mo + st];
      gm[f] = M[f * kp.ms + mo - st];
    }
    // 4-metric components at the two neighbours
    double g4p[10], g4m[10];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double* m = t == 0 ? gp : gm;
      double* o = t == 0 ? g4p : g4m;
      const double blx = m[M_GXX] * m[M_BX] + m[M_GXY] * m[M_BY] + m[M_GXZ] * m[M_BZ];
      const double bly = m[M_GXY] * m[M_BX] + m[M_GYY] * m[M_BY] + m[M_GYZ] * m[M_BZ];
      const double blz = m[M_GXZ] * m[M_BX] + m[M_GYZ] * m[M_BY] + m[M_GZZ] * m[M_BZ];
      o[0] = -m[M_ALP] * m[M_ALP] + (blx * m[M_BX] + bly * m[M_BY] + blz * m[M_BZ]);
      o[1] = blx;
      o[2] = bly;
      o[3] = blz;
      o[4] = m[M_GXX];
      o[5] = m[M_GXY];
      o[6] = m[M_GXZ];
      o[7] = m[M_GYY];
      o[8] = m[M_GYZ];
      o[9] = m[M_GZZ];
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const double dg = g4p[q] - g4m[q];
      if (dg != 0.0) any = true;
      const double two = (q == 0 || q == 4 || q == 7 || q == 9) ? 1.0 : 2.0;
      Mb[q] += wgt * two * dg;
    }
  }
  if (CLEAN) Pb[P_PSI] += -kp.kappa * G.alp * G.sqrtg * Lb[U_PSI];
  if (!any) return;
  // T^{ab} = w_t u^a u^b + p_t g^{ab} - b^a b^b, components in the order of Mb
  const double ia2 = G.ialp * G.ialp;
  const double u4[4] = {S.ut, S.ux, S.uy, S.uz};
  const double b4[4] = {S.bt, S.bx, S.by, S.bz};
  const double wt = S.w + S.b2;
  double wtb = 0.0, ptb = 0.0, u4b[4] = {0, 0, 0, 0}, b4b[4] = {0, 0, 0, 0};
  if constexpr (DIAG) {
    // diagonal components tt, xx, yy, zz only
    const double gi[4] = {-ia2, G.ixx, G.iyy, G.izz};
    const int qd[4] = {0, 4, 7, 9};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double t = Mb[qd[a]];
      wtb += t * u4[a] * u4[a];
      ptb += t * gi[a];
      u4b[a] += 2.0 * t * wt * u4[a];
      b4b[a] -= 2.0 * t * b4[a];
    }
  } else {
  const double gi[10] = {-ia2, G.bx * ia2, G.by * ia2, G.bz * ia2,
                         G.ixx - G.bx * G.bx * ia2, G.ixy - G.bx * G.by * ia2,
                         G.ixz - G.bx * G.bz * ia2, G.iyy - G.by * G.by * ia2,
                         G.iyz - G.by * G.bz * ia2, G.izz - G.bz * G.bz * ia2};
  const int ia[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
  const int ib[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const double t = Mb[q];
    const int a = ia[q], b = ib[q];
    wtb += t * u4[a] * u4[b];
    ptb += t * gi[q];
    u4b[a] += t * wt * u4[b];
    u4b[b] += t * wt * u4[a];
    b4b[a] -= t * b4[b];
    b4b[b] -= t * b4[a];
  }
  }
  SBar s;
  zero(s);
  s.w += wtb;
  s.b2 += wtb + 0.5 * ptb;
  s.p += ptb;
  s.ut += u4b[0];
  s.ux += u4b[1];
  s.uy += u4b[2];
  s.uz += u4b[3];
  s.bt += b4b[0];
  s.bx += b4b[1];
  s.by += b4b[2];
  s.bz += b4b[3];
  state_rev<DIAG>(G, S, Pc, c.gfac, s, Pb);
}

// (dU/dP)^T v at one state: the conserved-vector adjoint v pushed back to the primitives.
template <bool CLEAN, bool DIAG>
__device__ __forceinline__ void cons_vjp(const Geom<double>& G, const State<double>& S,
                                         const double Pc[9], const Consts<double>& c,
                                         const double v[9], double out[9]) {
  SBar s;
  zero(s);
  cons_rev<CLEAN>(G, S, v, s);
  state_rev<DIAG>(G, S, Pc, c.gfac, s, out);
}

// One column of the elimination (partial pivoting) of the 5 x 5 system; COL is a template
// argument so that every array index is known at compile time and the arrays stay in registers.
template <int COL>
__device__ __forceinline__ void elim5(double At[5][5], double r[5], double inv[5]) {
  if constexpr (COL < 5) {
    int piv = COL;
    double best = fabs(At[COL][COL]);
#pragma unroll
    for (int rr = COL + 1; rr < 5; ++rr)
      if (fabs(At[rr][COL]) > best) {
        best = fabs(At[rr][COL]);
        piv = rr;
      }
#pragma unroll
    for (int rr = COL + 1; rr < 5; ++rr) {
      if (rr == piv) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const double t = At[COL][q];
          At[COL][q] = At[rr][q];
          At[rr][q] = t;
        }
        const double t = r[COL];
        r[COL] = r[rr];
        r[rr] = t;
      }
    }
    inv[COL] = rcp_fast(At[COL][COL]);
#pragma unroll
    for (int rr = COL + 1; rr < 5; ++rr) {
      const double fct = At[rr][COL] * inv[COL];
#pragma unroll
      for (int q = COL; q < 5; ++q) At[rr][q] -= fct * At[COL][q];
      r[rr] -= fct * r[COL];
    }
    elim5<COL + 1>(At, r, inv);
  }
}

// Solve A^T x = r for the 5 x 5 hydrodynamic block (partial pivoting; back substitution with
// the pivots' reciprocals).  At[m][k] = dU_k/dP_m.
__device__ __forceinline__ void solve5(double At[5][5], double r[5]) {
  double inv[5];
  elim5<0>(At, r, inv);
#pragma unroll
  for (int col = 4; col >= 0; --col) {
    double t = r[col];
#pragma unroll
    for (int q = col + 1; q < 5; ++q) t -= At[col][q] * r[q];
    r[col] = t * inv[col];
  }
}

// Row KQ of dU/dP (the conserved component KQ against every primitive) by one VJP with the
// unit vector e_KQ; KQ is a template argument so that every index is known at compile time.
template <int KQ, bool CLEAN, bool DIAG>
__device__ __forceinline__ void jac_row(const Geom<double>& G, const State<double>& S,
                                        const double Pc[9], const Consts<double>& c,
                                        double At[5][5], double Cb[5][3]) {
  double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  e[KQ] = 1.0;
  double row[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  cons_vjp<CLEAN, DIAG>(G, S, Pc, c, e, row);
#pragma unroll
  for (int m = 0; m < 5; ++m) At[m][KQ] = row[m];
#pragma unroll
  for (int q = 0; q < 3; ++q) Cb[KQ][q] = row[P_BX + q];
}

// mu = (dU/dP)^{-T} lamP at the state (implicit-function adjoint of the recovery).
template <bool CLEAN, bool DIAG>
__device__ __forceinline__ void ift(const Geom<double>& G, const State<double>& S, const double Pc[9],
                    const Consts<double>& c, const double lamP[9], double mu[9]) {
  // rows k of dU/dP for the hydrodynamic components D, T_t, T_x, T_y, T_z
  double At[5][5], Cb[5][3];
  jac_row<0, CLEAN, DIAG>(G, S, Pc, c, At, Cb);
  jac_row<1, CLEAN, DIAG>(G, S, Pc, c, At, Cb);
  jac_row<2, CLEAN, DIAG>(G, S, Pc, c, At, Cb);
  jac_row<3, CLEAN, DIAG>(G, S, Pc, c, At, Cb);
  jac_row<4, CLEAN, DIAG>(G, S, Pc, c, At, Cb);
  double x[5] = {lamP[0], lamP[1], lamP[2], lamP[3], lamP[4]};
  solve5(At, x);
  const double isg = rcp_fast(G.sqrtmg);
#pragma unroll
  for (int m = 0; m < 5; ++m) mu[m] = x[m];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double t = lamP[P_BX + q];
#pragma unroll
    for (int kq = 0; kq < 5; ++kq) t -= Cb[kq][q] * x[kq];
    mu[P_BX + q] = t * isg;
  }
  mu[8] = CLEAN ? lamP[8] * rcp_fast(G.sqrtg) : 0.0;
}

#ifdef __CUDACC__  // the kernels and their launchers (the reverse physics above also builds for the host)
// One thread per face of every active axis: flux adjoint from lam_L, face reverse, store the
// adjoints of the two reconstructed states.
template <bool CLEAN, bool DIAG>
__global__ void __launch_bounds__(128) k_adj_face(const KParams kp, const AdjShape sh,
                                                  const double* __restrict__ P,
                                                  const double* __restrict__ M, AdjBufs bufs) {
  const int D = blockIdx.y;
  const int nxf = kp.nx + (D == 0), nyf = kp.ny + (D == 1), nzf = kp.nz + (D == 2);
  const long long nfaces = (long long)nxf * nyf * nzf;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nfaces;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nxf);
    const int j = (int)((q / nxf) % nyf);
    const int k = (int)(q / ((long long)nxf * nyf));
    const int id = D == 0 ? i : (D == 1 ? j : k);
    const int nd = D == 0 ? kp.nx : (D == 1 ? kp.ny : kp.nz);
    const double idd = D == 0 ? kp.idx : (D == 1 ? kp.idy : kp.idz);
    const long long cR = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    const long long step = D == 0 ? 1 : (D == 1 ? kp.pitch : kp.plane);
    double Fb[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      const double r = id < nd ? bufs.lamL[f * kp.fs + cR] : 0.0;
      const double l = id >= 1 ? bufs.lamL[f * kp.fs + cR - step] : 0.0;
      Fb[f] = (r - l) * idd;
    }
    double PLb[9], PRb[9];
    if (D == 0) face_rev<0, CLEAN, DIAG>(kp, P, M, i, j, k, Fb, PLb, PRb);
    else if (D == 1) face_rev<1, CLEAN, DIAG>(kp, P, M, i, j, k, Fb, PLb, PRb);
    else face_rev<2, CLEAN, DIAG>(kp, P, M, i, j, k, Fb, PLb, PRb);
    const long long fo = (long long)k * sh.fplane + (long long)j * sh.fpitch + i;
    double* fl = D == 0 ? bufs.fL[0] : (D == 1 ? bufs.fL[1] : bufs.fL[2]);
    double* fr = D == 0 ? bufs.fR[0] : (D == 1 ? bufs.fR[1] : bufs.fR[2]);
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      fl[f * sh.ffs + fo] = PLb[f];
      fr[f * sh.ffs + fo] = PRb[f];
    }
  }
}

// Adjoint gathered along D at cell (i, j, k): the contributions of every virtual stencil
// position v that reads this cell (v = the cell itself, plus the ghost positions that copy it
// under the boundary condition).
template <int D, int NV>
__device__ __forceinline__ void gather_axis(const KParams& kp, const AdjShape& sh,
                                            const double* __restrict__ P, const AdjBufs& bufs,
                                            int i, int j, int k, double lamP[9]) {
  const int n = D == 0 ? kp.nx : (D == 1 ? kp.ny : kp.nz);
  const int bc = D == 0 ? kp.bcx : (D == 1 ? kp.bcy : kp.bcz);
  const int c = D == 0 ? i : (D == 1 ? j : k);
  int vs[3];
  int nv = 0;
  vs[nv++] = c;
  if (bc) {
    if (c == 0) vs[nv++] = n;
    if (c == 1) vs[nv++] = n + 1;
    if (c == n - 1) vs[nv++] = -1;
    if (c == n - 2 && nv < 3) vs[nv++] = -2;
  } else {
    if (c == 0) {
      vs[nv++] = -1;
      vs[nv++] = -2;
    } else if (c == n - 1) {
      vs[nv++] = n;
      vs[nv++] = n + 1;
    }
  }
  const double* fl = bufs.fL[D];
  const double* fr = bufs.fR[D];
  for (int t = 0; t < nv; ++t) {
    const int v = vs[t];
    long long po[5];  // primitive offsets of positions v-2 .. v+2 (clamped / wrapped)
    long long fo[4];  // face offsets of faces v-1 .. v+2 (face q between cells q-1 and q)
    bool fok[4];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int q = bc_idx(v + s - 2, n, bc);
      const int ii = D == 0 ? q : i, jj = D == 1 ? q : j, kk = D == 2 ? q : k;
      po[s] = (long long)kk * kp.plane + (long long)jj * kp.pitch + ii;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int q = v - 1 + s;
      fok[s] = q >= 0 && q <= n;
      const int qq = fok[s] ? q : 0;
      const int ii = D == 0 ? qq : i, jj = D == 1 ? qq : j, kk = D == 2 ? qq : k;
      fo[s] = (long long)kk * sh.fplane + (long long)jj * sh.fpitch + ii;
    }
#pragma unroll
    for (int f = 0; f < NV; ++f) {
      const double* pf = P + f * kp.fs;
      double p[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) p[s] = pf[po[s]];
      double L[4], R[4];  // lam of the left / right state at faces v-1 .. v+2
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        L[s] = fok[s] ? fl[f * sh.ffs + fo[s]] : 0.0;
        R[s] = fok[s] ? fr[f * sh.ffs + fo[s]] : 0.0;
      }
      // face v+1/2 (index 2) takes its left state from v; face v-1/2 (index 1) its right state
      double acc = L[2] + R[1];
      // slopes of u = v-1, v, v+1: lam_sigma_u = (lam_L(face u+1/2) - lam_R(face u-1/2)) / 2
      double cm, cp;
      const double gsm = 0.5 * (L[1] - R[0]);
      if (gsm != 0.0) {
        mc_coef(p[1] - p[0], p[2] - p[1], cm, cp);
        acc += cp * gsm;
      }
      const double gs0 = 0.5 * (L[2] - R[1]);
      if (gs0 != 0.0) {
        mc_coef(p[2] - p[1], p[3] - p[2], cm, cp);
        acc += (cm - cp) * gs0;
      }
      const double gsp = 0.5 * (L[3] - R[2]);
      if (gsp != 0.0) {
        mc_coef(p[3] - p[2], p[4] - p[3], cm, cp);
        acc -= cm * gsp;
      }
      lamP[f] += acc;
    }
  }
}

// One thread per cell: (1) lam_P at the boundary state Pb -- gathered from the faces of the
// later substep plus its source reverse, or read from lamP; (2) the implicit-function step of
// the earlier substep (or, at the initial state, the adjoint of the initial primitives).
template <bool CLEAN, bool DIAG>
__global__ void __launch_bounds__(128) k_adj_cell(const KParams kp, const AdjShape sh,
                                                  const double* __restrict__ Pb,
                                                  const double* __restrict__ M, AdjBufs bufs) {
  constexpr int NV = CLEAN ? 9 : 8;
  const long long ncell = (long long)kp.nx * kp.ny * kp.nz;
  Consts<double> c;
  c.gamma = kp.gamma;
  c.gfac = kp.gfac;
  c.ch = kp.ch;
  c.ch2 = kp.ch * kp.ch;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % kp.nx);
    const int j = (int)((q / kp.nx) % kp.ny);
    const int k = (int)(q / ((long long)kp.nx * kp.ny));
    const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
    const long long mo = (long long)(k + kp.gz) * kp.mplane + (long long)(j + kp.gy) * kp.mpitch + (i + kp.gx);
    double Pc[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) Pc[f] = f < NV ? Pb[f * kp.fs + off] : 0.0;
    Geom<double> G;
    if constexpr (DIAG) {
      G = geo_load<double>(kp.geo_c, mo, kp.ms);
    } else {
      double m[10];
#pragma unroll
      for (int f = 0; f < 10; ++f) m[f] = M[f * kp.ms + mo];
      G = make_geom<false>(m);
    }
    const State<double> S = make_state<DIAG>(G, Pc, c);
    double lamP[9];
    if (sh.gather) {
#pragma unroll
      for (int f = 0; f < 9; ++f) lamP[f] = 0.0;
      gather_axis<0, NV>(kp, sh, Pb, bufs, i, j, k, lamP);
      if (kp.ny > 1) gather_axis<1, NV>(kp, sh, Pb, bufs, i, j, k, lamP);
      if (kp.nz > 1) gather_axis<2, NV>(kp, sh, Pb, bufs, i, j, k, lamP);
      double Lb[9];
#pragma unroll
      for (int f = 0; f < 9; ++f) Lb[f] = f < NV ? bufs.lamL[f * kp.fs + off] : 0.0;
      source_rev<CLEAN, DIAG>(kp, M, mo, G, S, Pc, Lb, c, lamP);
    } else {
#pragma unroll
      for (int f = 0; f < 9; ++f) lamP[f] = f < NV ? bufs.lamP[f * kp.fs + off] : 0.0;
    }
    double lamU[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) lamU[f] = f < NV ? bufs.lamU[f * kp.fs + off] : 0.0;
    if (sh.stage == 3) {
      // initial state: U(0) = w(P(0)), so lam_P(0) += (dU/dP)^T lam_U(0)
      cons_vjp<CLEAN, DIAG>(G, S, Pc, c, lamU, lamP);
#pragma unroll
      for (int f = 0; f < NV; ++f) bufs.out[f * kp.fs + off] = lamP[f];
      continue;
    }
    // frozen recovery outcome at Pb: atmosphere reset, pressure floor, or a plain recovery
    const bool atm = Pc[P_RHO] == kp.rho_floor && Pc[P_PRS] == kp.p_atm && Pc[P_UX] == 0.0 &&
                     Pc[P_UY] == 0.0 && Pc[P_UZ] == 0.0;
    const bool pfl = !atm && Pc[P_PRS] == kp.p_floor;
    double mu[9];
    if (atm || pfl) {
      // the reset rewrote U = w(P): fold lam_U into lam_P first
      double tot[9];
#pragma unroll
      for (int f = 0; f < 9; ++f) tot[f] = lamP[f];
      cons_vjp<CLEAN, DIAG>(G, S, Pc, c, lamU, tot);
      if (atm) {
        // only B (and psi) of the atmosphere state depend on the conserved input
#pragma unroll
        for (int f = 0; f < 5; ++f) mu[f] = 0.0;
#pragma unroll
        for (int f = 0; f < 3; ++f) mu[P_BX + f] = tot[P_BX + f] / G.sqrtmg;
        mu[8] = CLEAN ? tot[8] / G.sqrtg : 0.0;
      } else {
        tot[P_PRS] = 0.0;
        ift<CLEAN, DIAG>(G, S, Pc, c, tot, mu);
      }
    } else {
      ift<CLEAN, DIAG>(G, S, Pc, c, lamP, mu);
#pragma unroll
      for (int f = 0; f < 9; ++f) mu[f] += lamU[f];
    }
#pragma unroll
    for (int f = 0; f < NV; ++f) {
      const long long o = f * kp.fs + off;
      bufs.lamL[o] = sh.b * sh.dt * mu[f];
      double acc;
      if (sh.stage == 2) acc = sh.a * mu[f];
      else acc = bufs.lamA[o] + sh.a * mu[f];
      if (sh.stage == 0) {
        bufs.lamU[o] = sh.b * mu[f] + acc;
      } else {
        bufs.lamU[o] = sh.b * mu[f];
        bufs.lamA[o] = acc;
      }
    }
  }
}

// Host launchers (declared in hzn_adj.h, instantiated once per metric class).
template <bool DIAG>
void adj_launch_cell(bool clean, int blocks, int threads, cudaStream_t st, const KParams& kp,
                     const AdjShape& sh, const double* Pb, const double* M, const AdjBufs& bufs) {
  if (clean) k_adj_cell<true, DIAG><<<blocks, threads, 0, st>>>(kp, sh, Pb, M, bufs);
  else k_adj_cell<false, DIAG><<<blocks, threads, 0, st>>>(kp, sh, Pb, M, bufs);
}

template <bool DIAG>
void adj_launch_face(bool clean, dim3 grid, int threads, cudaStream_t st, const KParams& kp,
                     const AdjShape& sh, const double* P, const double* M, const AdjBufs& bufs) {
  if (clean) k_adj_face<true, DIAG><<<grid, threads, 0, st>>>(kp, sh, P, M, bufs);
  else k_adj_face<false, DIAG><<<grid, threads, 0, st>>>(kp, sh, P, M, bufs);
}

#endif  // __CUDACC__

}  // namespace adj
}  // namespace hzn
