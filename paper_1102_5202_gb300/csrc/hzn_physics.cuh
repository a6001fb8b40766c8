// hzn_physics.cuh -- per-point GRMHD physics of the finite-volume update, device side.
//
// State algebra of §2.1 (u^mu, b^mu, T^mu_nu, the conserved vector and the flux vector of
// Eq. 2), the fast-magnetosonic speeds used by the HLLE solver (§2.2, §3.2), the MC limiter
// (§3.2), and the Newton-Raphson recovery of the primitive variables (§2.2, §3.2: the 2D
// scheme in the unknowns Z = rho h W^2 and v^2).  Everything is written for the real type R
// so that the same code serves FP64 and the FP32 parts of the mixed-precision path.
//
// Variables: primitive u~^i = W v^i = u^i + W beta^i / alpha (§5.2 footnote); B^i = *F^{it};
// Eulerian field Bn^i = alpha B^i; enthalpy density w = rho + gamma/(gamma-1) p; magnetic
// pressure b^2/2.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hzn {

// Field indices of the primitive vector, of the conserved vector and of the metric.
enum { P_RHO = 0, P_PRS, P_UX, P_UY, P_UZ, P_BX, P_BY, P_BZ, P_PSI };
enum { U_D = 0, U_TT, U_TX, U_TY, U_TZ, U_BX, U_BY, U_BZ, U_PSI };
enum { M_ALP = 0, M_BX, M_BY, M_BZ, M_GXX, M_GXY, M_GXZ, M_GYY, M_GYZ, M_GZZ };

template <typename R>
struct Consts {
  R gamma;  // adiabatic index
  R gfac;   // gamma / (gamma - 1)
  R ch2;    // cleaning speed squared
};

// 3+1 geometry at one point (face or centre), with the derived quantities the flux, speed and
// source formulas need.  Built from the ten metric values alpha, beta^i, gamma_ij.
template <typename R>
struct Geom {
  R alp, ialp;                      // alpha, 1/alpha
  R bx, by, bz;                     // beta^i
  R blx, bly, blz;                  // beta_i = gamma_ij beta^j
  R gtt;                            // g_tt = -alpha^2 + beta_i beta^i
  R gxx, gxy, gxz, gyy, gyz, gzz;   // gamma_ij
  R ixx, ixy, ixz, iyy, iyz, izz;   // gamma^ij
  R sqrtg, sqrtmg;                  // sqrt(gamma), sqrt(-g) = alpha sqrt(gamma)
};

template <typename R>
__device__ __forceinline__ Geom<R> make_geom(const R m[10]) {
  Geom<R> G;
  G.alp = m[M_ALP];
  G.ialp = R(1) / G.alp;
  G.bx = m[M_BX];
  G.by = m[M_BY];
  G.bz = m[M_BZ];
  G.gxx = m[M_GXX];
  G.gxy = m[M_GXY];
  G.gxz = m[M_GXZ];
  G.gyy = m[M_GYY];
  G.gyz = m[M_GYZ];
  G.gzz = m[M_GZZ];
  const R cxx = G.gyy * G.gzz - G.gyz * G.gyz;
  const R cxy = G.gxz * G.gyz - G.gxy * G.gzz;
  const R cxz = G.gxy * G.gyz - G.gyy * G.gxz;
  const R det = G.gxx * cxx + G.gxy * cxy + G.gxz * cxz;
  const R idet = R(1) / det;
  G.ixx = cxx * idet;
  G.ixy = cxy * idet;
  G.ixz = cxz * idet;
  G.iyy = (G.gxx * G.gzz - G.gxz * G.gxz) * idet;
  G.iyz = (G.gxy * G.gxz - G.gxx * G.gyz) * idet;
  G.izz = (G.gxx * G.gyy - G.gxy * G.gxy) * idet;
  G.sqrtg = sqrt(det);
  G.sqrtmg = G.alp * G.sqrtg;
  G.blx = G.gxx * G.bx + G.gxy * G.by + G.gxz * G.bz;
  G.bly = G.gxy * G.bx + G.gyy * G.by + G.gyz * G.bz;
  G.blz = G.gxz * G.bx + G.gyz * G.by + G.gzz * G.bz;
  G.gtt = -G.alp * G.alp + (G.blx * G.bx + G.bly * G.by + G.blz * G.bz);
  return G;
}

template <int D, typename R>
__device__ __forceinline__ R sel(R x, R y, R z) {
  return D == 0 ? x : (D == 1 ? y : z);
}

// Fluid + field four-vectors of one primitive state.
template <typename R>
struct State {
  R rho, p, w, b2, psi;
  R W, ut, iut;            // Lorentz factor, u^t, 1/u^t
  R ux, uy, uz;            // u^i
  R lx, ly, lz, l_t;       // u_i (= gamma_ij u~^j) and u_t
  R bt, bx, by, bz;        // b^mu
  R b_t, b_x, b_y, b_z;    // b_mu
  R Bx, By, Bz;            // B^i
};

template <typename R>
__device__ __forceinline__ State<R> make_state(const Geom<R>& G, const R P[9], const Consts<R>& c) {
  State<R> S;
  S.rho = P[P_RHO];
  S.p = P[P_PRS];
  S.psi = P[P_PSI];
  const R vx = P[P_UX], vy = P[P_UY], vz = P[P_UZ];
  S.Bx = P[P_BX];
  S.By = P[P_BY];
  S.Bz = P[P_BZ];
  // u_i = gamma_ij u~^j (the shift term of u^i drops out of the spatial covariant part)
  S.lx = G.gxx * vx + G.gxy * vy + G.gxz * vz;
  S.ly = G.gxy * vx + G.gyy * vy + G.gyz * vz;
  S.lz = G.gxz * vx + G.gyz * vy + G.gzz * vz;
  const R q = R(1) + (S.lx * vx + S.ly * vy + S.lz * vz);
  const R rW = rsqrt(q);
  S.W = q * rW;                    // W = sqrt(1 + gamma_ij u~^i u~^j)
  S.ut = S.W * G.ialp;
  S.iut = G.alp * rW;
  S.ux = vx - S.ut * G.bx;         // u^i = u~^i - W beta^i / alpha
  S.uy = vy - S.ut * G.by;
  S.uz = vz - S.ut * G.bz;
  S.l_t = -G.alp * S.W + (G.bx * S.lx + G.by * S.ly + G.bz * S.lz);
  // b^t = B^i u_i ; b^i = (B^i + b^t u^i) / u^t
  S.bt = S.Bx * S.lx + S.By * S.ly + S.Bz * S.lz;
  S.bx = (S.Bx + S.bt * S.ux) * S.iut;
  S.by = (S.By + S.bt * S.uy) * S.iut;
  S.bz = (S.Bz + S.bt * S.uz) * S.iut;
  // b_mu = g_{mu nu} b^nu
  S.b_x = G.blx * S.bt + (G.gxx * S.bx + G.gxy * S.by + G.gxz * S.bz);
  S.b_y = G.bly * S.bt + (G.gxy * S.bx + G.gyy * S.by + G.gyz * S.bz);
  S.b_z = G.blz * S.bt + (G.gxz * S.bx + G.gyz * S.by + G.gzz * S.bz);
  S.b_t = G.gtt * S.bt + (G.blx * S.bx + G.bly * S.by + G.blz * S.bz);
  S.b2 = S.bt * S.b_t + (S.bx * S.b_x + S.by * S.b_y + S.bz * S.b_z);
  S.w = S.rho + c.gfac * S.p;
  return S;
}

// Conserved vector w(u) (§2.2), with Psi = sqrt(gamma) psi.
template <bool CLEAN, typename R>
__device__ __forceinline__ void cons_of(const Geom<R>& G, const State<R>& S, R U[9]) {
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R a = wt * S.ut;
  U[U_D] = G.sqrtmg * S.rho * S.ut;
  U[U_TT] = G.sqrtmg * (a * S.l_t + pt - S.bt * S.b_t);
  U[U_TX] = G.sqrtmg * (a * S.lx - S.bt * S.b_x);
  U[U_TY] = G.sqrtmg * (a * S.ly - S.bt * S.b_y);
  U[U_TZ] = G.sqrtmg * (a * S.lz - S.bt * S.b_z);
  U[U_BX] = G.sqrtmg * S.Bx;
  U[U_BY] = G.sqrtmg * S.By;
  U[U_BZ] = G.sqrtmg * S.Bz;
  if (CLEAN) U[U_PSI] = G.sqrtg * S.psi;
}

// Flux vector along D (§2.1 Eq. 2): sqrt(-g) rho u^D, sqrt(-g) T^D_nu, and the induction flux
// sqrt(-g)(b^j u^D - b^D u^j) = sqrt(-g)(B^j u^D - B^D u^j) / u^t; cleaning adds
// sqrt(-g) gamma^{Dj} psi to B^j and sqrt(gamma)(c_h^2 alpha^2 B^D - beta^D psi) on Psi.
template <int D, bool CLEAN, typename R>
__device__ __forceinline__ void flux_of(const Geom<R>& G, const State<R>& S, const Consts<R>& c,
                                        R F[9]) {
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R bd = sel<D>(S.bx, S.by, S.bz);
  const R a = wt * ud;
  F[U_D] = G.sqrtmg * S.rho * ud;
  F[U_TT] = G.sqrtmg * (a * S.l_t - bd * S.b_t);
  F[U_TX] = G.sqrtmg * (a * S.lx - bd * S.b_x + (D == 0 ? pt : R(0)));
  F[U_TY] = G.sqrtmg * (a * S.ly - bd * S.b_y + (D == 1 ? pt : R(0)));
  F[U_TZ] = G.sqrtmg * (a * S.lz - bd * S.b_z + (D == 2 ? pt : R(0)));
  const R Bd = sel<D>(S.Bx, S.By, S.Bz);
  const R f = G.sqrtmg * S.iut;
  F[U_BX] = D == 0 ? R(0) : f * (S.Bx * ud - Bd * S.ux);
  F[U_BY] = D == 1 ? R(0) : f * (S.By * ud - Bd * S.uy);
  F[U_BZ] = D == 2 ? R(0) : f * (S.Bz * ud - Bd * S.uz);
  if (CLEAN) {
    const R gp = G.sqrtmg * S.psi;
    F[U_BX] += gp * sel<D>(G.ixx, G.ixy, G.ixz);
    F[U_BY] += gp * sel<D>(G.ixy, G.iyy, G.iyz);
    F[U_BZ] += gp * sel<D>(G.ixz, G.iyz, G.izz);
    F[U_PSI] = G.sqrtg * (c.ch2 * G.alp * G.alp * Bd - sel<D>(G.bx, G.by, G.bz) * S.psi);
  }
}

// Squared fast-magnetosonic speed c^2 = cs^2 + vA^2 - cs^2 vA^2 with cs^2 = gamma p / w and
// vA^2 = b^2 / (w + b^2), written over one common denominator.
template <typename R>
__device__ __forceinline__ R cms2_of(const State<R>& S, const Consts<R>& c) {
  const R gp = c.gamma * S.p;
  const R wt = S.w + S.b2;
  return (gp * wt + S.b2 * (S.w - gp)) / (S.w * wt);
}

// Characteristic speeds along D: roots of A l^2 + B l + C = 0 from the dispersion relation
// (u^D - l u^t)^2 = c^2 [g^tt l^2 - 2 g^tD l + g^DD + (u^D - l u^t)^2].
template <int D, typename R>
__device__ __forceinline__ void speeds_of(const Geom<R>& G, const State<R>& S, R c2, R& lm, R& lp) {
  const R ia2 = G.ialp * G.ialp;
  const R bd = sel<D>(G.bx, G.by, G.bz);
  const R gtt = -ia2;
  const R gtd = bd * ia2;
  const R gdd = sel<D>(G.ixx, G.iyy, G.izz) - bd * bd * ia2;
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R oc = R(1) - c2;
  const R A = oc * S.ut * S.ut - c2 * gtt;
  const R B = R(-2) * (oc * S.ut * ud - c2 * gtd);
  const R C = oc * ud * ud - c2 * gdd;
  R disc = B * B - R(4) * A * C;
  disc = disc > R(0) ? disc : R(0);
  const R sq = sqrt(disc);
  const R i2a = R(0.5) / A;
  lp = (-B + sq) * i2a;
  lm = (-B - sq) * i2a;
}

// Coordinate speed bound of the cleaning pair along D: |beta^D| + c_h alpha sqrt(gamma^DD).
template <int D, typename R>
__device__ __forceinline__ void clean_speeds(const Geom<R>& G, R ch, R& lm, R& lp) {
  const R a = ch * G.alp * sqrt(sel<D>(G.ixx, G.iyy, G.izz));
  const R bd = sel<D>(G.bx, G.by, G.bz);
  lm = -bd - a;
  lp = -bd + a;
}

// Monotonized-central limited slope (TVD reconstruction with the MC limiter, §3.2).
template <typename R>
__device__ __forceinline__ R mc_slope(R dm, R dp) {
  const R a = fmin(fmin(R(2) * fabs(dm), R(2) * fabs(dp)), R(0.5) * fabs(dm + dp));
  const R s = dp > R(0) ? a : -a;
  return dm * dp > R(0) ? s : R(0);
}

// ------------------------------------------------------------------------------------------
// Recovery of the primitive state from the conserved one (§2.2: Newton-Raphson, §3.2: the 2D
// scheme).  With normal-observer quantities D = rho W, S_i, E, Bn^i and the unknowns
// Z = w W^2, v^2 the conserved data satisfy
//   r1 = (Z + Bn^2)^2 v^2 - (S.Bn)^2 (2Z + Bn^2) / Z^2 - S^2 = 0
//   r2 = Z - p + Bn^2 (1 + v^2)/2 - (S.Bn)^2 / (2 Z^2) - E = 0,
//   p  = (gamma - 1)/gamma (Z (1 - v^2) - D sqrt(1 - v^2)),
// solved by Newton with the analytic 2x2 Jacobian from the previous primitive state.
// ------------------------------------------------------------------------------------------
struct C2PResult {
  int ok;
  int iters;
};

// Normal-observer invariants of one conserved state: D, E, S^2, (S.Bn)^2, Bn^2, (gamma-1)/gamma.
struct C2PScalars {
  double D, E, S2, SB2, B2, g1;
};

__device__ __forceinline__ double c2p_v2(const C2PScalars& q, double Z) {
  const double ZB = Z + q.B2;
  return (Z * Z * q.S2 + q.SB2 * (2.0 * Z + q.B2)) / (Z * Z * ZB * ZB);
}

// Energy residual with v^2 = v^2(Z) substituted, and its Z derivative.
__device__ __forceinline__ double c2p_f1d(const C2PScalars& q, double Z, double* dfdZ) {
  const double ZB = Z + q.B2;
  const double N = Z * Z * q.S2 + q.SB2 * (2.0 * Z + q.B2);
  const double Dn = Z * Z * ZB * ZB;
  const double v2 = N / Dn;
  const double dv2 = ((2.0 * Z * q.S2 + 2.0 * q.SB2) * Dn - N * (2.0 * Z * ZB * (2.0 * Z + q.B2))) / (Dn * Dn);
  const double sq = sqrt(1.0 - v2);
  const double p = q.g1 * (Z * (1.0 - v2) - q.D * sq);
  const double iZ2 = 1.0 / (Z * Z);
  *dfdZ = 1.0 - q.g1 * (1.0 - v2) - q.g1 * (0.5 * q.D / sq - Z) * dv2 + 0.5 * q.B2 * dv2 +
          q.SB2 * iZ2 / Z;
  return Z - p + 0.5 * q.B2 * (1.0 + v2) - 0.5 * q.SB2 * iZ2 - q.E;
}

// Fallback recovery: Newton on the 1D residual kept inside a bracket [Zlo, gamma E] by
// bisection (the 'rtsafe' safeguard of Press et al.).  gamma E bounds Z from above because
// E >= Z - p >= Z / gamma; Zlo is found by bisection where v^2(Z) drops below 1 - 1e-12.
// Returns false when no root is bracketed (an unphysical conserved state).
__device__ __noinline__ bool c2p_bracketed(const C2PScalars q, double Zguess, double& Zout,
                                           double& v2out, int& iters) {
  const double v2cap = 1.0 - 1e-12;
  const double Zhi = q.E / (1.0 - q.g1);  // gamma E
  if (!(c2p_v2(q, Zhi) < v2cap)) return false;
  double Zlo = Zhi * 1e-100;
  if (!(c2p_v2(q, Zlo) < v2cap)) {
    double a = Zlo, b = Zhi;
    for (int k = 0; k < 400 && b - a > 1e-14 * b; ++k) {
      const double m = 0.5 * (a + b);
      if (c2p_v2(q, m) < v2cap) b = m; else a = m;
    }
    Zlo = b;
  }
  double df;
  if (!(c2p_f1d(q, Zlo, &df) < 0.0)) return false;
  if (!(c2p_f1d(q, Zhi, &df) >= 0.0)) return false;
  double lo = Zlo, hi = Zhi;
  double Z = (Zguess > lo && Zguess < hi) ? Zguess : 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    ++iters;
    const double f = c2p_f1d(q, Z, &df);
    if (f == 0.0) break;
    if (f < 0.0) lo = Z; else hi = Z;
    double Zn = Z - f / df;
    if (!(Zn > lo && Zn < hi)) Zn = 0.5 * (lo + hi);
    const bool conv = fabs(Zn - Z) <= 1e-15 * Z || hi - lo <= 4e-16 * hi;
    Z = Zn;
    if (conv) break;
  }
  const double v2 = c2p_v2(q, Z);
  if (!(v2 < 1.0) || !(Z > 0.0)) return false;
  Zout = Z;
  v2out = v2;
  return true;
}

template <bool CLEAN>
__device__ __forceinline__ C2PResult con2prim(const Geom<double>& G, const double U[9],
                                              const double Pg[9], const Consts<double>& c,
                                              int maxit, double tol, double P[9]) {
  const double isg = 1.0 / G.sqrtg;
  const double D = U[U_D] * isg;
  const double Sx = U[U_TX] * isg, Sy = U[U_TY] * isg, Sz = U[U_TZ] * isg;
  const double Bx = U[U_BX] * isg, By = U[U_BY] * isg, Bz = U[U_BZ] * isg;
  const double E = (-U[U_TT] + (G.bx * U[U_TX] + G.by * U[U_TY] + G.bz * U[U_TZ])) * isg * G.ialp;
  // S^i = gamma^ij S_j ; Bn_i = gamma_ij Bn^j
  const double Sux = G.ixx * Sx + G.ixy * Sy + G.ixz * Sz;
  const double Suy = G.ixy * Sx + G.iyy * Sy + G.iyz * Sz;
  const double Suz = G.ixz * Sx + G.iyz * Sy + G.izz * Sz;
  const double S2 = Sux * Sx + Suy * Sy + Suz * Sz;
  const double Blx = G.gxx * Bx + G.gxy * By + G.gxz * Bz;
  const double Bly = G.gxy * Bx + G.gyy * By + G.gyz * Bz;
  const double Blz = G.gxz * Bx + G.gyz * By + G.gzz * Bz;
  const double B2 = Blx * Bx + Bly * By + Blz * Bz;
  const double SB = Sx * Bx + Sy * By + Sz * Bz;
  const double SB2 = SB * SB;
  const double g1 = (c.gamma - 1.0) / c.gamma;

  C2PResult res;
  res.ok = 0;
  res.iters = 0;
  if (!(D > 0.0) || !(E > 0.0)) return res;

  // initial guess from the previous primitive state
  double Z, v2;
  {
    const double vx = Pg[P_UX], vy = Pg[P_UY], vz = Pg[P_UZ];
    const double uu = (G.gxx * vx + G.gxy * vy + G.gxz * vz) * vx +
                      (G.gxy * vx + G.gyy * vy + G.gyz * vz) * vy +
                      (G.gxz * vx + G.gyz * vy + G.gzz * vz) * vz;
    const double wg = Pg[P_RHO] + c.gfac * Pg[P_PRS];
    Z = wg * (1.0 + uu);
    v2 = uu / (1.0 + uu);
    if (!(Z > 0.0)) Z = E;
  }
  bool done = false;
  int it = 0;
  for (; it < maxit; ++it) {
    const double sq = sqrt(1.0 - v2);
    const double iZ = 1.0 / Z;
    const double iZ2 = iZ * iZ;
    const double ZB = Z + B2;
    const double p = g1 * (Z * (1.0 - v2) - D * sq);
    const double r1 = ZB * ZB * v2 - SB2 * (2.0 * Z + B2) * iZ2 - S2;
    const double r2 = Z - p + 0.5 * B2 * (1.0 + v2) - 0.5 * SB2 * iZ2 - E;
    const double j11 = 2.0 * ZB * v2 + 2.0 * SB2 * ZB * iZ2 * iZ;
    const double j12 = ZB * ZB;
    const double j21 = 1.0 - g1 * (1.0 - v2) + SB2 * iZ2 * iZ;
    const double j22 = g1 * (Z - 0.5 * D / sq) + 0.5 * B2;
    const double idet = 1.0 / (j11 * j22 - j12 * j21);
    const double dZ = -(j22 * r1 - j12 * r2) * idet;
    const double dv = -(j11 * r2 - j21 * r1) * idet;
    double Zn = Z + dZ;
    double vn = v2 + dv;
    if (!(Zn > 0.0)) Zn = 0.5 * Z;
    if (vn < 0.0) vn = 0.0;
    if (!(vn < 1.0)) vn = 0.5 * (v2 + 1.0);
    const bool conv = fabs(dZ) <= tol * Z && fabs(dv) <= tol;
    Z = Zn;
    v2 = vn;
    if (conv) {
      done = true;
      ++it;
      break;
    }
  }
  res.iters = it;
  if (!done || !(v2 < 1.0) || !(Z > 0.0)) {
    // the 2D iteration did not settle: bracketed 1D solve in Z (v^2 eliminated)
    const C2PScalars q = {D, E, S2, SB2, B2, g1};
    if (!c2p_bracketed(q, Z, Z, v2, res.iters)) return res;
  }
  const double rW = sqrt(1.0 - v2);  // 1/W
  const double W = 1.0 / rW;
  const double p = g1 * (Z * (1.0 - v2) - D * rW);
  const double iZB = 1.0 / (Z + B2);
  const double sbz = SB / Z;
  P[P_RHO] = D * rW;
  P[P_PRS] = p;
  P[P_UX] = W * (Sux + sbz * Bx) * iZB;
  P[P_UY] = W * (Suy + sbz * By) * iZB;
  P[P_UZ] = W * (Suz + sbz * Bz) * iZB;
  P[P_BX] = Bx * G.ialp;
  P[P_BY] = By * G.ialp;
  P[P_BZ] = Bz * G.ialp;
  P[P_PSI] = CLEAN ? U[U_PSI] * isg : 0.0;
  res.ok = 1;
  return res;
}

}  // namespace hzn
