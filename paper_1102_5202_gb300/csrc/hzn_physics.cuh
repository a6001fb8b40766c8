// hzn_physics.cuh -- per-point GRMHD physics of the finite-volume update, device side.
//
// State algebra of §2.1 (u^mu, b^mu, T^mu_nu, the conserved vector and the flux vector of
// Eq. 2), the fast-magnetosonic speeds used by the HLLE solver (§2.2, §3.2), the MC limiter
// (§3.2), and the Newton-Raphson recovery of the primitive variables (§2.2, §3.2: the 2D
// scheme in the unknowns Z = rho h W^2 and v^2).
//
// Everything is written for the real type R (double for the FP64 path; float for the face,
// flux and source work of the mixed-precision path; the double-word f32x2 of hzn_f32x2.cuh for
// the pair path) and for two metric classes: DIAG (zero
// shift, diagonal gamma_ij -- Minkowski, isotropic and conformally flat static metrics) and
// the general 3+1 metric.  DIAG drops terms that are identically zero, nothing else.
//
// Variables: primitive u~^i = W v^i = u^i + W beta^i / alpha (§5.2 footnote); B^i = *F^{it};
// Eulerian field Bn^i = alpha B^i; enthalpy density w = rho + gamma/(gamma-1) p; magnetic
// pressure b^2/2.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hzn_f32x2.cuh"

namespace hzn {

// Field indices of the primitive vector, of the conserved vector and of the metric.
enum { P_RHO = 0, P_PRS, P_UX, P_UY, P_UZ, P_BX, P_BY, P_BZ, P_PSI };
enum { U_D = 0, U_TT, U_TX, U_TY, U_TZ, U_BX, U_BY, U_BZ, U_PSI };
enum { M_ALP = 0, M_BX, M_BY, M_BZ, M_GXX, M_GXY, M_GXZ, M_GYY, M_GYZ, M_GZZ };

template <typename R>
struct Consts {
  R gamma;  // adiabatic index
  R gfac;   // gamma / (gamma - 1)
  R ch;     // cleaning speed
  R ch2;    // cleaning speed squared
};

// Quotient and square root in the FP32 arithmetic of the mixed path's faces and of the
// recovery's FP32 stage: the hardware approximations (__fdividef, within 2 ulps; x rsqrtf(x))
// instead of the correctly rounded sequences, which that arithmetic's own rounding does not
// need.  FP64 and double-word values keep the correctly rounded operations.
template <typename R>
__device__ __forceinline__ R fdiv(R a, R b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
template <typename R>
__device__ __forceinline__ R fsqrt(R x) { return sqrt(x); }
__device__ __forceinline__ float fsqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

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

template <bool DIAG, typename R>
__device__ __forceinline__ Geom<R> make_geom(const R m[10]) {
  Geom<R> G;
  G.alp = m[M_ALP];
  G.ialp = fdiv(R(1), G.alp);
  G.gxx = m[M_GXX];
  G.gyy = m[M_GYY];
  G.gzz = m[M_GZZ];
  if constexpr (DIAG) {
    G.bx = G.by = G.bz = R(0);
    G.blx = G.bly = G.blz = R(0);
    G.gxy = G.gxz = G.gyz = R(0);
    G.ixy = G.ixz = G.iyz = R(0);
    const R gyz2 = G.gyy * G.gzz;
    const R det = G.gxx * gyz2;
    const R idet = fdiv(R(1), det);
    G.ixx = gyz2 * idet;
    G.iyy = (G.gxx * G.gzz) * idet;
    G.izz = (G.gxx * G.gyy) * idet;
    G.sqrtg = fsqrt(det);
    G.gtt = -G.alp * G.alp;
  } else {
    G.bx = m[M_BX];
    G.by = m[M_BY];
    G.bz = m[M_BZ];
    G.gxy = m[M_GXY];
    G.gxz = m[M_GXZ];
    G.gyz = m[M_GYZ];
    const R cxx = G.gyy * G.gzz - G.gyz * G.gyz;
    const R cxy = G.gxz * G.gyz - G.gxy * G.gzz;
    const R cxz = G.gxy * G.gyz - G.gyy * G.gxz;
    const R det = G.gxx * cxx + G.gxy * cxy + G.gxz * cxz;
    const R idet = fdiv(R(1), det);
    G.ixx = cxx * idet;
    G.ixy = cxy * idet;
    G.ixz = cxz * idet;
    G.iyy = (G.gxx * G.gzz - G.gxz * G.gxz) * idet;
    G.iyz = (G.gxy * G.gxz - G.gxx * G.gyz) * idet;
    G.izz = (G.gxx * G.gyy - G.gxy * G.gxy) * idet;
    G.sqrtg = fsqrt(det);
    G.blx = G.gxx * G.bx + G.gxy * G.by + G.gxz * G.bz;
    G.bly = G.gxy * G.bx + G.gyy * G.by + G.gyz * G.bz;
    G.blz = G.gxz * G.bx + G.gyz * G.by + G.gzz * G.bz;
    G.gtt = -G.alp * G.alp + (G.blx * G.bx + G.bly * G.by + G.blz * G.bz);
  }
  G.sqrtmg = G.alp * G.sqrtg;
  return G;
}

// Geometry of a DIAG metric from a table of GEO_N fields at stride ms (alpha, 1/alpha, gamma_xx,
// _yy, _zz, gamma^xx, ^yy, ^zz, sqrt(gamma), sqrt(-g)): the values make_geom<true> computes.
template <typename R>
__device__ __forceinline__ Geom<R> geo_load(const double* __restrict__ g, long long off, long long ms) {
  Geom<R> G;
  G.alp = ldc<R>(g + off);
  G.ialp = ldc<R>(g + ms + off);
  G.gxx = ldc<R>(g + 2 * ms + off);
  G.gyy = ldc<R>(g + 3 * ms + off);
  G.gzz = ldc<R>(g + 4 * ms + off);
  G.ixx = ldc<R>(g + 5 * ms + off);
  G.iyy = ldc<R>(g + 6 * ms + off);
  G.izz = ldc<R>(g + 7 * ms + off);
  G.sqrtg = ldc<R>(g + 8 * ms + off);
  G.sqrtmg = ldc<R>(g + 9 * ms + off);
  G.bx = G.by = G.bz = R(0);
  G.blx = G.bly = G.blz = R(0);
  G.gxy = G.gxz = G.gyz = R(0);
  G.ixy = G.ixz = G.iyz = R(0);
  G.gtt = -G.alp * G.alp;
  return G;
}

template <typename R>
__device__ __forceinline__ void geo_store(double* __restrict__ g, long long off, long long ms,
                                          const Geom<R>& G) {
  g[off] = G.alp;
  g[ms + off] = G.ialp;
  g[2 * ms + off] = G.gxx;
  g[3 * ms + off] = G.gyy;
  g[4 * ms + off] = G.gzz;
  g[5 * ms + off] = G.ixx;
  g[6 * ms + off] = G.iyy;
  g[7 * ms + off] = G.izz;
  g[8 * ms + off] = G.sqrtg;
  g[9 * ms + off] = G.sqrtmg;
}

// 1/x from the hardware reciprocal approximation (rcp.approx.ftz.f64) refined by two steps of
// the Newton-Raphson iteration for the reciprocal, r <- r + r (1 - x r) (Newton's method on
// f(r) = 1/r - x; each step squares the relative error, so the approximation's error falls to
// a few ulps): a few FP64 instructions fewer than the correctly rounded quotient.  x must be a
// normal number.  float: the plain quotient.
__device__ __forceinline__ double rcp_fast(double x) {
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
#else
  return 1.0 / x;
#endif
}
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }

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

template <bool DIAG, typename R>
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
  if constexpr (DIAG) {
    S.lx = G.gxx * vx;
    S.ly = G.gyy * vy;
    S.lz = G.gzz * vz;
  } else {
    S.lx = G.gxx * vx + G.gxy * vy + G.gxz * vz;
    S.ly = G.gxy * vx + G.gyy * vy + G.gyz * vz;
    S.lz = G.gxz * vx + G.gyz * vy + G.gzz * vz;
  }
  const R q = R(1) + (S.lx * vx + S.ly * vy + S.lz * vz);
  const R rW = rsqrt(q);
  S.W = q * rW;                    // W = sqrt(1 + gamma_ij u~^i u~^j)
  S.ut = S.W * G.ialp;
  S.iut = G.alp * rW;
  // b^t = B^i u_i
  S.bt = S.Bx * S.lx + S.By * S.ly + S.Bz * S.lz;
  if constexpr (DIAG) {
    S.ux = vx;                     // u^i = u~^i - W beta^i / alpha, zero shift
    S.uy = vy;
    S.uz = vz;
    S.l_t = -G.alp * S.W;
  } else {
    S.ux = vx - S.ut * G.bx;
    S.uy = vy - S.ut * G.by;
    S.uz = vz - S.ut * G.bz;
    S.l_t = -G.alp * S.W + (G.bx * S.lx + G.by * S.ly + G.bz * S.lz);
  }
  // b^i = (B^i + b^t u^i) / u^t ; b_mu = g_{mu nu} b^nu
  S.bx = (S.Bx + S.bt * S.ux) * S.iut;
  S.by = (S.By + S.bt * S.uy) * S.iut;
  S.bz = (S.Bz + S.bt * S.uz) * S.iut;
  if constexpr (DIAG) {
    S.b_x = G.gxx * S.bx;
    S.b_y = G.gyy * S.by;
    S.b_z = G.gzz * S.bz;
    S.b_t = G.gtt * S.bt;
  } else {
    S.b_x = G.blx * S.bt + (G.gxx * S.bx + G.gxy * S.by + G.gxz * S.bz);
    S.b_y = G.bly * S.bt + (G.gxy * S.bx + G.gyy * S.by + G.gyz * S.bz);
    S.b_z = G.blz * S.bt + (G.gxz * S.bx + G.gyz * S.by + G.gzz * S.bz);
    S.b_t = G.gtt * S.bt + (G.blx * S.bx + G.bly * S.by + G.blz * S.bz);
  }
  S.b2 = S.bt * S.b_t + (S.bx * S.b_x + S.by * S.b_y + S.bz * S.b_z);
  S.w = S.rho + c.gfac * S.p;
  return S;
}

// Conserved vector w(u) (§2.2), with Psi = sqrt(gamma) psi.  UNSCALED: the vector divided by
// sqrt(-g) (Psi by sqrt(-g) as well, i.e. psi / alpha); a face flux scales once at the end.
template <bool CLEAN, bool UNSCALED = false, typename R>
__device__ __forceinline__ void cons_of(const Geom<R>& G, const State<R>& S, R U[9]) {
  const R sg = UNSCALED ? R(1) : G.sqrtmg;
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R a = wt * S.ut;
  U[U_D] = sg * S.rho * S.ut;
  U[U_TT] = sg * (a * S.l_t + pt - S.bt * S.b_t);
  U[U_TX] = sg * (a * S.lx - S.bt * S.b_x);
  U[U_TY] = sg * (a * S.ly - S.bt * S.b_y);
  U[U_TZ] = sg * (a * S.lz - S.bt * S.b_z);
  U[U_BX] = sg * S.Bx;
  U[U_BY] = sg * S.By;
  U[U_BZ] = sg * S.Bz;
  if (CLEAN) U[U_PSI] = (UNSCALED ? G.ialp : G.sqrtg) * S.psi;
}

// Flux vector along D (§2.1 Eq. 2): sqrt(-g) rho u^D, sqrt(-g) T^D_nu, and the induction flux
// sqrt(-g)(b^j u^D - b^D u^j) = sqrt(-g)(B^j u^D - B^D u^j) / u^t; cleaning adds
// sqrt(-g) gamma^{Dj} psi to B^j and sqrt(gamma)(c_h^2 alpha^2 B^D - beta^D psi) on Psi.
// UNSCALED: the flux divided by sqrt(-g), as for cons_of.
template <int D, bool CLEAN, bool DIAG, bool UNSCALED = false, typename R>
__device__ __forceinline__ void flux_of(const Geom<R>& G, const State<R>& S, const Consts<R>& c,
                                        R F[9]) {
  const R sg = UNSCALED ? R(1) : G.sqrtmg;
  const R sgp = UNSCALED ? G.ialp : G.sqrtg;  // scale of Psi
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R bd = sel<D>(S.bx, S.by, S.bz);
  const R a = wt * ud;
  F[U_D] = sg * S.rho * ud;
  F[U_TT] = sg * (a * S.l_t - bd * S.b_t);
  F[U_TX] = sg * (a * S.lx - bd * S.b_x + (D == 0 ? pt : R(0)));
  F[U_TY] = sg * (a * S.ly - bd * S.b_y + (D == 1 ? pt : R(0)));
  F[U_TZ] = sg * (a * S.lz - bd * S.b_z + (D == 2 ? pt : R(0)));
  const R Bd = sel<D>(S.Bx, S.By, S.Bz);
  const R f = sg * S.iut;
  F[U_BX] = D == 0 ? R(0) : f * (S.Bx * ud - Bd * S.ux);
  F[U_BY] = D == 1 ? R(0) : f * (S.By * ud - Bd * S.uy);
  F[U_BZ] = D == 2 ? R(0) : f * (S.Bz * ud - Bd * S.uz);
  if (CLEAN) {
    const R gp = sg * S.psi;
    if constexpr (DIAG) {
      if (D == 0) F[U_BX] += gp * G.ixx;
      if (D == 1) F[U_BY] += gp * G.iyy;
      if (D == 2) F[U_BZ] += gp * G.izz;
      F[U_PSI] = sgp * (c.ch2 * G.alp * G.alp * Bd);
    } else {
      F[U_BX] += gp * sel<D>(G.ixx, G.ixy, G.ixz);
      F[U_BY] += gp * sel<D>(G.ixy, G.iyy, G.iyz);
      F[U_BZ] += gp * sel<D>(G.ixz, G.iyz, G.izz);
      F[U_PSI] = sgp * (c.ch2 * G.alp * G.alp * Bd - sel<D>(G.bx, G.by, G.bz) * S.psi);
    }
  }
}

// Centre 4-metric quantities used by the source: g_tt, beta_i, gamma_ij at one cell.
template <typename R>
struct G4 {
  R gtt, blx, bly, blz, gxx, gxy, gxz, gyy, gyz, gzz;
};

// Contravariant stress-energy T^{ab} = (w + b^2) u^a u^b + (p + b^2/2) g^{ab} - b^a b^b.
template <typename R>
struct Tup {
  R tt, tx, ty, tz, xx, xy, xz, yy, yz, zz;
};

template <bool DIAG, typename R>
__device__ __forceinline__ Tup<R> tup_of(const Geom<R>& G, const State<R>& S) {
  const R wt = S.w + S.b2, pt = S.p + R(0.5) * S.b2;
  const R ia2 = G.ialp * G.ialp;
  Tup<R> T;
  T.tt = wt * S.ut * S.ut - pt * ia2 - S.bt * S.bt;
  if constexpr (DIAG) {
    T.tx = wt * S.ut * S.ux - S.bt * S.bx;
    T.ty = wt * S.ut * S.uy - S.bt * S.by;
    T.tz = wt * S.ut * S.uz - S.bt * S.bz;
    T.xx = wt * S.ux * S.ux + pt * G.ixx - S.bx * S.bx;
    T.yy = wt * S.uy * S.uy + pt * G.iyy - S.by * S.by;
    T.zz = wt * S.uz * S.uz + pt * G.izz - S.bz * S.bz;
    T.xy = T.xz = T.yz = R(0);  // multiplied by identically zero metric derivatives
  } else {
    T.tx = wt * S.ut * S.ux + pt * G.bx * ia2 - S.bt * S.bx;
    T.ty = wt * S.ut * S.uy + pt * G.by * ia2 - S.bt * S.by;
    T.tz = wt * S.ut * S.uz + pt * G.bz * ia2 - S.bt * S.bz;
    T.xx = wt * S.ux * S.ux + pt * (G.ixx - G.bx * G.bx * ia2) - S.bx * S.bx;
    T.xy = wt * S.ux * S.uy + pt * (G.ixy - G.bx * G.by * ia2) - S.bx * S.by;
    T.xz = wt * S.ux * S.uz + pt * (G.ixz - G.bx * G.bz * ia2) - S.bx * S.bz;
    T.yy = wt * S.uy * S.uy + pt * (G.iyy - G.by * G.by * ia2) - S.by * S.by;
    T.yz = wt * S.uy * S.uz + pt * (G.iyz - G.by * G.bz * ia2) - S.by * S.bz;
    T.zz = wt * S.uz * S.uz + pt * (G.izz - G.bz * G.bz * ia2) - S.bz * S.bz;
  }
  return T;
}

// T^{ab} (g_ab(+) - g_ab(-)) between the neighbours gp and gm (unscaled centred difference).
template <bool DIAG, typename R>
__device__ __forceinline__ R tdg(const Tup<R>& T, const G4<R>& gp, const G4<R>& gm) {
  R s = T.tt * (gp.gtt - gm.gtt) + T.xx * (gp.gxx - gm.gxx) + T.yy * (gp.gyy - gm.gyy) +
        T.zz * (gp.gzz - gm.gzz);
  if constexpr (!DIAG)
    s += R(2) * (T.tx * (gp.blx - gm.blx) + T.ty * (gp.bly - gm.bly) + T.tz * (gp.blz - gm.blz) +
                 T.xy * (gp.gxy - gm.gxy) + T.xz * (gp.gxz - gm.gxz) + T.yz * (gp.gyz - gm.gyz));
  return s;
}

// Squared fast-magnetosonic speed c^2 = cs^2 + vA^2 - cs^2 vA^2 with cs^2 = gamma p / w and
// vA^2 = b^2 / (w + b^2), written over one common denominator.
// FAST (FP64 only): the quotient through rcp_fast (within a few ulps of the correctly rounded one).
template <typename R, bool FAST = false>
__device__ __forceinline__ R cms2_of(const State<R>& S, const Consts<R>& c) {
  const R gp = c.gamma * S.p;
  const R wt = S.w + S.b2;
  if constexpr (FAST) return (gp * wt + S.b2 * (S.w - gp)) * rcp_fast(S.w * wt);
  else return fdiv(gp * wt + S.b2 * (S.w - gp), S.w * wt);
}

// Characteristic speeds along D: roots of A l^2 + B l + C = 0 from the dispersion relation
// (u^D - l u^t)^2 = c^2 [g^tt l^2 - 2 g^tD l + g^DD + (u^D - l u^t)^2].
// FAST (FP64 only): the square root as disc / sqrt(disc) through the reciprocal square root and
// 1 / (2A) through rcp_fast (each within a few ulps of the correctly rounded value).
template <int D, bool DIAG, typename R, bool FAST = false>
__device__ __forceinline__ void speeds_of(const Geom<R>& G, const State<R>& S, R c2, R& lm, R& lp) {
  const R ia2 = G.ialp * G.ialp;
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R oc = R(1) - c2;
  const R A = oc * S.ut * S.ut + c2 * ia2;  // - c^2 g^tt, g^tt = -1/alpha^2
  R B, C;
  if constexpr (DIAG) {
    B = R(-2) * (oc * S.ut * ud);
    C = oc * ud * ud - c2 * sel<D>(G.ixx, G.iyy, G.izz);
  } else {
    const R bd = sel<D>(G.bx, G.by, G.bz);
    const R gtd = bd * ia2;
    const R gdd = sel<D>(G.ixx, G.iyy, G.izz) - bd * bd * ia2;
    B = R(-2) * (oc * S.ut * ud - c2 * gtd);
    C = oc * ud * ud - c2 * gdd;
  }
  R disc = B * B - R(4) * A * C;
  disc = disc > R(0) ? disc : R(0);
  R sq, i2a;
  if constexpr (FAST) {
    sq = disc > R(0) ? disc * rsqrt(disc) : R(0);
    i2a = R(0.5) * rcp_fast(A);
  } else {
    sq = fsqrt(disc);
    i2a = fdiv(R(0.5), A);
  }
  lp = (-B + sq) * i2a;
  lm = (-B - sq) * i2a;
}

// The same quadratic multiplied through by w (w + b^2), so that c^2 = N / Dd enters without a
// division: A' = (Dd - N) (u^t)^2 + N / alpha^2, B', C' likewise, with B' halved: returns A',
// b = B' / 2 and sq = sqrt(max(b^2 - A'C', 0)); the roots, the speeds, are (-b +- sq) / A'.
template <int D, bool DIAG, typename R>
__device__ __forceinline__ void speed_quadratic(const Geom<R>& G, const State<R>& S, const Consts<R>& c,
                                                R& A, R& B, R& sq) {
  const R gp = c.gamma * S.p;
  const R wt = S.w + S.b2;
  const R N = gp * wt + S.b2 * (S.w - gp);
  const R Dd = S.w * wt;
  const R ia2 = G.ialp * G.ialp;
  const R ud = sel<D>(S.ux, S.uy, S.uz);
  const R oc = Dd - N;
  A = oc * S.ut * S.ut + N * ia2;
  R C;
  if constexpr (DIAG) {
    B = -(oc * S.ut * ud);
    C = oc * ud * ud - N * sel<D>(G.ixx, G.iyy, G.izz);
  } else {
    const R bd = sel<D>(G.bx, G.by, G.bz);
    const R gtd = bd * ia2;
    const R gdd = sel<D>(G.ixx, G.iyy, G.izz) - bd * bd * ia2;
    B = -(oc * S.ut * ud - N * gtd);
    C = oc * ud * ud - N * gdd;
  }
  R disc = B * B - A * C;
  // sqrt as disc / sqrt(disc) through the reciprocal square root (a few FP64 instructions
  // fewer than the correctly rounded square root; the speeds set the HLLE bounds only)
  sq = disc > R(0) ? disc * rsqrt(disc) : R(0);
}

// Characteristic speeds of the cleaning pair (B^D, Psi) along D:
// -beta^D / 2 -+ sqrt((beta^D / 2)^2 + c_h^2 alpha^2 gamma^DD), i.e. -+ c_h alpha sqrt(gamma^DD)
// with zero shift.
template <int D, bool DIAG, typename R>
__device__ __forceinline__ void clean_speeds(const Geom<R>& G, R ch, R& lm, R& lp) {
  const R a = ch * G.alp * fsqrt(sel<D>(G.ixx, G.iyy, G.izz));
  if constexpr (DIAG) {
    lm = -a;
    lp = a;
  } else {
    // roots of l^2 + beta^D l - a^2 = 0: the pair's fluxes are alpha gamma^DD Psi and
    // c_h^2 alpha sqrt(-g) B^D - beta^D Psi
    const R hb = R(0.5) * sel<D>(G.bx, G.by, G.bz);
    const R r = fsqrt(hb * hb + a * a);
    lm = -hb - r;
    lp = -hb + r;
  }
}

// Half of the monotonized-central limited slope (TVD reconstruction with the MC limiter,
// §3.2): sign(dp) min(|dm|, |dp|, |dm + dp| / 4) when dm and dp have the same strict sign,
// else 0.  The face values are P_i -+ this.  For FP64 the sign test and the three-way minimum
// are taken on the IEEE bit patterns (the order of non-negative doubles is the order of their
// bits) and the quarter by exponent arithmetic, so that only the sum runs on the FP64 pipe; the
// result is the number the floating-point operations give (for |dm + dp| >= 2^-1020).
__device__ __forceinline__ double mc_half_slope(double dm, double dp) {
  const long long bm = __double_as_longlong(dm), bp = __double_as_longlong(dp);
  const long long am = bm & 0x7fffffffffffffffLL, ap = bp & 0x7fffffffffffffffLL;
  // |dm + dp| / 4 by lowering the exponent field by 2: exact for |dm + dp| >= 2^-1020, and
  // taken as 0 below that (no FP64 multiply)
  const long long as = __double_as_longlong(dm + dp) & 0x7fffffffffffffffLL;
  const long long aq = as >= (3LL << 52) ? as - (2LL << 52) : 0LL;
  long long m = am < ap ? am : ap;
  m = m < aq ? m : aq;
  const bool same = ((bm ^ bp) >= 0) && am != 0 && ap != 0;
  const long long r = same ? (m | (bp & (long long)0x8000000000000000ULL)) : 0LL;
  return __longlong_as_double(r);
}

__device__ __forceinline__ float mc_half_slope(float dm, float dp) {
  const float a = fminf(fminf(fabsf(dm), fabsf(dp)), 0.25f * fabsf(dm + dp));
  const float s = dp > 0.f ? a : -a;
  return dm * dp > 0.f ? s : 0.f;
}

// Half MC slope in double-word arithmetic (the same definition as the FP64 and FP32 versions:
// sign(dp) min(|dm|, |dp|, |dm + dp| / 4) for a strict common sign, else 0; the sign of a
// normalised pair is the sign of its leading float, and the quarter is exact).
__device__ __forceinline__ f32x2 mc_half_slope(f32x2 dm, f32x2 dp) {
  const bool same = (dm.hi > 0.0f && dp.hi > 0.0f) || (dm.hi < 0.0f && dp.hi < 0.0f);
  if (!same) return f32x2(0.0f, 0.0f);
  const f32x2 s = dm + dp;
  const f32x2 aq(fabsf(s.hi) * 0.25f, (s.hi < 0.0f ? -s.lo : s.lo) * 0.25f);
  const f32x2 m = fmin(fmin(fabs(dm), fabs(dp)), aq);
  return dp.hi > 0.0f ? m : -m;
}

// PPM (§3.2; the piecewise parabolic method of Colella and Woodward as used by Marti and
// Muller).  Interface value between cells a and b from their values and MC half slopes:
//   e = (qa + qb)/2 - (sigma_b - sigma_a)/6 = (qa + qb)/2 - (hb - ha)/3,
// which is the interface value of the parabola through the neighbouring cells.
template <typename R>
__device__ __forceinline__ R ppm_edge(R qa, R qb, R ha, R hb) {
  return R(0.5) * (qa + qb) - (hb - ha) * (R(1) / R(3));
}

// Monotonicity constraints of one cell's parabola (edge values aL, aR, cell value q): a cell at
// a local extremum becomes flat; an edge that puts the parabola's extremum inside the cell is
// moved to 3q - 2 (other edge), which places the extremum on the opposite edge.
template <typename R>
__device__ __forceinline__ void ppm_limit(R& aL, R q, R& aR) {
  if ((aR - q) * (q - aL) <= R(0)) {
    aL = q;
    aR = q;
    return;
  }
  const R d = aR - aL;
  const R m6 = R(6) * (q - R(0.5) * (aL + aR));
  if (d * m6 > d * d) aL = R(3) * q - R(2) * aR;
  else if (-(d * d) > d * m6) aR = R(3) * q - R(2) * aL;
}

// Left / right states at the face between cells c-1 and c from the cells c-3 .. c+2.
template <typename R>
__device__ __forceinline__ void ppm_face(R q0, R q1, R q2, R q3, R q4, R q5, R& left, R& right) {
  const R h0 = mc_half_slope(q1 - q0, q2 - q1);  // cell c-2
  const R h1 = mc_half_slope(q2 - q1, q3 - q2);  // cell c-1
  const R h2 = mc_half_slope(q3 - q2, q4 - q3);  // cell c
  const R h3 = mc_half_slope(q4 - q3, q5 - q4);  // cell c+1
  const R e0 = ppm_edge(q1, q2, h0, h1);
  R e1 = ppm_edge(q2, q3, h1, h2);
  const R e2 = ppm_edge(q3, q4, h2, h3);
  R aL1 = e0, aR1 = e1;  // cell c-1
  ppm_limit(aL1, q2, aR1);
  R aL2 = e1, aR2 = e2;  // cell c
  ppm_limit(aL2, q3, aR2);
  left = aR1;
  right = aL2;
}

// ------------------------------------------------------------------------------------------
// Recovery of the primitive state from the conserved one (§2.2: Newton-Raphson, §3.2: the 2D
// scheme).  With normal-observer quantities D = rho W, S_i, E, Bn^i, and the unknowns
// z = Z / D = w W^2 / D and v^2 (scaled by D so that every quantity is O(1), which keeps the
// FP32 stage of the iteration in range for any density), the conserved data satisfy
//   r1 = (z + b)^2 v^2 - q (2z + b) / z^2 - s = 0
//   r2 = z - p + b (1 + v^2)/2 - q / (2 z^2) - e = 0,
//   p  = (gamma - 1)/gamma (z (1 - v^2) - sqrt(1 - v^2)),
// with b = Bn^2 / D, s = S^2 / D^2, q = (S.Bn)^2 / D^3, e = E / D and p the pressure over D.
// Newton with the analytic 2x2 Jacobian runs in FP32 from the previous primitive state until
// it settles to FP32 accuracy, then in FP64 to the tolerance; a bracketed 1D solve takes over
// if the FP64 iteration does not settle.
// ------------------------------------------------------------------------------------------
struct C2PResult {
  int ok;
  int iters;
};

// Scaled invariants of one conserved state.
struct C2PScalars {
  double e, s, q, b, g1;
};

template <typename R>
struct NewtonStep {
  R dz, dv;
};

template <typename R>
__device__ __forceinline__ NewtonStep<R> c2p_newton(R z, R v2, R e, R s, R q, R b, R g1) {
  // sqrt(1 - v^2) and 1 / (2 sqrt(1 - v^2)) from one reciprocal square root (v^2 < 1)
  const R om = R(1) - v2;
  const R rs = rsqrt(om);
  const R sq = om * rs;
  const R iz = rcp_fast(z);
  const R iz2 = iz * iz;
  const R zb = z + b;
  const R p = g1 * (z * (R(1) - v2) - sq);
  const R r1 = zb * zb * v2 - q * (R(2) * z + b) * iz2 - s;
  const R r2 = z - p + R(0.5) * b * (R(1) + v2) - R(0.5) * q * iz2 - e;
  const R j11 = R(2) * zb * v2 + R(2) * q * zb * iz2 * iz;
  const R j12 = zb * zb;
  const R j21 = R(1) - g1 * (R(1) - v2) + q * iz2 * iz;
  const R j22 = g1 * (z - R(0.5) * rs) + R(0.5) * b;
  const R idet = fdiv(R(1), j11 * j22 - j12 * j21);
  NewtonStep<R> st;
  st.dz = -(j22 * r1 - j12 * r2) * idet;
  st.dv = -(j11 * r2 - j21 * r1) * idet;
  return st;
}

__device__ __forceinline__ double c2p_v2(const C2PScalars& q, double z) {
  const double zb = z + q.b;
  return (z * z * q.s + q.q * (2.0 * z + q.b)) / (z * z * zb * zb);
}

// Energy residual with v^2 = v^2(z) substituted, and its z derivative.
__device__ __forceinline__ double c2p_f1d(const C2PScalars& q, double z, double* dfdz) {
  const double zb = z + q.b;
  const double N = z * z * q.s + q.q * (2.0 * z + q.b);
  const double Dn = z * z * zb * zb;
  const double v2 = N / Dn;
  const double dv2 = ((2.0 * z * q.s + 2.0 * q.q) * Dn - N * (2.0 * z * zb * (2.0 * z + q.b))) / (Dn * Dn);
  const double sq = sqrt(1.0 - v2);
  const double p = q.g1 * (z * (1.0 - v2) - sq);
  const double iz2 = 1.0 / (z * z);
  *dfdz = 1.0 - q.g1 * (1.0 - v2) - q.g1 * (0.5 / sq - z) * dv2 + 0.5 * q.b * dv2 + q.q * iz2 / z;
  return z - p + 0.5 * q.b * (1.0 + v2) - 0.5 * q.q * iz2 - q.e;
}

// Fallback recovery: Newton on the 1D residual kept inside a bracket [zlo, gamma e] by
// bisection (the 'rtsafe' safeguard of Press et al.).  gamma e bounds z from above because
// E >= Z - p >= Z / gamma; zlo is found by bisection where v^2(z) drops below 1 - 1e-12.
// Returns false when no root is bracketed (an unphysical conserved state).
static __device__ __noinline__ bool c2p_bracketed(const C2PScalars q, double zguess, double& zout,
                                           double& v2out, int& iters) {
  const double v2cap = 1.0 - 1e-12;
  const double zhi = q.e / (1.0 - q.g1);  // gamma e
  if (!(c2p_v2(q, zhi) < v2cap)) return false;
  double zlo = zhi * 1e-100;
  if (!(c2p_v2(q, zlo) < v2cap)) {
    double a = zlo, b = zhi;
    for (int k = 0; k < 400 && b - a > 1e-14 * b; ++k) {
      const double m = 0.5 * (a + b);
      if (c2p_v2(q, m) < v2cap) b = m; else a = m;
    }
    zlo = b;
  }
  double df;
  if (!(c2p_f1d(q, zlo, &df) < 0.0)) return false;
  if (!(c2p_f1d(q, zhi, &df) >= 0.0)) return false;
  double lo = zlo, hi = zhi;
  double z = (zguess > lo && zguess < hi) ? zguess : 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    ++iters;
    const double f = c2p_f1d(q, z, &df);
    if (f == 0.0) break;
    if (f < 0.0) lo = z; else hi = z;
    double zn = z - f / df;
    if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
    const bool conv = fabs(zn - z) <= 1e-15 * z || hi - lo <= 4e-16 * hi;
    z = zn;
    if (conv) break;
  }
  const double v2 = c2p_v2(q, z);
  if (!(v2 < 1.0) || !(z > 0.0)) return false;
  zout = z;
  v2out = v2;
  return true;
}

// sqrt(a) to FP64 accuracy from the FP32 square root of a nearby float af: two steps of Heron's
// iteration s <- s + (a - s^2) / (2 s), with 1 / (2 s) kept at its FP32 value (each step
// multiplies the relative error by about the FP32 root's, 2^-24).  Four FP64 instructions and
// two conversions instead of a correctly rounded FP64 square root.  a > 0, af > 0.
__device__ __forceinline__ double sqrt_from_f32(double a, float af) {
  const float s = fsqrt(af);
  const double sd = (double)s, h = (double)__fdividef(0.5f, s);
  double r = fma(fma(-sd, sd, a), h, sd);
  return fma(fma(-r, r, a), h, r);
}

// Inverse of the recovery's 2x2 Jacobian (the derivatives of r1, r2 of c2p_newton) formed in
// FP32 at an FP32 root (zf, vf).
struct C2PJac32 {
  float a11, a12, a21, a22;  // J^-1
  float iz2;                 // 1 / zf^2
};

__device__ __forceinline__ C2PJac32 c2p_jac32(float zf, float vf, float bf, float qf, float gf) {
  const float omf = 1.0f - vf;
  const float rs = rsqrtf(omf);
  const float iz = __fdividef(1.0f, zf);
  const float iz2 = iz * iz;
  const float zbf = zf + bf;
  const float j11 = 2.0f * zbf * vf + 2.0f * qf * zbf * iz2 * iz;
  const float j12 = zbf * zbf;
  const float j21 = 1.0f - gf * omf + qf * iz2 * iz;
  const float j22 = gf * (zf - 0.5f * rs) + 0.5f * bf;
  const float idet = __fdividef(1.0f, j11 * j22 - j12 * j21);
  C2PJac32 J;
  J.a11 = j22 * idet;
  J.a12 = -j12 * idet;
  J.a21 = -j21 * idet;
  J.a22 = j11 * idet;
  J.iz2 = iz2;
  return J;
}

// One correction of a root (z, v^2) of the recovery equations: the residuals are formed in FP64
// (they are differences of nearly equal O(1) terms, the pressure above all), multiplied through
// by z^2 so that they need no FP64 division,
//   R1 = z^2 ((z + b)^2 v^2 - s) - q (2z + b),   R2 = z^2 (z - p + b (1 + v^2)/2 - e) - q / 2,
// and the step -J^-1 (R1, R2) / z^2 is taken with the FP32 Jacobian J of an FP32 root nearby.
// Each correction multiplies the error by about J's relative error (2^-24): one takes an FP32
// root to the accuracy of a full FP64 Newton step from it, two to FP64 accuracy.  om_seed is
// 1 - v^2 in FP32 (seed of the FP64 square root).  Writes the step (dz, dv).
__device__ __forceinline__ void c2p_correct(const C2PScalars& q, const C2PJac32& J, float om_seed,
                                            double z, double v2, float& dz, float& dv) {
  const double om = 1.0 - v2;
  const double sq = sqrt_from_f32(om, om_seed);
  const double z2 = z * z, zb = z + q.b;
  const double R1 = fma(z2, fma(zb * zb, v2, -q.s), -q.q * fma(2.0, z, q.b));
  const double p = q.g1 * fma(z, om, -sq);
  const double hb = 0.5 * q.b;
  const double R2 = fma(z2, ((z - p) + fma(hb, v2, hb)) - q.e, -0.5 * q.q);
  const float r1 = (float)R1 * J.iz2, r2 = (float)R2 * J.iz2;
  dz = -(J.a11 * r1 + J.a12 * r2);
  dv = -(J.a21 * r1 + J.a22 * r2);
}

// Guarded Newton update: keep z > 0 and 0 <= v^2 < 1.  Returns false when the step had to be
// replaced by halving the distance to the bound z = 0 or v^2 = 1: a run of such steps shrinks
// geometrically without converging, so it may not end the iteration.  A step below v^2 = 0 is
// projected onto it and counts as a plain step (gas at rest has its root there).
template <typename R>
__device__ __forceinline__ bool c2p_apply(R& z, R& v2, NewtonStep<R> st) {
  R zn = z + st.dz;
  R vn = v2 + st.dv;
  bool plain = true;
  if (!(zn > R(0))) {
    zn = R(0.5) * z;
    plain = false;
  }
  if (vn < R(0)) vn = R(0);
  if (!(vn < R(1))) {
    vn = R(0.5) * (v2 + R(1));
    plain = false;
  }
  z = zn;
  v2 = vn;
  return plain;
}

// Recovery at one cell.  G is the FP64 centre geometry; U the FP64 conserved vector; Pg the
// previous primitive state (initial guess).  maxit caps the FP64 iterations; they stop once a
// Newton step is below step_tol (relative in z, absolute in v^2): the iteration converges
// quadratically there, so the error left is about the square of that step.  ONE_FINISH:
// when the FP32 stage has settled, apply a single FP64 Newton correction (quadratic
// convergence takes the 1e-7 FP32 error to ~1e-14, ample when the result is stored in FP32).
//
// one_d: the 1D scheme instead (§3.2 names a 1D and a 2D recovery): Newton in z alone with v^2
// eliminated, from the previous state's z, kept in its bracket by bisection (c2p_bracketed).
//
// TG, TP: element types of the guess and of the result.  float for the mixed path, whose
// primitive state is stored in FP32: the guess is formed in FP32, and of the result only the
// pressure (a difference of nearly equal terms in cold gas) is formed in FP64.
template <bool CLEAN, bool DIAG, bool ONE_FINISH = false, typename TG = double, typename TP = double>
__device__ __forceinline__ C2PResult con2prim(const Geom<double>& G, const double U[9],
                                              const TG Pg[9], const Consts<double>& c,
                                              int maxit, double step_tol, TP P[9], int one_d = 0) {
  const double isg = rcp_fast(G.sqrtg);
  const double Dd = U[U_D] * isg;
  const double Sx = U[U_TX] * isg, Sy = U[U_TY] * isg, Sz = U[U_TZ] * isg;
  const double Bx = U[U_BX] * isg, By = U[U_BY] * isg, Bz = U[U_BZ] * isg;
  double E;
  double Sux, Suy, Suz, Blx, Bly, Blz;
  if constexpr (DIAG) {
    E = -U[U_TT] * isg * G.ialp;
    Sux = G.ixx * Sx;
    Suy = G.iyy * Sy;
    Suz = G.izz * Sz;
    Blx = G.gxx * Bx;
    Bly = G.gyy * By;
    Blz = G.gzz * Bz;
  } else {
    E = (-U[U_TT] + (G.bx * U[U_TX] + G.by * U[U_TY] + G.bz * U[U_TZ])) * isg * G.ialp;
    Sux = G.ixx * Sx + G.ixy * Sy + G.ixz * Sz;
    Suy = G.ixy * Sx + G.iyy * Sy + G.iyz * Sz;
    Suz = G.ixz * Sx + G.iyz * Sy + G.izz * Sz;
    Blx = G.gxx * Bx + G.gxy * By + G.gxz * Bz;
    Bly = G.gxy * Bx + G.gyy * By + G.gyz * Bz;
    Blz = G.gxz * Bx + G.gyz * By + G.gzz * Bz;
  }
  const double S2 = Sux * Sx + Suy * Sy + Suz * Sz;
  const double B2 = Blx * Bx + Bly * By + Blz * Bz;
  const double SB = Sx * Bx + Sy * By + Sz * Bz;
  const double g1 = (c.gamma - 1.0) / c.gamma;

  C2PResult res;
  res.ok = 0;
  res.iters = 0;
  if (!(Dd > 0.0) || !(E > 0.0)) return res;
  const double iD = rcp_fast(Dd);
  C2PScalars q;
  q.e = E * iD;
  q.b = B2 * iD;
  q.s = S2 * iD * iD;
  q.q = SB * SB * iD * iD * iD;
  q.g1 = g1;

  // initial guess from the previous primitive state: z = w W^2 / D, v^2 = uu / (1 + uu)
  double z = 0.0, v2 = 0.0;
  float zg32 = 0.f, vg32 = 0.f;  // ONE_FINISH: the guess stays in FP32
  {
    using T = TG;
    const T vx = Pg[P_UX], vy = Pg[P_UY], vz = Pg[P_UZ];
    T uu;
    if constexpr (DIAG) uu = (T)G.gxx * vx * vx + (T)G.gyy * vy * vy + (T)G.gzz * vz * vz;
    else
      uu = ((T)G.gxx * vx + (T)G.gxy * vy + (T)G.gxz * vz) * vx +
           ((T)G.gxy * vx + (T)G.gyy * vy + (T)G.gyz * vz) * vy +
           ((T)G.gxz * vx + (T)G.gyz * vy + (T)G.gzz * vz) * vz;
    const T wg = Pg[P_RHO] + (T)c.gfac * Pg[P_PRS];
    if constexpr (ONE_FINISH) {
      zg32 = (float)(wg * (T(1) + uu) * (T)iD);
      vg32 = (float)(uu / (T(1) + uu));
      if (!(zg32 > 0.f) || !(zg32 < 1e30f)) zg32 = (float)q.e;
    } else {
      z = (double)(wg * (T(1) + uu) * (T)iD);
      v2 = (double)(uu / (T(1) + uu));
      if (!(z > 0.0) || !(z < 1e30)) z = q.e;
    }
  }
  bool settled = false;
  bool done = false;
  float om_seed = -1.f;  // ONE_FINISH: 1 - v^2 in FP32 after the FP64 correction
  if (one_d) {
    if constexpr (ONE_FINISH) {
      z = (double)zg32;
      v2 = (double)vg32;
    }
    if (!c2p_bracketed(q, z, z, v2, res.iters)) return res;
    done = true;
  }
  // FP32 stage
  if (!done) {
    float zf = ONE_FINISH ? zg32 : (float)z, vf = ONE_FINISH ? vg32 : (float)v2;
    const float ef = (float)q.e, sf = (float)q.s, qf = (float)q.q, bf = (float)q.b, gf = (float)g1;
    for (int it = 0; it < 30; ++it) {
      const NewtonStep<float> st = c2p_newton<float>(zf, vf, ef, sf, qf, bf, gf);
      const bool plain = c2p_apply(zf, vf, st);
      ++res.iters;
      if (plain && fabsf(st.dz) <= 3e-6f * zf && fabsf(st.dv) <= 3e-6f) {
        settled = true;
        break;
      }
    }
    const bool valid = zf > 0.f && vf >= 0.f && vf < 1.f && isfinite(zf);
    if (valid) {
      z = (double)zf;
      v2 = (double)vf;
    } else if constexpr (ONE_FINISH) {
      z = (double)zg32;
      v2 = (double)vg32;
    }
    // FP64 corrections with the FP32 Jacobian (c2p_correct): one for a result stored in FP32
    // (ONE_FINISH), until a step falls below step_tol (at most three) otherwise.  The full FP64
    // Newton iteration below runs only if they do not settle or leave 0 < z, 0 <= v^2 < 1.
    if (valid && settled) {
      const C2PJac32 J = c2p_jac32(zf, vf, bf, qf, gf);
      const float seed = 1.0f - vf;
      const double tol = ONE_FINISH ? 1e-5 : step_tol;
      for (int k = 0; k < (ONE_FINISH ? 1 : 3); ++k) {
        float dz, dv;
        c2p_correct(q, J, seed, z, v2, dz, dv);
        ++res.iters;
        const double zn = z + (double)dz, vn = v2 + (double)dv;
        if (!(zn > 0.0) || !(vn < 1.0) || !(fabsf(dz) <= 1e-5f * zf) || !(fabsf(dv) <= 1e-5f)) break;
        z = zn;
        v2 = vn < 0.0 ? 0.0 : vn;
        if (fabs((double)dz) <= tol * z && fabs((double)dv) <= tol) {
          done = true;
          om_seed = seed - dv;
          break;
        }
      }
    }
  }
  // FP64 stage
  for (int it = 0; !done && it < maxit; ++it) {
    const NewtonStep<double> st = c2p_newton<double>(z, v2, q.e, q.s, q.q, q.b, g1);
    const bool plain = c2p_apply(z, v2, st);
    ++res.iters;
    if (plain && fabs(st.dz) <= step_tol * z && fabs(st.dv) <= step_tol) {
      done = true;
      break;
    }
  }
  if (!done || !(v2 < 1.0) || !(z > 0.0)) {
    if (!c2p_bracketed(q, z, z, v2, res.iters)) return res;
  }
  const double om = 1.0 - v2;
  double rW, W = 0.0;  // 1/W = sqrt(1 - v^2), W
  if constexpr (ONE_FINISH) {
    if (om_seed < 0.f) om_seed = (float)om;  // after the FP64 iteration
    rW = sqrt_from_f32(om, om_seed);
  } else {
    W = rsqrt(om);
    rW = om * W;
  }
  const double Z = z * Dd;
  const double p = g1 * (Z * (1.0 - v2) - Dd * rW);
  if constexpr (sizeof(TP) == sizeof(double)) {
    if constexpr (ONE_FINISH) W = 1.0 / rW;
    const double iZB = rcp_fast(Z + B2);
    const double sbz = SB * rcp_fast(Z);
    P[P_RHO] = Dd * rW;
    P[P_PRS] = p;
    P[P_UX] = W * (Sux + sbz * Bx) * iZB;
    P[P_UY] = W * (Suy + sbz * By) * iZB;
    P[P_UZ] = W * (Suz + sbz * Bz) * iZB;
    P[P_BX] = Bx * G.ialp;
    P[P_BY] = By * G.ialp;
    P[P_BZ] = Bz * G.ialp;
    P[P_PSI] = CLEAN ? U[U_PSI] * isg : 0.0;
  } else {
    // result stored in FP32: everything but p from FP32 copies of the FP64 quantities
    const TP rWf = ONE_FINISH ? fsqrt(om_seed) : store_as<TP>(rW);
    const TP Zf = store_as<TP>(Z), ia = store_as<TP>(G.ialp);
    const TP Bxf = store_as<TP>(Bx), Byf = store_as<TP>(By), Bzf = store_as<TP>(Bz);
    const TP W = fdiv(TP(1), rWf);
    const TP iZB = fdiv(TP(1), Zf + store_as<TP>(B2));
    const TP sbz = fdiv(store_as<TP>(SB), Zf);
    P[P_RHO] = store_as<TP>(Dd) * rWf;
    P[P_PRS] = store_as<TP>(p);
    P[P_UX] = W * (store_as<TP>(Sux) + sbz * Bxf) * iZB;
    P[P_UY] = W * (store_as<TP>(Suy) + sbz * Byf) * iZB;
    P[P_UZ] = W * (store_as<TP>(Suz) + sbz * Bzf) * iZB;
    P[P_BX] = Bxf * ia;
    P[P_BY] = Byf * ia;
    P[P_BZ] = Bzf * ia;
    P[P_PSI] = CLEAN ? store_as<TP>(U[U_PSI] * isg) : TP(0);
  }
  res.ok = 1;
  return res;
}

}  // namespace hzn
