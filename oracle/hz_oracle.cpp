// hz_oracle.cpp -- plain FP64 CPU oracle of the HORIZON GRMHD finite-volume update
// (Zink, "HORIZON: Accelerated General Relativistic Magnetohydrodynamics", arXiv:1102.5202).
//
// TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header, table or
// helper with the CUDA library; both read the same seeded inputs and nothing else.
//
// What it computes (one explicit RK3 step of the conservation system, §2.1 Eq. 2, in the
// compact form of §2.2 Eq. 3):
//   ghost fill -> MC reconstruction of primitives (§2.2, §3.2) -> face metric -> flux and
//   conserved vector of the left and right states -> fast-magnetosonic speeds -> HLLE face
//   flux (§2.2, §3.2) -> flux divergence + metric source (§2.1 Eq. 2, §2.2) -> Runge-Kutta
//   stage (§3.2) -> conservative-to-primitive recovery (§2.2 Newton-Raphson iteration, §3.2).
// Every step runs over the whole grid before the next one starts: no fusion, no tiling.
//
// Readings of points where the paper is silent:
//   * induction flux along i of sqrt(-g) B^j is sqrt(-g)(b^j u^i - b^i u^j), the sign that
//     follows from the dual Maxwell equation with B^i = *F^{it} (§2.1 Eq. 1-2);
//   * RK3 is the Shu-Osher strong-stability-preserving scheme;
//   * the face metric is the mean of the two adjacent centre values, and the metric source
//     uses 1/2 sqrt(-g) T^{kl} d_i g_{kl} with a centred difference of the centre 4-metric;
//   * the recovery result is the unique primitive state whose conserved vector equals the
//     input; the oracle reaches it by a bracketed, bisection-safeguarded Newton iteration in
//     Z = rho h W^2 alone (v^2 eliminated), which is not the 2D scheme the GPU path uses;
//   * divergence cleaning (§3.2): generalised-Lagrange-multiplier field psi with conserved
//     Psi = sqrt(gamma) psi, extra flux sqrt(-g) gamma^{dj} psi on B^j, flux
//     sqrt(gamma)(c_h^2 alpha^2 B^d - beta^d psi) on Psi, source -kappa alpha Psi; the pair
//     (B^d, Psi) uses HLLE bounds at its own characteristic speeds,
//     -beta^d / 2 -+ sqrt((beta^d / 2)^2 + c_h^2 alpha^2 gamma^dd) (-+ c_h alpha sqrt(gamma^dd)
//     without shift);
//   * floors: a cell with D/sqrt(gamma) < rho_atm, a failed recovery, or a recovered
//     rho < rho_floor is set to atmosphere (rho_floor, p_atm, zero velocity, same B and psi);
//     p < p_floor is raised to p_floor; every reset recomputes the conserved vector;
//   * the time step is dt = CFL / max over cells of sum_d max|lambda_d| / dx_d, the Courant
//     condition of an update that treats all axes at once (the same as the per-axis form in
//     1-D).
//
// Every function is written for a scalar type R: double, or std::complex<double> for
// complex-step differentiation (d J / d q = Im J(q + i h) / h, exact to round-off for the
// discrete scheme with its branch decisions frozen).  Decisions (limiter, wave-speed bounds,
// floors) use real parts; |x| is continued analytically; the recovery root found on the real
// part is polished by complex Newton steps, which carries its derivative exactly.
//
// Numerics are compiled with -ffp-contract=off so that x86 and Arm give the same bits.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace hzo {

// Field order of the primitive vector P, of the conserved vector U and of the metric.
enum { RHO = 0, PRS, UTX, UTY, UTZ, BCX, BCY, BCZ, PSI, NPRIM };
enum { CD = 0, CTT, CTX, CTY, CTZ, CBX, CBY, CBZ, CPSI, NCONS };
enum { ALP = 0, BEX, BEY, BEZ, GXX, GXY, GXZ, GYY, GYZ, GZZ, NMET };

using cplx = std::complex<double>;

// Real part used for every decision; |x| continued analytically; min/max by real part.
inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double absv(double x) { return std::fabs(x); }
inline cplx absv(const cplx& x) { return x.real() < 0.0 ? -x : x; }
inline double minv(double a, double b) { return std::min(a, b); }
inline double maxv(double a, double b) { return std::max(a, b); }
inline cplx minv(const cplx& a, const cplx& b) { return b.real() < a.real() ? b : a; }
inline cplx maxv(const cplx& a, const cplx& b) { return a.real() < b.real() ? b : a; }

}  // namespace hzo

extern "C" {

// Uniform Cartesian grid of n[0] x n[1] x n[2] cells; an axis with n = 1 is inactive (no
// flux, no metric derivative).  bc[d] = 0 outflow (zero-gradient), 1 periodic.
typedef struct {
  int n[3];
  int bc[3];
  double dx[3];
} hzo_grid;

typedef struct {
  double gamma;      // ideal-gas adiabatic index, p = (gamma - 1) rho eps
  int cleaning;      // 1: evolve the divergence-cleaning field psi
  double ch;         // cleaning speed (fraction of light speed)
  double kappa;      // cleaning damping rate
  double rho_floor;  // atmosphere density
  double p_floor;    // pressure floor
  double atm_K;      // atmosphere pressure = atm_K rho_floor^gamma if > 0, else p_floor
  int c2p_maxit;     // iteration cap of the recovery
  double rho_atm;    // cells with D / sqrt(gamma) below rho_atm are set to the atmosphere (0: off)
  int recon;         // 0: TVD with the MC limiter; 1: PPM (§3.2)
} hzo_opts;

}  // extern "C"

namespace hzo {

// ----------------------------------------------------------------------------------------
// 3+1 geometry at one point: lapse alpha, shift beta^i, spatial metric gamma_ij (§2.1).
// ----------------------------------------------------------------------------------------
template <class R>
struct Geom {
  R alp, beta[3], g[3][3];
  R ginv[3][3];   // gamma^{ij}
  R sqrtgam;      // sqrt(det gamma_ij)
  R sqrtmg;       // sqrt(-g) = alpha sqrt(gamma)
  R g4[4][4];     // g_{mu nu}
  R g4inv[4][4];  // g^{mu nu}
};

template <class R>
static Geom<R> make_geom(const R m[NMET]) {
  Geom<R> G;
  G.alp = m[ALP];
  G.beta[0] = m[BEX];
  G.beta[1] = m[BEY];
  G.beta[2] = m[BEZ];
  G.g[0][0] = m[GXX];
  G.g[0][1] = G.g[1][0] = m[GXY];
  G.g[0][2] = G.g[2][0] = m[GXZ];
  G.g[1][1] = m[GYY];
  G.g[1][2] = G.g[2][1] = m[GYZ];
  G.g[2][2] = m[GZZ];
  // inverse by cofactors
  R c00 = G.g[1][1] * G.g[2][2] - G.g[1][2] * G.g[2][1];
  R c01 = G.g[1][2] * G.g[2][0] - G.g[1][0] * G.g[2][2];
  R c02 = G.g[1][0] * G.g[2][1] - G.g[1][1] * G.g[2][0];
  R det = G.g[0][0] * c00 + G.g[0][1] * c01 + G.g[0][2] * c02;
  R c11 = G.g[0][0] * G.g[2][2] - G.g[0][2] * G.g[2][0];
  R c12 = G.g[0][2] * G.g[1][0] - G.g[0][0] * G.g[1][2];
  R c22 = G.g[0][0] * G.g[1][1] - G.g[0][1] * G.g[1][0];
  G.ginv[0][0] = c00 / det;
  G.ginv[0][1] = G.ginv[1][0] = c01 / det;
  G.ginv[0][2] = G.ginv[2][0] = c02 / det;
  G.ginv[1][1] = c11 / det;
  G.ginv[1][2] = G.ginv[2][1] = c12 / det;
  G.ginv[2][2] = c22 / det;
  G.sqrtgam = std::sqrt(det);
  G.sqrtmg = G.alp * G.sqrtgam;
  // 4-metric: g_tt = -alpha^2 + beta_k beta^k, g_ti = beta_i, g_ij = gamma_ij
  R blow[3];
  for (int i = 0; i < 3; ++i) {
    blow[i] = 0.0;
    for (int j = 0; j < 3; ++j) blow[i] += G.g[i][j] * G.beta[j];
  }
  R bb = 0.0;
  for (int i = 0; i < 3; ++i) bb += blow[i] * G.beta[i];
  G.g4[0][0] = -G.alp * G.alp + bb;
  for (int i = 0; i < 3; ++i) {
    G.g4[0][i + 1] = G.g4[i + 1][0] = blow[i];
    for (int j = 0; j < 3; ++j) G.g4[i + 1][j + 1] = G.g[i][j];
  }
  // inverse 4-metric: g^tt = -1/alpha^2, g^ti = beta^i/alpha^2, g^ij = gamma^ij - beta^i beta^j/alpha^2
  R ia2 = 1.0 / (G.alp * G.alp);
  G.g4inv[0][0] = -ia2;
  for (int i = 0; i < 3; ++i) {
    G.g4inv[0][i + 1] = G.g4inv[i + 1][0] = G.beta[i] * ia2;
    for (int j = 0; j < 3; ++j) G.g4inv[i + 1][j + 1] = G.ginv[i][j] - G.beta[i] * G.beta[j] * ia2;
  }
  return G;
}

// ----------------------------------------------------------------------------------------
// Fluid + field state of one primitive vector (§2.1): u^mu, b^mu, b^2, enthalpy density.
// Primitive velocity u~^i = W v^i = u^i + W beta^i / alpha (§5.2 footnote); B^i = *F^{it}.
// ----------------------------------------------------------------------------------------
template <class R>
struct State {
  R rho, p, w;  // w = rho h = rho + gamma p / (gamma - 1)
  R W;          // Lorentz factor
  R u[4], ul[4];
  R b[4], bl[4];
  R b2;
  R B[3];
  R psi;
};

template <class R>
static State<R> make_state(const Geom<R>& G, const R P[NPRIM], double gamma) {
  State<R> S;
  S.rho = P[RHO];
  S.p = P[PRS];
  S.w = S.rho + gamma / (gamma - 1.0) * S.p;
  R ut[3] = {P[UTX], P[UTY], P[UTZ]};
  R uu = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) uu += G.g[i][j] * ut[i] * ut[j];
  S.W = std::sqrt(1.0 + uu);
  S.u[0] = S.W / G.alp;
  for (int i = 0; i < 3; ++i) S.u[i + 1] = ut[i] - S.W * G.beta[i] / G.alp;
  for (int m = 0; m < 4; ++m) {
    S.ul[m] = 0.0;
    for (int n = 0; n < 4; ++n) S.ul[m] += G.g4[m][n] * S.u[n];
  }
  for (int i = 0; i < 3; ++i) S.B[i] = P[BCX + i];
  // b^t = B^i u_i ; b^i = (B^i + b^t u^i) / u^t
  S.b[0] = 0.0;
  for (int i = 0; i < 3; ++i) S.b[0] += S.B[i] * S.ul[i + 1];
  for (int i = 0; i < 3; ++i) S.b[i + 1] = (S.B[i] + S.b[0] * S.u[i + 1]) / S.u[0];
  for (int m = 0; m < 4; ++m) {
    S.bl[m] = 0.0;
    for (int n = 0; n < 4; ++n) S.bl[m] += G.g4[m][n] * S.b[n];
  }
  S.b2 = 0.0;
  for (int m = 0; m < 4; ++m) S.b2 += S.b[m] * S.bl[m];
  S.psi = P[PSI];
  return S;
}

// Mixed energy-momentum tensor T^mu_nu = (w + b^2) u^mu u_nu + (p + b^2/2) delta^mu_nu - b^mu b_nu.
template <class R>
static R Tmix(const State<R>& S, int mu, int nu) {
  R t = (S.w + S.b2) * S.u[mu] * S.ul[nu] - S.b[mu] * S.bl[nu];
  if (mu == nu) t += S.p + 0.5 * S.b2;
  return t;
}

// Contravariant T^{mu nu}.
template <class R>
static R Tup(const Geom<R>& G, const State<R>& S, int mu, int nu) {
  return (S.w + S.b2) * S.u[mu] * S.u[nu] + (S.p + 0.5 * S.b2) * G.g4inv[mu][nu] -
         S.b[mu] * S.b[nu];
}

// Conserved vector w(u) (§2.2: algebraic, evaluated per cell): sqrt(-g) J^t, sqrt(-g) T^t_mu,
// sqrt(-g) B^i (§2.1), plus Psi = sqrt(gamma) psi.
template <class R>
static void prim2cons(const Geom<R>& G, const State<R>& S, R U[NCONS]) {
  U[CD] = G.sqrtmg * S.rho * S.u[0];
  for (int nu = 0; nu < 4; ++nu) U[CTT + nu] = G.sqrtmg * Tmix(S, 0, nu);
  for (int i = 0; i < 3; ++i) U[CBX + i] = G.sqrtmg * S.B[i];
  U[CPSI] = G.sqrtgam * S.psi;
}

// Flux vector along axis d (§2.1 Eq. 2): sqrt(-g) J^d, sqrt(-g) T^d_mu,
// sqrt(-g)(b^j u^d - b^d u^j) [+ cleaning terms].
template <class R>
static void flux(const Geom<R>& G, const State<R>& S, int d, const hzo_opts& o, R F[NCONS]) {
  const int dd = d + 1;
  F[CD] = G.sqrtmg * S.rho * S.u[dd];
  for (int nu = 0; nu < 4; ++nu) F[CTT + nu] = G.sqrtmg * Tmix(S, dd, nu);
  for (int j = 0; j < 3; ++j)
    F[CBX + j] = G.sqrtmg * (S.b[j + 1] * S.u[dd] - S.b[dd] * S.u[j + 1]);
  F[CPSI] = 0.0;
  if (o.cleaning) {
    for (int j = 0; j < 3; ++j) F[CBX + j] += G.sqrtmg * G.ginv[d][j] * S.psi;
    F[CPSI] = G.sqrtgam * (o.ch * o.ch * G.alp * G.alp * S.B[d] - G.beta[d] * S.psi);
  }
}

// Fast-magnetosonic characteristic speeds dx^d/dt: roots of
//   (u^d - l u^t)^2 = c^2 [ g^tt l^2 - 2 g^td l + g^dd + (u^d - l u^t)^2 ],
// c^2 = cs^2 + vA^2 - cs^2 vA^2, cs^2 = gamma p / w, vA^2 = b^2 / (w + b^2).
template <class R>
static void speeds(const Geom<R>& G, const State<R>& S, int d, double gamma, R* lm, R* lp) {
  const int dd = d + 1;
  R cs2 = gamma * S.p / S.w;
  R va2 = S.b2 / (S.w + S.b2);
  R c2 = cs2 + va2 - cs2 * va2;
  R A = (1.0 - c2) * S.u[0] * S.u[0] - c2 * G.g4inv[0][0];
  R B = -2.0 * ((1.0 - c2) * S.u[0] * S.u[dd] - c2 * G.g4inv[0][dd]);
  R C = (1.0 - c2) * S.u[dd] * S.u[dd] - c2 * G.g4inv[dd][dd];
  R disc = B * B - 4.0 * A * C;
  if (re(disc) < 0.0) disc = 0.0;
  R sq = std::sqrt(disc);
  *lp = (-B + sq) / (2.0 * A);
  *lm = (-B - sq) / (2.0 * A);
}

// Characteristic speeds of the cleaning pair (B^d, Psi) along d.  In the conserved variables
// (sqrt(-g) B^d, Psi) its fluxes are alpha gamma^dd Psi and c_h^2 alpha sqrt(-g) B^d - beta^d Psi
// (the induction flux of B^d along d vanishes), so the speeds are the roots of
// l^2 + beta^d l - c_h^2 alpha^2 gamma^dd = 0:  l = -beta^d / 2 -+ sqrt((beta^d / 2)^2 + a^2),
// a = c_h alpha sqrt(gamma^dd); with zero shift, -+a.
template <class R>
static void clean_speeds(const Geom<R>& G, int d, double ch, R* lm, R* lp) {
  R a = ch * G.alp * std::sqrt(G.ginv[d][d]);
  R hb = 0.5 * G.beta[d];
  R r = std::sqrt(hb * hb + a * a);
  *lm = -hb - r;
  *lp = -hb + r;
}

// MC-limited slope (TVD reconstruction with the monotonized-central limiter, §3.2).
template <class R>
static R mc_slope(const R& dm, const R& dp) {
  if (re(dm) * re(dp) <= 0.0) return R(0.0);
  R a = minv(minv(2.0 * absv(dm), 2.0 * absv(dp)), 0.5 * absv(dm + dp));
  return re(dp) > 0.0 ? a : -a;
}

// PPM (§3.2, the piecewise parabolic method of Colella and Woodward as used by Marti and Muller):
// the interface value between cells u and u+1 interpolates the parabola through the
// neighbouring cell values, written with the MC-limited slopes sigma,
//   a_{u+1/2} = (q_u + q_{u+1}) / 2 - (sigma_{u+1} - sigma_u) / 6,
// then each cell's pair (aL, aR) is made monotone: a cell at a local extremum becomes flat
// (aL = aR = q); otherwise an edge value that would put the parabola's extremum inside the
// cell is moved to 3 q - 2 (other edge).  No contact steepening, no flattening (the paper
// names the method only).
template <class R>
static R ppm_edge(const R& qa, const R& qb, const R& sa, const R& sb) {
  return 0.5 * (qa + qb) - (sb - sa) / 6.0;
}

template <class R>
static void ppm_monotone(R& aL, const R& q, R& aR) {
  if (re(aR - q) * re(q - aL) <= 0.0) {
    aL = q;
    aR = q;
    return;
  }
  const R d = aR - aL;
  const R m6 = 6.0 * (q - 0.5 * (aL + aR));
  if (re(d) * re(m6) > re(d) * re(d)) aL = 3.0 * q - 2.0 * aR;
  else if (-re(d) * re(d) > re(d) * re(m6)) aR = 3.0 * q - 2.0 * aL;
}

// Left and right states at the face between cells c-1 and c from the six cells c-3 .. c+2
// (q[0] .. q[5]): MC uses q[1] .. q[4], PPM all six.
template <class R>
static void reconstruct(int recon, const R q[6], R* left, R* right) {
  if (recon == 0) {
    R sigL = mc_slope(q[2] - q[1], q[3] - q[2]);  // slope in cell c-1
    R sigR = mc_slope(q[3] - q[2], q[4] - q[3]);  // slope in cell c
    *left = q[2] + 0.5 * sigL;
    *right = q[3] - 0.5 * sigR;
    return;
  }
  R sig[4];  // MC slopes of cells c-2 .. c+1
  for (int u = 0; u < 4; ++u) sig[u] = mc_slope(q[u + 1] - q[u], q[u + 2] - q[u + 1]);
  R e0 = ppm_edge(q[1], q[2], sig[0], sig[1]);  // between c-2 and c-1
  R e1 = ppm_edge(q[2], q[3], sig[1], sig[2]);  // between c-1 and c
  R e2 = ppm_edge(q[3], q[4], sig[2], sig[3]);  // between c and c+1
  R aL1 = e0, aR1 = e1;                         // cell c-1
  ppm_monotone(aL1, q[2], aR1);
  R aL2 = e1, aR2 = e2;                         // cell c
  ppm_monotone(aL2, q[3], aR2);
  *left = aR1;
  *right = aL2;
}

// HLLE flux of one component (§2.2: needs only the two fluxes and the two wave-speed bounds).
template <class R>
static R hlle(const R& sl, const R& sr, const R& FL, const R& FR, const R& UL, const R& UR) {
  if (re(sr - sl) == 0.0) return 0.5 * (FL + FR);
  return (sr * FL - sl * FR + sl * sr * (UR - UL)) / (sr - sl);
}

// ----------------------------------------------------------------------------------------
// Conservative-to-primitive recovery (§2.2: u(w) is not algebraic, solved iteratively).
// Normal-observer quantities: D = rho W, S_i, E = n_mu n_nu T^{mu nu}, B_n^i = alpha B^i.
// With Z = w W^2 and v^2 the conserved data satisfy
//   S^2 = (Z + Bn^2)^2 v^2 - (S.Bn)^2 (2Z + Bn^2) / Z^2
//   E   = Z - p + Bn^2 (1 + v^2)/2 - (S.Bn)^2 / (2 Z^2),
//   p   = (gamma-1)/gamma (Z (1 - v^2) - D sqrt(1 - v^2)).
// The first line gives v^2(Z) in closed form; the second is solved for Z.
// ----------------------------------------------------------------------------------------
template <class R>
struct C2PIn {
  R D, E, S2, SB, B2;
  R Slow[3], Bn[3];
};

template <class R>
static R v2_of_Z(const C2PIn<R>& c, const R& Z) {
  R ZB = Z + c.B2;
  return (Z * Z * c.S2 + c.SB * c.SB * (2.0 * Z + c.B2)) / (Z * Z * ZB * ZB);
}

template <class R>
static R dv2_dZ(const C2PIn<R>& c, const R& Z) {
  R ZB = Z + c.B2;
  R N = Z * Z * c.S2 + c.SB * c.SB * (2.0 * Z + c.B2);
  R Dn = Z * Z * ZB * ZB;
  R dN = 2.0 * Z * c.S2 + 2.0 * c.SB * c.SB;
  R dDn = 2.0 * Z * ZB * (2.0 * Z + c.B2);
  return (dN * Dn - N * dDn) / (Dn * Dn);
}

template <class R>
static R pres_of(const C2PIn<R>& c, const R& Z, const R& v2, double gamma) {
  R sq = std::sqrt(1.0 - v2);
  return (gamma - 1.0) / gamma * (Z * (1.0 - v2) - c.D * sq);
}

template <class R>
static R f_of_Z(const C2PIn<R>& c, const R& Z, double gamma) {
  R v2 = v2_of_Z(c, Z);
  R p = pres_of(c, Z, v2, gamma);
  return Z - p + 0.5 * c.B2 * (1.0 + v2) - 0.5 * c.SB * c.SB / (Z * Z) - c.E;
}

template <class R>
static R df_dZ(const C2PIn<R>& c, const R& Z, double gamma) {
  R v2 = v2_of_Z(c, Z);
  R dv2 = dv2_dZ(c, Z);
  double g1 = (gamma - 1.0) / gamma;
  R sq = std::sqrt(1.0 - v2);
  R dp_dZ = g1 * (1.0 - v2);
  R dp_dv2 = g1 * (-Z + 0.5 * c.D / sq);
  return 1.0 - dp_dZ - dp_dv2 * dv2 + 0.5 * c.B2 * dv2 + c.SB * c.SB / (Z * Z * Z);
}

// Bracketed root of the energy equation for real data.  Returns 0 and the root in *Zout, or 1
// on failure (no bracket, no convergence).
static int solve_Z(const C2PIn<double>& c, double Zg, const hzo_opts& o, double* Zout, int* iters) {
  const double gamma = o.gamma;
  *iters = 0;
  if (!(c.D > 0.0) || !(c.E > 0.0)) return 1;
  // Upper bound: E >= Z - p >= Z / gamma, so Z <= gamma E.
  double Zhi = gamma * c.E;
  const double v2cap = 1.0 - 1e-12;
  if (!(v2_of_Z(c, Zhi) < v2cap)) return 1;
  // Lower bound: v^2(Z) decreases monotonically in Z; bisect for a point with v^2 < v2cap.
  double Zlo = Zhi * 1e-100;
  if (!(v2_of_Z(c, Zlo) < v2cap)) {
    double a = Zlo, b = Zhi;
    for (int k = 0; k < 400 && b - a > 1e-14 * b; ++k) {
      double m = 0.5 * (a + b);
      if (v2_of_Z(c, m) < v2cap) b = m; else a = m;
    }
    Zlo = b;
  }
  double flo = f_of_Z(c, Zlo, gamma);
  double fhi = f_of_Z(c, Zhi, gamma);
  if (!(flo < 0.0)) return 1;
  if (!(fhi >= 0.0)) return 1;
  if (fhi == 0.0) Zlo = Zhi;

  // Bisection-safeguarded Newton (the 'rtsafe' scheme of Press et al., Numerical Recipes).
  double Z = (Zg > Zlo && Zg < Zhi) ? Zg : 0.5 * (Zlo + Zhi);
  double lo = Zlo, hi = Zhi;
  int it;
  int conv = 0;
  for (it = 0; it < o.c2p_maxit; ++it) {
    double f = f_of_Z(c, Z, gamma);
    if (f == 0.0) { conv = 1; break; }
    if (f < 0.0) lo = Z; else hi = Z;
    double fp = df_dZ(c, Z, gamma);
    double Zn = Z - f / fp;
    if (!(Zn > lo && Zn < hi)) Zn = 0.5 * (lo + hi);
    if (std::fabs(Zn - Z) <= 1e-15 * Z || hi - lo <= 4e-16 * hi) { Z = Zn; conv = 1; break; }
    Z = Zn;
  }
  *iters = it + 1;
  if (!conv) return 1;
  *Zout = Z;
  return 0;
}

// Newton polish of the root for complex data (the real part is already the root): the
// imaginary part converges to the implicit-function derivative.  Nothing to do for double.
static void polish_Z(const C2PIn<double>&, double&, double) {}
static void polish_Z(const C2PIn<cplx>& c, cplx& Z, double gamma) {
  for (int k = 0; k < 4; ++k) Z = Z - f_of_Z(c, Z, gamma) / df_dZ(c, Z, gamma);
}

// Returns 0 on success, 1 on failure (no bracket, no convergence, unphysical root).
template <class R>
static int con2prim(const Geom<R>& G, const R U[NCONS], const R Pguess[NPRIM],
                    const hzo_opts& o, R P[NPRIM], int* iters) {
  C2PIn<R> c;
  R isg = 1.0 / G.sqrtgam;
  c.D = U[CD] * isg;
  for (int i = 0; i < 3; ++i) {
    c.Slow[i] = U[CTX + i] * isg;
    c.Bn[i] = U[CBX + i] * isg;
  }
  R bS = 0.0;
  for (int i = 0; i < 3; ++i) bS += G.beta[i] * U[CTX + i];
  c.E = (-U[CTT] + bS) / (G.alp * G.sqrtgam);
  c.S2 = 0.0;
  c.B2 = 0.0;
  c.SB = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      c.S2 += G.ginv[i][j] * c.Slow[i] * c.Slow[j];
      c.B2 += G.g[i][j] * c.Bn[i] * c.Bn[j];
    }
  for (int i = 0; i < 3; ++i) c.SB += c.Slow[i] * c.Bn[i];
  const double gamma = o.gamma;

  // root of the real part, then (complex step only) Newton polish
  C2PIn<double> cr;
  cr.D = re(c.D);
  cr.E = re(c.E);
  cr.S2 = re(c.S2);
  cr.SB = re(c.SB);
  cr.B2 = re(c.B2);
  double Zg = -1.0;
  if (Pguess) {
    State<R> Sg = make_state(G, Pguess, gamma);
    Zg = re(Sg.w * Sg.W * Sg.W);
  }
  double Zr = 0.0;
  if (solve_Z(cr, Zg, o, &Zr, iters)) return 1;
  R Z = Zr;
  polish_Z(c, Z, gamma);

  R v2 = v2_of_Z(c, Z);
  if (!(re(v2) < 1.0) || !(re(Z) > 0.0)) return 1;
  R W = 1.0 / std::sqrt(1.0 - v2);
  R p = pres_of(c, Z, v2, gamma);
  // v^i = (S^i + (S.Bn / Z) Bn^i) / (Z + Bn^2)
  R Sup[3];
  for (int i = 0; i < 3; ++i) {
    Sup[i] = 0.0;
    for (int j = 0; j < 3; ++j) Sup[i] += G.ginv[i][j] * c.Slow[j];
  }
  P[RHO] = c.D / W;
  P[PRS] = p;
  for (int i = 0; i < 3; ++i) {
    R vi = (Sup[i] + c.SB / Z * c.Bn[i]) / (Z + c.B2);
    P[UTX + i] = W * vi;
    P[BCX + i] = c.Bn[i] / G.alp;
  }
  P[PSI] = U[CPSI] * isg;
  return 0;
}

// Recovery plus atmosphere / floor treatment; may rewrite U.  Returns 1 if the cell was reset.
template <class R>
static int recover_cell(const Geom<R>& G, R U[NCONS], const R Pguess[NPRIM], const hzo_opts& o,
                        R P[NPRIM], int* iters) {
  // atmosphere: a cell whose rest-mass density D / sqrt(gamma) = rho W is below rho_atm is
  // not recovered but set to the atmosphere state (the decision uses the conserved state only)
  const bool atm = o.rho_atm > 0.0 && re(U[CD] / G.sqrtgam) < o.rho_atm;
  int fail = 0;
  *iters = 0;
  if (!atm) fail = con2prim(G, U, Pguess, o, P, iters);
  int reset = 0;
  if (atm || fail || re(P[RHO]) < o.rho_floor) {
    R Bkeep[3] = {U[CBX] / G.sqrtmg, U[CBY] / G.sqrtmg, U[CBZ] / G.sqrtmg};
    P[RHO] = o.rho_floor;
    double patm = o.atm_K > 0.0 ? o.atm_K * std::pow(o.rho_floor, o.gamma) : o.p_floor;
    if (patm < o.p_floor) patm = o.p_floor;
    P[PRS] = patm;
    P[UTX] = P[UTY] = P[UTZ] = 0.0;
    for (int i = 0; i < 3; ++i) P[BCX + i] = Bkeep[i];
    P[PSI] = U[CPSI] / G.sqrtgam;
    reset = 1;
  } else if (re(P[PRS]) < o.p_floor) {
    P[PRS] = o.p_floor;
    reset = 1;
  }
  if (reset) {
    State<R> S = make_state(G, P, o.gamma);
    prim2cons(G, S, U);
  }
  return fail;
}

// ----------------------------------------------------------------------------------------
// Grid storage.  Grid functions are plain arrays, x fastest, one array per field.
// Primitive arrays are copied into a ghost-padded work array (width NG = 3 on active axes);
// the metric comes with one ghost layer on active axes.
// ----------------------------------------------------------------------------------------
constexpr int NG = 3;

struct Mesh {
  hzo_grid g;
  int act[3];
  int gp[3];   // ghost width of the padded primitive array per axis
  int np[3];   // padded primitive dims
  int gm[3];   // ghost width of the metric per axis
  int nm[3];   // metric dims
  long ncell;
  explicit Mesh(const hzo_grid& gr) : g(gr) {
    ncell = 1;
    for (int d = 0; d < 3; ++d) {
      act[d] = g.n[d] > 1;
      gp[d] = act[d] ? NG : 0;
      np[d] = g.n[d] + 2 * gp[d];
      gm[d] = act[d] ? 1 : 0;
      nm[d] = g.n[d] + 2 * gm[d];
      ncell *= g.n[d];
    }
  }
  long cell(int i, int j, int k) const { return i + (long)g.n[0] * (j + (long)g.n[1] * k); }
  long pcell(int i, int j, int k) const {  // i,j,k interior-relative, may be negative
    return (i + gp[0]) + (long)np[0] * ((j + gp[1]) + (long)np[1] * (k + gp[2]));
  }
  long mcell(int i, int j, int k) const {
    return (i + gm[0]) + (long)nm[0] * ((j + gm[1]) + (long)nm[1] * (k + gm[2]));
  }
  long npad() const { return (long)np[0] * np[1] * np[2]; }
  long nmet() const { return (long)nm[0] * nm[1] * nm[2]; }
};

template <class R>
static void load_metric(const Mesh& M, const double* met, long mc, R m[NMET]) {
  const long nmt = M.nmet();
  for (int f = 0; f < NMET; ++f) m[f] = met[f * nmt + mc];
}

// Ghost fill (outflow = copy of the nearest interior cell; periodic = wrap), axis by axis.
template <class R>
static void fill_ghosts(const Mesh& M, const R* prim, std::vector<R>& Pp) {
  const long npd = M.npad();
  Pp.assign((size_t)npd * NPRIM, R(0.0));
  const int* n = M.g.n;
  for (int k = -M.gp[2]; k < n[2] + M.gp[2]; ++k)
    for (int j = -M.gp[1]; j < n[1] + M.gp[1]; ++j)
      for (int i = -M.gp[0]; i < n[0] + M.gp[0]; ++i) {
        int s[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          if (s[d] < 0 || s[d] >= n[d]) {
            if (M.g.bc[d] == 1) s[d] = ((s[d] % n[d]) + n[d]) % n[d];
            else s[d] = s[d] < 0 ? 0 : n[d] - 1;
          }
        }
        long src = M.cell(s[0], s[1], s[2]);
        long dst = M.pcell(i, j, k);
        for (int f = 0; f < NPRIM; ++f) Pp[(size_t)f * npd + dst] = prim[(size_t)f * M.ncell + src];
      }
}

// Metric source S_mu = sqrt(-g) T^k_l Gamma^l_{mu k} = 1/2 sqrt(-g) T^{kl} d_mu g_{kl} of the
// momentum equations (§2.1 Eq. 2), with d_i g_{kl} the centred difference (g(i+1) - g(i-1)) /
// (2 dx_i) of the centre 4-metric; static metric: S_t = 0; mass and induction have no source.
// Cleaning damping -kappa alpha Psi.  Added to L[f * ncell + cell].
template <class R>
static void add_sources(const Mesh& M, const hzo_opts& o, const double* met, const R* prim,
                        std::vector<R>& L) {
  const int* n = M.g.n;
  const long nc = M.ncell;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    int i = (int)(c % n[0]);
    int j = (int)((c / n[0]) % n[1]);
    int k = (int)(c / ((long)n[0] * n[1]));
    R m0[NMET];
    load_metric(M, met, M.mcell(i, j, k), m0);
    Geom<R> G = make_geom(m0);
    R P[NPRIM];
    for (int f = 0; f < NPRIM; ++f) P[f] = prim[(size_t)f * nc + c];
    State<R> S = make_state(G, P, o.gamma);
    for (int d = 0; d < 3; ++d) {
      if (!M.act[d]) continue;
      int e[3] = {0, 0, 0};
      e[d] = 1;
      R mp[NMET], mm[NMET];
      load_metric(M, met, M.mcell(i + e[0], j + e[1], k + e[2]), mp);
      load_metric(M, met, M.mcell(i - e[0], j - e[1], k - e[2]), mm);
      Geom<R> Gp = make_geom(mp), Gm = make_geom(mm);
      R src = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          R dg = (Gp.g4[a][b] - Gm.g4[a][b]) / (2.0 * M.g.dx[d]);
          src += Tup(G, S, a, b) * dg;
        }
      L[(size_t)(CTX + d) * nc + c] += 0.5 * G.sqrtmg * src;
    }
    if (o.cleaning) {
      R Psi = G.sqrtgam * S.psi;
      L[(size_t)CPSI * nc + c] += -o.kappa * G.alp * Psi;
    }
  }
}

// Spatial operator L(U) = - sum_d (F_{d,i+1/2} - F_{d,i-1/2}) / dx_d + S (§2.2), from the
// primitive state.  The result is stored in L[f * ncell + cell].
template <class R>
static void rhs(const Mesh& M, const hzo_opts& o, const double* met, const R* prim,
                std::vector<R>& L) {
  const int* n = M.g.n;
  const long nc = M.ncell;
  L.assign((size_t)nc * NCONS, R(0.0));
  std::vector<R> Pp;
  fill_ghosts(M, prim, Pp);
  const long npd = M.npad();

  for (int d = 0; d < 3; ++d) {
    if (!M.act[d]) continue;
    int e[3] = {0, 0, 0};
    e[d] = 1;
    int nf[3] = {n[0], n[1], n[2]};
    nf[d] += 1;  // faces i - 1/2 for i = 0 .. n_d
    long nfaces = (long)nf[0] * nf[1] * nf[2];
    std::vector<R> Ff((size_t)nfaces * NCONS);
#pragma omp parallel for schedule(static)
    for (long fidx = 0; fidx < nfaces; ++fidx) {
      int i = (int)(fidx % nf[0]);
      int j = (int)((fidx / nf[0]) % nf[1]);
      int k = (int)(fidx / ((long)nf[0] * nf[1]));
      // face between cell c-1 and c along d, c = (i,j,k)
      R PL[NPRIM], PR[NPRIM];
      for (int f = 0; f < NPRIM; ++f) {
        auto at = [&](int s) {
          return Pp[(size_t)f * npd + M.pcell(i + s * e[0], j + s * e[1], k + s * e[2])];
        };
        R q[6] = {at(-3), at(-2), at(-1), at(0), at(1), at(2)};
        reconstruct(o.recon, q, &PL[f], &PR[f]);
      }
      R mA[NMET], mB[NMET], mf[NMET];
      load_metric(M, met, M.mcell(i - e[0], j - e[1], k - e[2]), mA);
      load_metric(M, met, M.mcell(i, j, k), mB);
      for (int f = 0; f < NMET; ++f) mf[f] = 0.5 * (mA[f] + mB[f]);
      Geom<R> G = make_geom(mf);
      State<R> SL = make_state(G, PL, o.gamma), SR = make_state(G, PR, o.gamma);
      R FL[NCONS], FR[NCONS], UL[NCONS], UR[NCONS];
      flux(G, SL, d, o, FL);
      flux(G, SR, d, o, FR);
      prim2cons(G, SL, UL);
      prim2cons(G, SR, UR);
      R lmL, lpL, lmR, lpR;
      speeds(G, SL, d, o.gamma, &lmL, &lpL);
      speeds(G, SR, d, o.gamma, &lmR, &lpR);
      R sl = minv(R(0.0), minv(lmL, lmR));
      R sr = maxv(R(0.0), maxv(lpL, lpR));
      R* out = &Ff[(size_t)fidx * NCONS];
      for (int q = 0; q < NCONS; ++q) out[q] = hlle(sl, sr, FL[q], FR[q], UL[q], UR[q]);
      if (o.cleaning) {
        R cm, cp;
        clean_speeds(G, d, o.ch, &cm, &cp);
        R csl = minv(R(0.0), cm), csr = maxv(R(0.0), cp);
        out[CBX + d] = hlle(csl, csr, FL[CBX + d], FR[CBX + d], UL[CBX + d], UR[CBX + d]);
        out[CPSI] = hlle(csl, csr, FL[CPSI], FR[CPSI], UL[CPSI], UR[CPSI]);
      }
    }
    // flux divergence
    const double idx = 1.0 / M.g.dx[d];
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; ++c) {
      int i = (int)(c % n[0]);
      int j = (int)((c / n[0]) % n[1]);
      int k = (int)(c / ((long)n[0] * n[1]));
      long fm = i + (long)nf[0] * (j + (long)nf[1] * k);
      long fp = (i + e[0]) + (long)nf[0] * ((j + e[1]) + (long)nf[1] * (k + e[2]));
      for (int q = 0; q < NCONS; ++q)
        L[(size_t)q * nc + c] -= (Ff[(size_t)fp * NCONS + q] - Ff[(size_t)fm * NCONS + q]) * idx;
    }
  }

  add_sources(M, o, met, prim, L);
}

// Conserved state of the grid from its primitive state.
template <class R>
static void grid_prim2cons(const Mesh& M, const hzo_opts& o, const double* met, const R* prim, R* cons) {
  const long nc = M.ncell;
  const int* n = M.g.n;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    int i = (int)(c % n[0]);
    int j = (int)((c / n[0]) % n[1]);
    int k = (int)(c / ((long)n[0] * n[1]));
    R m[NMET], P[NPRIM], U[NCONS];
    load_metric(M, met, M.mcell(i, j, k), m);
    for (int f = 0; f < NPRIM; ++f) P[f] = prim[(size_t)f * nc + c];
    Geom<R> G = make_geom(m);
    State<R> S = make_state(G, P, o.gamma);
    prim2cons(G, S, U);
    for (int f = 0; f < NCONS; ++f) cons[(size_t)f * nc + c] = U[f];
  }
}

// One Shu-Osher RK3 step of size dt (§3.2) on (prim, cons); returns the recovery failures.
template <class R>
static long step(const Mesh& M, const hzo_opts& o, const double* met, R* prim, R* cons, double dt) {
  const long nc = M.ncell;
  const int* n = M.g.n;
  const size_t N = (size_t)nc * NCONS;
  std::vector<R> U0(cons, cons + N), U1(N), L;
  std::vector<R> P(prim, prim + (size_t)nc * NPRIM);
  long fails = 0;
  for (int stage = 0; stage < 3; ++stage) {
    rhs(M, o, met, P.data(), L);
    // U^(1) = U0 + dt L(U0);  U^(2) = 3/4 U0 + 1/4 (U1 + dt L(U1));  U^(3) = 1/3 U0 + 2/3 (U2 + dt L(U2))
    for (size_t q = 0; q < N; ++q) {
      if (stage == 0) U1[q] = U0[q] + dt * L[q];
      else if (stage == 1) U1[q] = 0.75 * U0[q] + 0.25 * (U1[q] + dt * L[q]);
      else U1[q] = (1.0 / 3.0) * U0[q] + (2.0 / 3.0) * (U1[q] + dt * L[q]);
    }
    long sf = 0;
#pragma omp parallel for schedule(static) reduction(+ : sf)
    for (long c = 0; c < nc; ++c) {
      int i = (int)(c % n[0]);
      int j = (int)((c / n[0]) % n[1]);
      int k = (int)(c / ((long)n[0] * n[1]));
      R m[NMET], U[NCONS], Pg[NPRIM], Pn[NPRIM];
      load_metric(M, met, M.mcell(i, j, k), m);
      Geom<R> G = make_geom(m);
      for (int f = 0; f < NCONS; ++f) U[f] = U1[(size_t)f * nc + c];
      for (int f = 0; f < NPRIM; ++f) Pg[f] = P[(size_t)f * nc + c];
      int it;
      sf += recover_cell(G, U, Pg, o, Pn, &it);
      for (int f = 0; f < NCONS; ++f) U1[(size_t)f * nc + c] = U[f];
      for (int f = 0; f < NPRIM; ++f) P[(size_t)f * nc + c] = Pn[f];
    }
    fails += sf;
  }
  std::copy(P.begin(), P.end(), prim);
  std::copy(U1.begin(), U1.end(), cons);
  return fails;
}

}  // namespace hzo

using namespace hzo;

extern "C" {

// Conserved vector of n pointwise states.  met: n x 10, prim: n x 9, cons: n x 9 (row-major).
void hzo_prim2cons(long n, const hzo_opts* o, const double* met, const double* prim, double* cons) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    prim2cons(G, S, cons + c * NCONS);
  }
}

// Recovery of n pointwise states; guess may be null.  Returns the number of failures;
// status[c] = 0 ok / 1 failed (no atmosphere reset here), iters[c] = iterations used.
long hzo_cons2prim(long n, const hzo_opts* o, const double* met, const double* cons,
                   const double* guess, double* prim, int* status, int* iters) {
  long nf = 0;
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    int it = 0;
    int s = con2prim(G, cons + c * NCONS, guess ? guess + c * NPRIM : nullptr, *o,
                     prim + c * NPRIM, &it);
    if (status) status[c] = s;
    if (iters) iters[c] = it;
    nf += s;
  }
  return nf;
}

// Recovery with the atmosphere and floor rules of the step, pointwise.  cons is
// rewritten when a cell is reset; status[c] = 1 when the energy-based recovery failed.
long hzo_recover(long n, const hzo_opts* o, const double* met, double* cons, const double* guess,
                 double* prim, int* status) {
  long nf = 0;
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    int it = 0;
    const int s = recover_cell(G, cons + c * NCONS, guess ? guess + c * NPRIM : nullptr, *o,
                               prim + c * NPRIM, &it);
    if (status) status[c] = s;
    nf += s;
  }
  return nf;
}

// Pointwise flux along d, and characteristic speeds (lam: n x 2 = [minus, plus]).
void hzo_flux(long n, const hzo_opts* o, int d, const double* met, const double* prim, double* F) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    flux(G, S, d, *o, F + c * NCONS);
  }
}

void hzo_speeds(long n, const hzo_opts* o, int d, const double* met, const double* prim, double* lam) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    speeds(G, S, d, o->gamma, lam + 2 * c, lam + 2 * c + 1);
  }
}

// Pointwise 4-vectors and invariants for tests: out n x 14 = u^mu(4), b^mu(4), b^2, W,
// sqrt(gamma), alpha, T^t_t, w.
void hzo_state(long n, const hzo_opts* o, const double* met, const double* prim, double* out) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    double* r = out + c * 14;
    for (int m = 0; m < 4; ++m) { r[m] = S.u[m]; r[4 + m] = S.b[m]; }
    r[8] = S.b2; r[9] = S.W; r[10] = G.sqrtgam; r[11] = G.alp; r[12] = Tmix(S, 0, 0); r[13] = S.w;
  }
}

// Pointwise metric source given the centre metric, the centred derivatives of the 4-metric
// dg (n x 3 x 16, d_i g_{ab} row-major) and the primitive state: src n x 4 (S_t, S_x, S_y, S_z).
void hzo_source_pointwise(long n, const hzo_opts* o, const double* met, const double* dg,
                          const double* prim, double* src) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    src[c * 4 + 0] = 0.0;
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) s += Tup(G, S, a, b) * dg[c * 48 + d * 16 + a * 4 + b];
      src[c * 4 + 1 + d] = 0.5 * G.sqrtmg * s;
    }
  }
}

// Pointwise T^{mu nu} (n x 16) and g^{mu nu} (n x 16) for the Christoffel-form check.
void hzo_tensors(long n, const hzo_opts* o, const double* met, const double* prim, double* Tuu,
                 double* g4, double* g4inv) {
  for (long c = 0; c < n; ++c) {
    Geom<double> G = make_geom(met + c * NMET);
    State<double> S = make_state(G, prim + c * NPRIM, o->gamma);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        Tuu[c * 16 + a * 4 + b] = Tup(G, S, a, b);
        g4[c * 16 + a * 4 + b] = G.g4[a][b];
        g4inv[c * 16 + a * 4 + b] = G.g4inv[a][b];
      }
  }
}

// Grid conserved vector from grid primitives (field-major arrays, metric with ghosts).
void hzo_grid_prim2cons(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim,
                        double* cons) {
  Mesh M(*g);
  grid_prim2cons(M, *o, met, prim, cons);
}

// Spatial operator L on the grid (field-major), for tests.
void hzo_rhs(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim, double* L) {
  Mesh M(*g);
  std::vector<double> Lv;
  rhs(M, *o, met, prim, Lv);
  std::memcpy(L, Lv.data(), sizeof(double) * Lv.size());
}

// The metric source and cleaning damping of the grid alone (the part of hzo_rhs that is not a
// flux difference), field-major; zero for the fields without a source.  For tests.
void hzo_rhs_source(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim,
                    double* S) {
  Mesh M(*g);
  std::vector<double> Sv((size_t)M.ncell * NCONS, 0.0);
  add_sources(M, *o, met, prim, Sv);
  std::memcpy(S, Sv.data(), sizeof(double) * Sv.size());
}

// The CFL rate: max over cells of the sum over active axes of max(|l+|, |l-|) / dx_d (with the
// cleaning speed when on), so that dt = CFL / rate.  The RK3 stages update all axes at once
// (§3.2), so a grid-scale mode along a diagonal sees the sum of the axes' Courant numbers; with
// the per-axis maximum instead, CFL 0.5 in 3-D puts that mode at -3 on the real axis, outside
// RK3's stability interval [-2.51, 0].  In 1-D both definitions coincide.
double hzo_max_speed(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim) {
  Mesh M(*g);
  const long nc = M.ncell;
  double vmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : vmax)
  for (long c = 0; c < nc; ++c) {
    int i = (int)(c % g->n[0]);
    int j = (int)((c / g->n[0]) % g->n[1]);
    int k = (int)(c / ((long)g->n[0] * g->n[1]));
    double m[NMET], P[NPRIM];
    load_metric(M, met, M.mcell(i, j, k), m);
    for (int f = 0; f < NPRIM; ++f) P[f] = prim[(size_t)f * nc + c];
    Geom<double> G = make_geom(m);
    State<double> S = make_state(G, P, o->gamma);
    double rate = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!M.act[d]) continue;
      double lm, lp;
      speeds(G, S, d, o->gamma, &lm, &lp);
      double v = std::max(std::fabs(lm), std::fabs(lp));
      if (o->cleaning) {
        double cm, cp;
        clean_speeds(G, d, o->ch, &cm, &cp);
        v = std::max(v, std::max(std::fabs(cm), std::fabs(cp)));
      }
      rate += v / g->dx[d];
    }
    if (rate > vmax) vmax = rate;
  }
  return vmax;
}

// One Shu-Osher RK3 step of size dt (§3.2).  prim and cons (field-major, n_cell each) hold
// the state on entry and exit; cons must equal w(prim) on entry.  Returns the number of
// recovery failures (cells reset to atmosphere) over the three stages.
long hzo_step(const hzo_grid* g, const hzo_opts* o, const double* met, double* prim, double* cons,
              double dt) {
  Mesh M(*g);
  return step(M, *o, met, prim, cons, dt);
}

// Evolve to t_end with dt = cfl / max_speed (the last step clipped to t_end), or with the
// fixed step fixed_dt when fixed_dt > 0.  Stops after max_steps.  *t_out gets the time
// reached, *fails_out the recovery failures.  Returns the number of steps taken.
long hzo_evolve(const hzo_grid* g, const hzo_opts* o, const double* met, double* prim, double* cons,
                double t_end, double cfl, double fixed_dt, long max_steps, double* t_out,
                long* fails_out) {
  double t = 0.0;
  long steps = 0, fails = 0;
  while (t < t_end && steps < max_steps) {
    double dt = fixed_dt > 0.0 ? fixed_dt : cfl / hzo_max_speed(g, o, met, prim);
    if (t + dt > t_end) dt = t_end - t;
    fails += hzo_step(g, o, met, prim, cons, dt);
    t += dt;
    ++steps;
  }
  if (t_out) *t_out = t;
  if (fails_out) *fails_out = fails;
  return steps;
}

// Complex-step run: nsteps fixed-size steps from the complex primitive state
// prim_re + i prim_im (field-major, n_cell each); the final primitive state is written to
// out_re + i out_im and, when cons_re / cons_im are not null, the final conserved state
// there.  Returns the recovery failures.
long hzo_evolve_cs(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim_re,
                   const double* prim_im, double dt, long nsteps, double* out_re, double* out_im,
                   double* cons_re, double* cons_im) {
  Mesh M(*g);
  const size_t N = (size_t)M.ncell * NPRIM;
  std::vector<cplx> P(N), U(N);
  for (size_t q = 0; q < N; ++q) P[q] = cplx(prim_re[q], prim_im[q]);
  grid_prim2cons(M, *o, met, P.data(), U.data());
  long fails = 0;
  for (long s = 0; s < nsteps; ++s) fails += step(M, *o, met, P.data(), U.data(), dt);
  for (size_t q = 0; q < N; ++q) {
    out_re[q] = P[q].real();
    out_im[q] = P[q].imag();
    if (cons_re) cons_re[q] = U[q].real();
    if (cons_im) cons_im[q] = U[q].imag();
  }
  return fails;
}

// Left / right face states of a 1-D array q[0 .. n-1] (n >= 6) at the faces between cells c-1 and
// c for c = 3 .. n-3 (the faces whose six-cell stencil lies inside the array): left[c], right[c];
// the other entries are left untouched.  recon: 0 MC, 1 PPM.
void hzo_reconstruct_1d(int recon, long n, const double* q, double* left, double* right) {
  for (long c = 3; c + 2 < n; ++c) reconstruct(recon, q + c - 3, &left[c], &right[c]);
}

int hzo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Threads of the grid operations from now on (n >= 1); no effect without OpenMP.
void hzo_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

}  // extern "C"
