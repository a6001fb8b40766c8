// Host build of the substep's spatial operator L(P) = - sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d
// + S (§2.2) over a small grid: every face flux from the product's face_flux (FP64, MC or PPM)
// and face_flux_dw (double-word faces) templates, and for a DIAG metric the geometry tables with
// the product's make_geom / geo_store / g4_at, as the table kernel fills them.  The divergence,
// the metric source and the cleaning damping are formed here in the order the substep kernel
// uses.  Arrays in the oracle's layouts: met (10, nz+2gz, ny+2gy, nx+2gx), prim and out
// (9, nz, ny, nx); inside, odd pitches and field strides with NaN padding, so that a read outside
// the stencil or a wrong stride shows in the result.  Also the recovery with the atmosphere and
// floor rules (recover) and the CFL rate (cell_max_speed) of the same header.
#include <cmath>
#include <limits>
#include <vector>

#include "hzn_kernels.cuh"

using namespace hzn;

namespace {

struct Host {
  KParams kp;
  std::vector<double> P, M, gc, gf, gs;
  std::vector<float> Pf, Mf;  // FP32 storage of the mixed path
};

void setup(Host& h, const int n[3], const double dx[3], const int bc[3], double gamma, int clean,
           double ch, double kappa, const double* met, const double* prim) {
  const double nan = std::numeric_limits<double>::quiet_NaN();
  KParams& kp = h.kp;
  kp = KParams{};
  kp.nx = n[0];
  kp.ny = n[1];
  kp.nz = n[2];
  kp.bcx = bc[0];
  kp.bcy = bc[1];
  kp.bcz = bc[2];
  kp.gx = n[0] > 1;
  kp.gy = n[1] > 1;
  kp.gz = n[2] > 1;
  kp.pitch = n[0] + 3;
  kp.plane = (long long)kp.pitch * n[1];
  kp.fs = kp.plane * n[2] + 5;
  const int mx = n[0] + 2 * kp.gx, my = n[1] + 2 * kp.gy, mz = n[2] + 2 * kp.gz;
  kp.mpitch = mx + 1;
  kp.mny = my;
  kp.mplane = (long long)kp.mpitch * my;
  kp.ms = kp.mplane * mz + 7;
  kp.idx = 1.0 / dx[0];
  kp.idy = 1.0 / dx[1];
  kp.idz = 1.0 / dx[2];
  kp.gamma = gamma;
  kp.gfac = gamma / (gamma - 1.0);
  kp.ch = clean ? ch : 0.0;
  kp.kappa = clean ? kappa : 0.0;
  set_float_consts(kp);

  h.P.assign((size_t)(9 * kp.fs), nan);
  for (int f = 0; f < 9; ++f)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i)
          h.P[f * kp.fs + k * kp.plane + (long long)j * kp.pitch + i] =
              (f == 8 && !clean) ? 0.0 : prim[(((long long)f * n[2] + k) * n[1] + j) * n[0] + i];
  h.M.assign((size_t)(10 * kp.ms), nan);
  for (int f = 0; f < 10; ++f)
    for (int k = 0; k < mz; ++k)
      for (int j = 0; j < my; ++j)
        for (int i = 0; i < mx; ++i)
          h.M[f * kp.ms + k * kp.mplane + (long long)j * kp.mpitch + i] =
              met[(((long long)f * mz + k) * my + j) * mx + i];

  // geometry tables of a DIAG metric over the table kernel's index range
  h.gc.assign((size_t)(GEO_C * kp.ms), nan);
  h.gf.assign((size_t)(3 * GEO_F * kp.ms), nan);
  h.gs.assign((size_t)(3 * GEO_S * kp.ms), nan);
  const double* M = h.M.data();
  for (int k = 0; k < kp.nz + kp.gz; ++k)
    for (int j = 0; j < kp.ny + kp.gy; ++j)
      for (int i = 0; i < kp.nx + 1; ++i) {
        const long long mo = met_off(kp, i, j, k);
        const bool cell = i < kp.nx && j < kp.ny && k < kp.nz;
        if (cell) {
          double m[10];
          load_metric<true>(kp, M, mo, m);
          const Geom<double> Gc = make_geom<true>(m);
          geo_store(h.gc.data(), mo, kp.ms, Gc);
          // sum over active axes of alpha sqrt(gamma^dd) / dx_d, as the table kernel forms it
          double r = Gc.alp * std::sqrt(Gc.ixx) * kp.idx;
          if (kp.gy) r += Gc.alp * std::sqrt(Gc.iyy) * kp.idy;
          if (kp.gz) r += Gc.alp * std::sqrt(Gc.izz) * kp.idz;
          h.gc[GEO_N * kp.ms + mo] = r;
        }
        for (int d = 0; d < 3; ++d) {
          if ((d == 1 && !kp.gy) || (d == 2 && !kp.gz)) continue;
          const bool fin = (d == 0 ? i <= kp.nx : i < kp.nx) && (d == 1 ? j <= kp.ny : j < kp.ny) &&
                           (d == 2 ? k <= kp.nz : k < kp.nz);
          const long long st = d == 0 ? 1 : (d == 1 ? kp.mpitch : kp.mplane);
          if (fin) {
            double m0[10], m1[10], m[10];
            load_metric<true>(kp, M, mo - st, m0);
            load_metric<true>(kp, M, mo, m1);
            for (int f = 0; f < 10; ++f) m[f] = 0.5 * (m0[f] + m1[f]);
            const Geom<double> Gf = make_geom<true>(m);
            geo_store(h.gf.data() + d * GEO_F * kp.ms, mo, kp.ms, Gf);
            h.gf[(d * GEO_F + GEO_N) * kp.ms + mo] = Gf.alp * std::sqrt(d == 0 ? Gf.ixx : (d == 1 ? Gf.iyy : Gf.izz));
          }
          if (cell) {
            const G4<double> gp = g4_at<true, double>(kp, M, mo + st), gm = g4_at<true, double>(kp, M, mo - st);
            double* g = h.gs.data() + d * GEO_S * kp.ms + mo;
            g[0] = gp.gtt - gm.gtt;
            g[kp.ms] = gp.gxx - gm.gxx;
            g[2 * kp.ms] = gp.gyy - gm.gyy;
            g[3 * kp.ms] = gp.gzz - gm.gzz;
          }
        }
      }
  kp.geo_c = h.gc.data();
  kp.geo_f = h.gf.data();
  kp.geo_s = h.gs.data();
  h.Pf.assign(h.P.begin(), h.P.end());
  h.Mf.assign(h.M.begin(), h.M.end());
}

}  // namespace

namespace {

// Face fluxes of one axis, faces i - 1/2 of cells i = 0 .. n_d along d (NV fields each).
template <bool CLEAN, bool DIAG, int RECON, bool PAIR, bool MIXED, typename S>
void faces_of(const KParams& kp, const S* P, const S* M, int d,
              std::vector<typename FaceType<PAIR, MIXED>::R>& F, int nf[3]) {
  using R = typename FaceType<PAIR, MIXED>::R;
  constexpr int NV = CLEAN ? 9 : 8;
  nf[0] = kp.nx + (d == 0);
  nf[1] = kp.ny + (d == 1);
  nf[2] = kp.nz + (d == 2);
  F.assign((size_t)nf[0] * nf[1] * nf[2] * NV, R(0));
  for (int k = 0; k < nf[2]; ++k)
    for (int j = 0; j < nf[1]; ++j)
      for (int i = 0; i < nf[0]; ++i) {
        R o[9];
        for (int f = 0; f < 9; ++f) o[f] = R(0);
        if constexpr (PAIR) {
          face_flux_dw<CLEAN, DIAG>(kp, P, M, d, i, j, k, o, 1);
        } else {
          if (d == 0) face_flux<0, CLEAN, DIAG, RECON>(kp, P, M, i, j, k, o, 1);
          else if (d == 1) face_flux<1, CLEAN, DIAG, RECON>(kp, P, M, i, j, k, o, 1);
          else face_flux<2, CLEAN, DIAG, RECON>(kp, P, M, i, j, k, o, 1);
        }
        R* dst = F.data() + (((size_t)k * nf[1] + j) * nf[0] + i) * NV;
        for (int f = 0; f < NV; ++f) dst[f] = o[f];
      }
}

template <bool CLEAN, bool DIAG, int RECON, bool PAIR, bool MIXED = false>
void rhs_t(const Host& h, double* out) {
  using R = typename FaceType<PAIR, MIXED>::R;
  using S = typename Prec<MIXED>::S;
  constexpr int NV = CLEAN ? 9 : 8;
  const KParams& kp = h.kp;
  const S* P;
  const S* M;
  if constexpr (MIXED) {
    P = h.Pf.data();
    M = h.Mf.data();
  } else {
    P = h.P.data();
    M = h.M.data();
  }
  const bool act[3] = {true, kp.gy != 0, kp.gz != 0};
  std::vector<R> F[3];
  int nf[3][3] = {};
  for (int d = 0; d < 3; ++d)
    if (act[d]) faces_of<CLEAN, DIAG, RECON, PAIR, MIXED>(kp, P, M, d, F[d], nf[d]);
  const Consts<R> c = consts_of<R>(kp);
  const R rid[3] = {cvt<R>(kp.idx), cvt<R>(kp.idy), cvt<R>(kp.idz)};
  const R rhd[3] = {cvt<R>(0.5 * kp.idx), cvt<R>(0.5 * kp.idy), cvt<R>(0.5 * kp.idz)};
  const R rkappa = cvt<R>(kp.kappa);
  const long long mstep[3] = {1, kp.mpitch, kp.mplane};
  for (int k = 0; k < kp.nz; ++k)
    for (int j = 0; j < kp.ny; ++j)
      for (int i = 0; i < kp.nx; ++i) {
        const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
        const long long mo = met_off(kp, i, j, k);
        R L[9];
        for (int f = 0; f < 9; ++f) L[f] = R(0);
        for (int f = 0; f < NV; ++f) {
          R v = R(0);
          for (int d = 0; d < 3; ++d) {
            if (!act[d]) continue;
            const int* n = nf[d];
            const size_t lo = (((size_t)k * n[1] + j) * n[0] + i) * NV;
            const size_t hi = (((size_t)(k + (d == 2)) * n[1] + (j + (d == 1))) * n[0] + (i + (d == 0))) * NV;
            if (d == 0) v = -(F[d][hi + f] - F[d][lo + f]) * rid[d];
            else v -= (F[d][hi + f] - F[d][lo + f]) * rid[d];
          }
          L[f] = v;
        }
        Geom<R> G;
        if constexpr (DIAG && !MIXED) {
          G = geo_load<R>(kp.geo_c, mo, kp.ms);
        } else {
          R mc[10];
          load_metric<DIAG>(kp, M, mo, mc);
          G = make_geom<DIAG>(mc);
        }
        R Pc[9];
        for (int f = 0; f < NV; ++f) Pc[f] = ldc<R>(P + f * kp.fs + off);
        if (!CLEAN) Pc[8] = R(0);
        const State<R> St = make_state<DIAG>(G, Pc, c);
        const Tup<R> T = tup_of<DIAG>(G, St);
        const R hh = R(0.5) * G.sqrtmg;
        for (int d = 0; d < 3; ++d) {
          if (!act[d]) continue;
          if constexpr (DIAG && !MIXED) {
            const double* g = kp.geo_s + d * GEO_S * kp.ms + mo;
            const R s = T.tt * ldc<R>(g) + T.xx * ldc<R>(g + kp.ms) + T.yy * ldc<R>(g + 2 * kp.ms) +
                        T.zz * ldc<R>(g + 3 * kp.ms);
            L[U_TX + d] += hh * s * rhd[d];
          } else {
            const G4<R> gp = g4_at<DIAG, R>(kp, M, mo + mstep[d]), gm = g4_at<DIAG, R>(kp, M, mo - mstep[d]);
            L[U_TX + d] += hh * tdg<DIAG>(T, gp, gm) * rhd[d];
          }
        }
        if (CLEAN) L[U_PSI] += -rkappa * G.alp * (G.sqrtg * St.psi);
        const long long cell = ((long long)k * kp.ny + j) * kp.nx + i;
        const long long ncell = (long long)kp.nx * kp.ny * kp.nz;
        for (int f = 0; f < 9; ++f) out[f * ncell + cell] = f < NV ? to_dbl(L[f]) : 0.0;
      }
}

}  // namespace

// pair = 1: double-word faces, fluxes, divergence and source (MC only); pair = 2: the mixed
// path's FP32 storage and arithmetic (MC or PPM); else FP64; recon 0 MC, 1 PPM.  diag = 1: the DIAG instantiation with its tables (the metric must have zero
// shift and diagonal gamma).  Returns 0, or 1 for an unsupported combination.
extern "C" int dev_rhs(const int* n, const double* dx, const int* bc, double gamma, int clean, double ch,
                       double kappa, int diag, int recon, int pair, const double* met, const double* prim,
                       double* out) {
  Host h;
  setup(h, n, dx, bc, gamma, clean, ch, kappa, met, prim);
#define HZ_RHS(C, D, RC, PR) \
  if (clean == C && diag == D && recon == RC && pair == PR) { rhs_t<C, D, RC, PR>(h, out); return 0; }
  HZ_RHS(0, 0, 0, 0) HZ_RHS(0, 1, 0, 0) HZ_RHS(1, 0, 0, 0) HZ_RHS(1, 1, 0, 0)
  HZ_RHS(0, 0, 1, 0) HZ_RHS(0, 1, 1, 0) HZ_RHS(1, 0, 1, 0) HZ_RHS(1, 1, 1, 0)
  HZ_RHS(0, 0, 0, 1) HZ_RHS(0, 1, 0, 1) HZ_RHS(1, 0, 0, 1) HZ_RHS(1, 1, 0, 1)
#undef HZ_RHS
#define HZ_RHS_MIXED(C, D, RC) \
  if (clean == C && diag == D && recon == RC && pair == 2) { rhs_t<C, D, RC, false, true>(h, out); return 0; }
  HZ_RHS_MIXED(0, 0, 0) HZ_RHS_MIXED(0, 1, 0) HZ_RHS_MIXED(1, 0, 0) HZ_RHS_MIXED(1, 1, 0)
  HZ_RHS_MIXED(0, 0, 1) HZ_RHS_MIXED(0, 1, 1) HZ_RHS_MIXED(1, 0, 1) HZ_RHS_MIXED(1, 1, 1)
#undef HZ_RHS_MIXED
  return 1;
}

// Recovery of n pointwise states with the kernels' atmosphere and floor rules (recover in
// hzn_kernels.cuh): met n x 10, cons n x 9 (rewritten where a cell is reset), guess and prim
// n x 9; status[i] = 1 where the root solve failed.  p_atm: the atmosphere pressure; one_d: the
// one-dimensional Newton scheme (in z, v^2 eliminated) instead of the two-dimensional one.
extern "C" void dev_recover(long n, double gamma, int clean, int diag, double rho_floor, double p_floor,
                            double p_atm, double rho_atm, int maxit, double tol, int one_d, const double* met,
                            double* cons, const double* guess, double* prim, int* status) {
  KParams kp = KParams{};
  kp.c2p_1d = one_d;
  kp.gamma = gamma;
  kp.gfac = gamma / (gamma - 1.0);
  kp.rho_floor = rho_floor;
  kp.p_floor = p_floor;
  kp.p_atm = p_atm;
  kp.rho_atm = rho_atm;
  kp.c2p_maxit = maxit;
  kp.c2p_tol = tol;
  kp.c2p_step_tol = 0.01 * std::sqrt(tol);
  set_float_consts(kp);
  const Consts<double> c = consts_of<double>(kp);
  for (long q = 0; q < n; ++q) {
    double* U = cons + 9 * q;
    double Pg[9], P[9];
    for (int f = 0; f < 9; ++f) Pg[f] = guess[9 * q + f];
    if (!clean) {
      Pg[8] = 0.0;
      U[8] = 0.0;
    }
    int it = 0;
    if (diag) {
      const Geom<double> G = make_geom<true>(met + 10 * q);
      status[q] = clean ? recover<true, true>(kp, G, U, Pg, c, P, it) : recover<false, true>(kp, G, U, Pg, c, P, it);
    } else {
      const Geom<double> G = make_geom<false>(met + 10 * q);
      status[q] = clean ? recover<true, false>(kp, G, U, Pg, c, P, it) : recover<false, false>(kp, G, U, Pg, c, P, it);
    }
    for (int f = 0; f < 9; ++f) prim[9 * q + f] = P[f];
  }
}

namespace {

template <bool YA, bool ZA, bool CLEAN, bool DIAG>
double max_speed_t(const Host& h) {
  const KParams& kp = h.kp;
  const Consts<double> c = consts_of<double>(kp);
  double v = 0.0;
  for (int k = 0; k < kp.nz; ++k)
    for (int j = 0; j < kp.ny; ++j)
      for (int i = 0; i < kp.nx; ++i) {
        const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
        Geom<double> G;
        if constexpr (DIAG) {
          G = geo_load<double>(kp.geo_c, met_off(kp, i, j, k), kp.ms);
        } else {
          double m[10];
          load_metric<DIAG>(kp, h.M.data(), met_off(kp, i, j, k), m);
          G = make_geom<DIAG>(m);
        }
        double P[9];
        for (int f = 0; f < 9; ++f) P[f] = h.P[f * kp.fs + off];
        if (!CLEAN) P[8] = 0.0;
        v = std::fmax(v, cell_max_speed<YA, ZA, CLEAN, DIAG>(kp, G, P, c));
      }
  return v;
}

}  // namespace

// The CFL rate of the grid, max over cells of the sum over active axes of max |lambda| / dx (with the
// cleaning speed when on), from the kernels' cell_max_speed; layouts as dev_rhs.
extern "C" double dev_max_speed(const int* n, const double* dx, const int* bc, double gamma, int clean,
                                double ch, int diag, const double* met, const double* prim) {
  Host h;
  setup(h, n, dx, bc, gamma, clean, ch, 0.0, met, prim);
  const bool ya = n[1] > 1, za = n[2] > 1;
#define HZ_MS(Y, Z, C, D) \
  if (ya == Y && za == Z && clean == C && diag == D) return max_speed_t<Y, Z, C, D>(h);
  HZ_MS(false, false, 0, 0) HZ_MS(false, false, 0, 1) HZ_MS(false, false, 1, 0) HZ_MS(false, false, 1, 1)
  HZ_MS(true, false, 0, 0) HZ_MS(true, false, 0, 1) HZ_MS(true, false, 1, 0) HZ_MS(true, false, 1, 1)
  HZ_MS(true, true, 0, 0) HZ_MS(true, true, 0, 1) HZ_MS(true, true, 1, 0) HZ_MS(true, true, 1, 1)
#undef HZ_MS
  return -1.0;
}

// The CFL rate of a grid whose cells are all at rest on a zero-shift diagonal metric, from the
// closed form the kernels use for such cells (rest_cfl_rate); layouts as dev_rhs.
extern "C" double dev_rest_max_speed(const int* n, const double* dx, const int* bc, double gamma,
                                     int clean, double ch, const double* met, const double* prim) {
  Host h;
  setup(h, n, dx, bc, gamma, clean, ch, 0.0, met, prim);
  const KParams& kp = h.kp;
  double v = 0.0;
  for (int k = 0; k < kp.nz; ++k)
    for (int j = 0; j < kp.ny; ++j)
      for (int i = 0; i < kp.nx; ++i) {
        const long long off = (long long)k * kp.plane + (long long)j * kp.pitch + i;
        const long long mo = met_off(kp, i, j, k);
        double m[10];
        load_metric<true>(kp, h.M.data(), mo, m);
        const Geom<double> G = make_geom<true>(m);
        double P[9];
        for (int f = 0; f < 9; ++f) P[f] = h.P[f * kp.fs + off];
        if (P[P_UX] != 0.0 || P[P_UY] != 0.0 || P[P_UZ] != 0.0) return -1.0;
        const double b2 = G.alp * G.alp * (G.gxx * P[P_BX] * P[P_BX] + G.gyy * P[P_BY] * P[P_BY] +
                                           G.gzz * P[P_BZ] * P[P_BZ]);
        const double r = clean ? rest_cfl_rate<true>(kp, P[P_RHO], P[P_PRS], b2, h.gc[GEO_N * kp.ms + mo])
                               : rest_cfl_rate<false>(kp, P[P_RHO], P[P_PRS], b2, h.gc[GEO_N * kp.ms + mo]);
        v = std::fmax(v, r);
      }
  return v;
}
