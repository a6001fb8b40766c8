// Host build of the pointwise device physics of hzn_physics.cuh in FP64 for a general 3+1
// metric (the product's own templates, with the stand-in cuda_runtime.h of this folder), so
// that the CPU tests can compare them with the oracle's pointwise functions.  Layouts are the
// oracle's: met n x 10 (alpha, beta^i, gamma_xx, _xy, _xz, _yy, _yz, _zz), prim and cons n x 9,
// row-major.
#include "hzn_physics.cuh"

using namespace hzn;

namespace {

Consts<double> consts(double gamma, double ch) {
  Consts<double> c;
  c.gamma = gamma;
  c.gfac = gamma / (gamma - 1.0);
  c.ch = ch;
  c.ch2 = ch * ch;
  return c;
}

template <int D, bool CLEAN, bool DIAG>
void flux_at(const Geom<double>& G, const State<double>& S, const Consts<double>& c, double* F) {
  flux_of<D, CLEAN, DIAG>(G, S, c, F);
}

template <int D, bool DIAG>
void speeds_at(const Geom<double>& G, const State<double>& S, const Consts<double>& c, double* lam,
               double* lam_q) {
  double lm, lp;
  speeds_of<D, DIAG>(G, S, cms2_of(S, c), lm, lp);
  lam[0] = lm;
  lam[1] = lp;
  // the FP64 path's form: w(w + b^2) times the quadratic, halved linear coefficient
  double A, b, sq;
  speed_quadratic<D, DIAG>(G, S, c, A, b, sq);
  lam_q[0] = (-b - sq) / A;
  lam_q[1] = (-b + sq) / A;
}

template <bool DIAG>
void prim2cons_t(long n, double gamma, int clean, const double* met, const double* prim, double* cons) {
  const Consts<double> c = consts(gamma, 0.0);
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    double P[9];
    for (int f = 0; f < 9; ++f) P[f] = prim[9 * i + f];
    if (!clean) P[8] = 0.0;
    const State<double> S = make_state<DIAG>(G, P, c);
    if (clean) cons_of<true>(G, S, cons + 9 * i);
    else {
      cons_of<false>(G, S, cons + 9 * i);
      cons[9 * i + 8] = 0.0;
    }
  }
}

template <bool DIAG>
void flux_t(long n, double gamma, double ch, int clean, int d, const double* met, const double* prim,
            double* F) {
  const Consts<double> c = consts(gamma, ch);
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    double P[9];
    for (int f = 0; f < 9; ++f) P[f] = prim[9 * i + f];
    if (!clean) P[8] = 0.0;
    const State<double> S = make_state<DIAG>(G, P, c);
    double* o = F + 9 * i;
    o[8] = 0.0;
    if (clean) {
      if (d == 0) flux_at<0, true, DIAG>(G, S, c, o);
      else if (d == 1) flux_at<1, true, DIAG>(G, S, c, o);
      else flux_at<2, true, DIAG>(G, S, c, o);
    } else {
      if (d == 0) flux_at<0, false, DIAG>(G, S, c, o);
      else if (d == 1) flux_at<1, false, DIAG>(G, S, c, o);
      else flux_at<2, false, DIAG>(G, S, c, o);
    }
  }
}

template <bool DIAG>
void speeds_t(long n, double gamma, int d, const double* met, const double* prim, double* lam,
              double* lam_q) {
  const Consts<double> c = consts(gamma, 0.0);
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    const State<double> S = make_state<DIAG>(G, prim + 9 * i, c);
    if (d == 0) speeds_at<0, DIAG>(G, S, c, lam + 2 * i, lam_q + 2 * i);
    else if (d == 1) speeds_at<1, DIAG>(G, S, c, lam + 2 * i, lam_q + 2 * i);
    else speeds_at<2, DIAG>(G, S, c, lam + 2 * i, lam_q + 2 * i);
  }
}

template <bool DIAG>
void con2prim_t(long n, double gamma, int clean, const double* met, const double* cons,
                const double* guess, double tol, int maxit, double* prim, int* status) {
  const Consts<double> c = consts(gamma, 0.0);
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    double P[9];
    C2PResult r;
    if (clean) r = con2prim<true, DIAG>(G, cons + 9 * i, guess + 9 * i, c, maxit, 0.01 * std::sqrt(tol), P);
    else r = con2prim<false, DIAG>(G, cons + 9 * i, guess + 9 * i, c, maxit, 0.01 * std::sqrt(tol), P);
    for (int f = 0; f < 9; ++f) prim[9 * i + f] = P[f];
    status[i] = r.ok ? 0 : 1;
  }
}

}  // namespace

// diag = 1: the specialisation for zero shift and diagonal gamma (the metric must be such).
extern "C" {

void dev_prim2cons(long n, double gamma, int clean, int diag, const double* met, const double* prim,
                   double* cons) {
  if (diag) prim2cons_t<true>(n, gamma, clean, met, prim, cons);
  else prim2cons_t<false>(n, gamma, clean, met, prim, cons);
}

void dev_flux(long n, double gamma, double ch, int clean, int diag, int d, const double* met,
              const double* prim, double* F) {
  if (diag) flux_t<true>(n, gamma, ch, clean, d, met, prim, F);
  else flux_t<false>(n, gamma, ch, clean, d, met, prim, F);
}

void dev_speeds(long n, double gamma, int diag, int d, const double* met, const double* prim,
                double* lam, double* lam_q) {
  if (diag) speeds_t<true>(n, gamma, d, met, prim, lam, lam_q);
  else speeds_t<false>(n, gamma, d, met, prim, lam, lam_q);
}

// Recovery (the 2D Newton with its FP32 start and bracketed fallback) from the conserved
// vector and a guess; status[i] = 1 when it failed.
void dev_con2prim(long n, double gamma, int clean, int diag, const double* met, const double* cons,
                  const double* guess, double tol, int maxit, double* prim, int* status) {
  if (diag) con2prim_t<true>(n, gamma, clean, met, cons, guess, tol, maxit, prim, status);
  else con2prim_t<false>(n, gamma, clean, met, cons, guess, tol, maxit, prim, status);
}

}  // extern "C"

// Metric source S_i = 1/2 sqrt(-g) T^{ab} d_i g_ab from the kernels' algebra (tup_of, tdg) for
// given derivatives dg (n x 3 x 16, d_i g_ab row-major 4 x 4), as the oracle's
// source_pointwise: the derivative enters as the difference of two neighbours g(+) = dg / 2,
// g(-) = -dg / 2.  src n x 4 (S_t = 0, S_x, S_y, S_z).
static G4<double> g4_of(const double* m, double f) {
  G4<double> g;
  g.gtt = f * m[0];
  g.blx = f * m[1];
  g.bly = f * m[2];
  g.blz = f * m[3];
  g.gxx = f * m[5];
  g.gxy = f * m[6];
  g.gxz = f * m[7];
  g.gyy = f * m[10];
  g.gyz = f * m[11];
  g.gzz = f * m[15];
  return g;
}

template <bool DIAG>
static void source_t(long n, double gamma, const double* met, const double* dg, const double* prim,
                     double* src) {
  const Consts<double> c = consts(gamma, 0.0);
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    const State<double> S = make_state<DIAG>(G, prim + 9 * i, c);
    const Tup<double> T = tup_of<DIAG>(G, S);
    src[4 * i] = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double* m = dg + 48 * i + 16 * d;
      src[4 * i + 1 + d] = 0.5 * G.sqrtmg * tdg<DIAG>(T, g4_of(m, 0.5), g4_of(m, -0.5));
    }
  }
}

extern "C" void dev_source(long n, double gamma, int diag, const double* met, const double* dg,
                           const double* prim, double* src) {
  if (diag) source_t<true>(n, gamma, met, dg, prim, src);
  else source_t<false>(n, gamma, met, dg, prim, src);
}

extern "C" {

// Face states of a 1-D array at the faces between cells c-1 and c, c = 3 .. n-3 (as the
// oracle's reconstruct_1d): recon 0 MC (FP64), 1 PPM (FP64), 2 MC in double-word arithmetic
// (split inputs, result widened).
void dev_reconstruct(int recon, long n, const double* q, double* left, double* right) {
  for (long c = 3; c + 2 < n; ++c) {
    const double* v = q + c - 3;
    if (recon == 1) {
      ppm_face<double>(v[0], v[1], v[2], v[3], v[4], v[5], left[c], right[c]);
    } else if (recon == 0) {
      left[c] = v[2] + mc_half_slope(v[2] - v[1], v[3] - v[2]);
      right[c] = v[3] - mc_half_slope(v[3] - v[2], v[4] - v[3]);
    } else {
      const f32x2 a = dw::split(v[1]), b = dw::split(v[2]), cc = dw::split(v[3]), d = dw::split(v[4]);
      const f32x2 l = b + mc_half_slope(b - a, cc - b), r = cc - mc_half_slope(cc - b, d - cc);
      left[c] = (double)l.hi + (double)l.lo;
      right[c] = (double)r.hi + (double)r.lo;
    }
  }
}

}  // extern "C"
