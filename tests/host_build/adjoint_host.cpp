// Host build of the hand-written reverses of hzn_adjoint.cuh (state algebra, conserved vector,
// flux vector, wave speeds; the product's own templates, with the stand-in cuda_runtime.h of
// this folder): vector-Jacobian products (dX/dP)^T v at n pointwise states, for a check against
// finite differences of the forward functions.  Layouts as in physics_host.cpp.
#include "hzn_adjoint.cuh"

using namespace hzn;
using namespace hzn::adj;

namespace {

Consts<double> consts(double gamma, double ch) {
  Consts<double> c;
  c.gamma = gamma;
  c.gfac = gamma / (gamma - 1.0);
  c.ch = ch;
  c.ch2 = ch * ch;
  return c;
}

// what: 0 conserved vector, 1 flux along d, 2 wave speeds along d (v[0], v[1] weight lambda-,
// lambda+)
template <bool CLEAN, bool DIAG, int D>
void vjp_one(const Geom<double>& G, const double* Pin, const Consts<double>& c, int what,
             const double* v, double* out) {
  double P[9];
  for (int f = 0; f < 9; ++f) P[f] = Pin[f];
  if (!CLEAN) P[8] = 0.0;
  const State<double> S = make_state<DIAG>(G, P, c);
  SBar s;
  zero(s);
  if (what == 0) cons_rev<CLEAN>(G, S, v, s);
  else if (what == 1) flux_rev<D, CLEAN, DIAG>(G, S, c, v, s);
  else speeds_rev<D, DIAG>(G, S, c, v[0], v[1], s);
  for (int f = 0; f < 9; ++f) out[f] = 0.0;
  state_rev<DIAG>(G, S, P, c.gfac, s, out);
  if (!CLEAN) out[8] = 0.0;
}

template <bool CLEAN, bool DIAG>
void vjp_t(long n, const Consts<double>& c, int what, int d, const double* met, const double* prim,
           const double* v, double* out) {
  for (long i = 0; i < n; ++i) {
    const Geom<double> G = make_geom<DIAG>(met + 10 * i);
    if (d == 0) vjp_one<CLEAN, DIAG, 0>(G, prim + 9 * i, c, what, v + 9 * i, out + 9 * i);
    else if (d == 1) vjp_one<CLEAN, DIAG, 1>(G, prim + 9 * i, c, what, v + 9 * i, out + 9 * i);
    else vjp_one<CLEAN, DIAG, 2>(G, prim + 9 * i, c, what, v + 9 * i, out + 9 * i);
  }
}

}  // namespace

extern "C" void dev_vjp(long n, double gamma, double ch, int clean, int diag, int what, int d,
                        const double* met, const double* prim, const double* v, double* out) {
  const Consts<double> c = consts(gamma, ch);
  if (clean) {
    if (diag) vjp_t<true, true>(n, c, what, d, met, prim, v, out);
    else vjp_t<true, false>(n, c, what, d, met, prim, v, out);
  } else {
    if (diag) vjp_t<false, true>(n, c, what, d, met, prim, v, out);
    else vjp_t<false, false>(n, c, what, d, met, prim, v, out);
  }
}
