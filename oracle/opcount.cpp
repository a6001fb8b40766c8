// Op-counting instantiation of the oracle -- TEST AND MEASUREMENT INFRASTRUCTURE, NOT PRODUCT
// CODE.  The oracle's own templates (hz_oracle.cpp, included below, arithmetic unchanged) run
// one Shu-Osher RK3 step (§3.2) with a scalar type that counts its floating-point operations:
// additions / subtractions, multiplications, divisions and square roots, each one flop.
//
// Conventions of the count:
//   * an operation with an exact structural zero operand is not counted (a literal 0, or a
//     metric component that is zero, e.g. the shift and the off-diagonal gamma_ij of a diagonal
//     spacetime): x * 0 = 0 and x + 0 = x need no arithmetic.  Zeros of the evolved state
//     (a velocity component that happens to vanish) are counted like any other value;
//   * operations whose operands depend on the metric and on constants only (face averages,
//     inverse metric, sqrt(gamma), differences of g for the sources) go to the "geometry"
//     bucket: for a static spacetime they need computing once, not per step;
//   * everything else is attributed to the phase of the step it belongs to (reconstruction,
//     face states, fluxes and conserved vectors, wave speeds, HLLE, divergence, sources, RK
//     update, recovery, CFL maximum);
//   * the state read by each stage (P, U, U0) is data: values the recovery or the atmosphere
//     reset assigned (a zero velocity, the floor density) are counted like computed ones;
//   * the recovery's root solve runs in plain double inside the oracle (the complex-step path
//     needs a real root); its cost is added per call as the bracket set-up (two v^2(Z) and two
//     f(Z) evaluations) plus, per iteration, f(Z), f'(Z), the Newton update and the stopping
//     test, with the iteration count the oracle's solve reports.  Bisection fallbacks are
//     not counted (they do not occur on the workloads measured).
// The step is driven here face by face and cell by cell in the oracle's order, calling the
// oracle's functions; the count of its right-hand side is checked against the oracle's own
// rhs() run with the same scalar (equal counts, equal values).  Faces and cells are counted in
// parallel (OpenMP; each thread keeps its own graph and merges its counts).
#include <omp.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace hzo {

enum { OP_ADD, OP_MUL, OP_DIV, OP_SQRT, NOP };  // tallied kinds (a subtraction is an addition)
enum {
  PH_GEOMETRY,
  PH_RECON,
  PH_FACE_STATE,
  PH_FLUX,
  PH_SPEEDS,
  PH_HLLE,
  PH_DIVERGENCE,
  PH_SOURCES,
  PH_UPDATE,
  PH_C2P,
  PH_CFL,
  NPH
};
enum : unsigned char { N_ADD, N_SUB, N_MUL, N_DIV, N_SQRT, N_NEG, N_LEAF, N_CONST };

// Per thread: the phase being counted and the counts since the thread's last merge.
static thread_local int g_phase = PH_GEOMETRY;
static thread_local long long g_raw[NPH][NOP];    // every operation executed
static thread_local long long g_tally[NPH][NOP];  // distinct operations the unit's results need
static bool g_dag = true;  // record the expression graph (false: raw count only); set serially
static long long s_raw[NPH][NOP], s_tally[NPH][NOP];  // merged counts of all threads

// Expression graph of the current unit (one face, or one cell of one phase).
struct Node {
  long long a, b;
  unsigned char kind, phase;
  bool data, live;
};
static std::atomic<long long> g_next_gen{1};
static std::atomic<long long> g_serial{0};  // identity of values loaded from memory
static thread_local std::vector<Node> g_nodes;
static thread_local std::vector<int> g_roots;
static thread_local long long g_gen = g_next_gen.fetch_add(1);  // generation of the current unit
static size_t g_max_unit = 0;  // largest unit seen (nodes)

// open-addressing table of the unit's nodes by (kind, a, b) for common subexpressions
static const int HCAP = 1 << 14;  // above twice the largest unit (about 4,000 nodes)
static thread_local long long h_a[HCAP], h_b[HCAP];
static thread_local unsigned char h_kind[HCAP];
static thread_local int h_val[HCAP], h_stamp[HCAP];
static thread_local int h_cur = 1;

static int intern(unsigned char kind, long long a, long long b, bool data) {
  uint64_t h = (uint64_t)kind * 0x9E3779B97F4A7C15ull ^ (uint64_t)a * 0xC2B2AE3D27D4EB4Full ^
               (uint64_t)b * 0x165667B19E3779F9ull;
  h ^= h >> 29;
  for (uint64_t k = h & (HCAP - 1);; k = (k + 1) & (HCAP - 1)) {
    if (h_stamp[k] != h_cur) {
      h_stamp[k] = h_cur;
      h_kind[k] = kind;
      h_a[k] = a;
      h_b[k] = b;
      h_val[k] = (int)g_nodes.size();
      g_nodes.push_back(Node{a, b, kind, (unsigned char)g_phase, data, false});
      return h_val[k];
    }
    if (h_kind[k] == kind && h_a[k] == a && h_b[k] == b) return h_val[k];
  }
}

// z: structural zero (operations with it are free); data: depends on the evolved state.
// gen / id: node of generation gen; gen -1 a constant, -2 a value loaded from memory (id its
// identity).  A node of an earlier unit enters the current one as a leaf.
struct Counted {
  double v;
  bool z, data;
  long long gen;
  long long id;
  Counted() : v(0.0), z(true), data(false), gen(-1), id(0) {}
  Counted(double x) : v(x), z(x == 0.0), data(false), gen(-1), id(0) {}
};

inline Counted counted_data(double x) {
  Counted r;
  r.v = x;
  r.z = false;
  r.data = true;
  r.gen = -2;
  r.id = ++g_serial;  // atomic
  return r;
}

inline long long node_of(const Counted& x) {
  if (x.gen == g_gen) return x.id;
  if (x.gen == -1) {
    long long bits;
    std::memcpy(&bits, &x.v, sizeof(bits));
    return intern(N_CONST, bits, 0, false);
  }
  return intern(N_LEAF, x.id, x.gen, x.data);
}

inline int tally_kind(unsigned char kind) {
  return kind == N_MUL ? OP_MUL : (kind == N_DIV ? OP_DIV : (kind == N_SQRT ? OP_SQRT : OP_ADD));
}

inline Counted counted_op(unsigned char kind, const Counted& a, const Counted* b, double v) {
  const bool data = a.data || (b && b->data);
  if (kind != N_NEG) ++g_raw[data ? g_phase : PH_GEOMETRY][tally_kind(kind)];
  Counted r;
  r.v = v;
  r.z = false;
  r.data = data;
  r.gen = g_gen;
  r.id = 0;
  if (g_dag) {
    long long ia = node_of(a), ib = b ? node_of(*b) : -1;
    if ((kind == N_ADD || kind == N_MUL) && ia > ib) std::swap(ia, ib);
    r.id = intern(kind, ia, ib, data);
  } else {
    r.gen = -3;
  }
  return r;
}

// a value the unit's results or decisions depend on
inline void use(const Counted& x) {
  if (g_dag && x.gen == g_gen) g_roots.push_back((int)x.id);
}

// Close the unit: count the distinct operations reachable from its roots.
static void flush() {
  if (!g_dag) return;
  std::vector<int> stack(g_roots.begin(), g_roots.end());
  while (!stack.empty()) {
    const int k = stack.back();
    stack.pop_back();
    Node& n = g_nodes[k];
    if (n.live) continue;
    n.live = true;
    if (n.kind <= N_NEG) {
      stack.push_back((int)n.a);
      if (n.b >= 0) stack.push_back((int)n.b);
    }
  }
  for (const Node& n : g_nodes)
    if (n.live && n.kind < N_NEG) ++g_tally[n.data ? n.phase : PH_GEOMETRY][tally_kind(n.kind)];
  if (g_nodes.size() > g_max_unit) g_max_unit = g_nodes.size();  // a statistic: races harmless
  g_nodes.clear();
  g_roots.clear();
  ++h_cur;
  g_gen = g_next_gen.fetch_add(1);
}

// Parallel regions: each thread starts from zero and adds its counts to the merged ones.
static void counts_begin() {
  std::memset(g_raw, 0, sizeof(g_raw));
  std::memset(g_tally, 0, sizeof(g_tally));
}
static void counts_end() {
#pragma omp critical(hzo_opcount_merge)
  for (int p = 0; p < NPH; ++p)
    for (int q = 0; q < NOP; ++q) {
      s_raw[p][q] += g_raw[p][q];
      s_tally[p][q] += g_tally[p][q];
    }
  counts_begin();
}

// The oracle's own loops run on one thread while they are counted or must not be.
struct OneThread {
  int n;
  OneThread() : n(omp_get_max_threads()) { omp_set_num_threads(1); }
  ~OneThread() { omp_set_num_threads(n); }
};

inline Counted operator-(const Counted& a) {
  if (a.z) return a;
  Counted r = counted_op(N_NEG, a, nullptr, -a.v);
  return r;
}
inline Counted operator+(const Counted& a, const Counted& b) {
  if (a.z) return b;
  if (b.z) return a;
  return counted_op(N_ADD, a, &b, a.v + b.v);
}
inline Counted operator-(const Counted& a, const Counted& b) {
  if (b.z) return a;
  if (a.z) return -b;
  return counted_op(N_SUB, a, &b, a.v - b.v);
}
inline Counted operator*(const Counted& a, const Counted& b) {
  if (a.z || b.z) return Counted();
  return counted_op(N_MUL, a, &b, a.v * b.v);
}
inline Counted operator/(const Counted& a, const Counted& b) {
  if (a.z) return Counted();
  return counted_op(N_DIV, a, &b, a.v / b.v);
}
inline Counted& operator+=(Counted& a, const Counted& b) { return a = a + b; }
inline Counted& operator-=(Counted& a, const Counted& b) { return a = a - b; }
inline Counted& operator*=(Counted& a, const Counted& b) { return a = a * b; }
inline Counted& operator/=(Counted& a, const Counted& b) { return a = a / b; }

// decisions on the value, sign and min / max: no arithmetic, but the operands are needed
inline double re(const Counted& x) {
  use(x);
  return x.v;
}
inline Counted absv(const Counted& x) {
  use(x);
  return x.v < 0.0 ? -x : x;
}
inline Counted minv(const Counted& a, const Counted& b) {
  use(a);
  use(b);
  return b.v < a.v ? b : a;
}
inline Counted maxv(const Counted& a, const Counted& b) {
  use(a);
  use(b);
  return a.v < b.v ? b : a;
}

}  // namespace hzo

namespace std {
inline hzo::Counted sqrt(const hzo::Counted& a) {
  if (a.z) return a;
  return hzo::counted_op(hzo::N_SQRT, a, nullptr, std::sqrt(a.v));
}
}  // namespace std

#include "hz_oracle.cpp"

namespace hzo {

// The oracle solves for the root in double; nothing to polish for the counting scalar.
static void polish_Z(const C2PIn<Counted>&, Counted&, double) {}

// Counts (raw and distinct) of the recovery's root solve, which the oracle runs in double:
// the bracket set-up, and one Newton iteration with its stopping test.
struct SolveCost {
  long long raw_bracket[NOP], raw_iter[NOP], dag_bracket[NOP], dag_iter[NOP];
};

static SolveCost solve_costs(double gamma) {
  SolveCost sc;
  long long save_raw[NPH][NOP], save_tally[NPH][NOP];
  std::memcpy(save_raw, g_raw, sizeof(save_raw));
  std::memcpy(save_tally, g_tally, sizeof(save_tally));
  const int ph = g_phase;
  g_phase = PH_C2P;
  flush();
  C2PIn<Counted> c;
  c.D = counted_data(1.0);
  c.E = counted_data(2.0);
  c.S2 = counted_data(0.3);
  c.SB = counted_data(0.1);
  c.B2 = counted_data(0.2);
  const Counted Z = counted_data(1.5);
  std::memset(g_raw, 0, sizeof(g_raw));
  std::memset(g_tally, 0, sizeof(g_tally));
  {
    const Counted Zhi = gamma * c.E;
    const Counted Zlo = Zhi * 1e-100;
    use(v2_of_Z(c, Zhi));
    use(v2_of_Z(c, Zlo));
    use(f_of_Z(c, Zlo, gamma));
    use(f_of_Z(c, Zhi, gamma));
    flush();
  }
  for (int q = 0; q < NOP; ++q) {
    sc.raw_bracket[q] = g_raw[PH_C2P][q];
    sc.dag_bracket[q] = g_tally[PH_C2P][q];
  }
  std::memset(g_raw, 0, sizeof(g_raw));
  std::memset(g_tally, 0, sizeof(g_tally));
  {
    const Counted f = f_of_Z(c, Z, gamma);
    const Counted fp = df_dZ(c, Z, gamma);
    const Counted Zn = Z - f / fp;
    use(Zn);
    use(Zn - Z);  // |Zn - Z| against the tolerance
    use(1e-15 * Z);
    flush();
  }
  for (int q = 0; q < NOP; ++q) {
    sc.raw_iter[q] = g_raw[PH_C2P][q];
    sc.dag_iter[q] = g_tally[PH_C2P][q];
  }
  std::memcpy(g_raw, save_raw, sizeof(save_raw));
  std::memcpy(g_tally, save_tally, sizeof(save_tally));
  g_phase = ph;
  return sc;
}
// The oracle's right-hand side, face by face and cell by cell, with the phase of each call.
// Units: one face (reconstruction to HLLE, its fluxes the results), one cell of the divergence
// of one axis, one cell of the sources.
static void rhs_phased(const Mesh& M, const hzo_opts& o, const double* met, const Counted* prim,
                       std::vector<Counted>& L) {
  const int* n = M.g.n;
  const long nc = M.ncell;
  L.assign((size_t)nc * NCONS, Counted(0.0));
  std::vector<Counted> Pp;
  fill_ghosts(M, prim, Pp);
  const long npd = M.npad();
  for (int d = 0; d < 3; ++d) {
    if (!M.act[d]) continue;
    int e[3] = {0, 0, 0};
    e[d] = 1;
    int nf[3] = {n[0], n[1], n[2]};
    nf[d] += 1;
    const long nfaces = (long)nf[0] * nf[1] * nf[2];
    std::vector<Counted> Ff((size_t)nfaces * NCONS);
#pragma omp parallel
    {
    counts_begin();
#pragma omp for schedule(dynamic, 64)
    for (long fidx = 0; fidx < nfaces; ++fidx) {
      const int i = (int)(fidx % nf[0]);
      const int j = (int)((fidx / nf[0]) % nf[1]);
      const int k = (int)(fidx / ((long)nf[0] * nf[1]));
      Counted PL[NPRIM], PR[NPRIM];
      g_phase = PH_RECON;
      for (int f = 0; f < NPRIM; ++f) {
        auto at = [&](int s) { return Pp[(size_t)f * npd + M.pcell(i + s * e[0], j + s * e[1], k + s * e[2])]; };
        Counted q[6] = {at(-3), at(-2), at(-1), at(0), at(1), at(2)};
        reconstruct(o.recon, q, &PL[f], &PR[f]);
      }
      g_phase = PH_FACE_STATE;
      Counted mA[NMET], mB[NMET], mf[NMET];
      load_metric(M, met, M.mcell(i - e[0], j - e[1], k - e[2]), mA);
      load_metric(M, met, M.mcell(i, j, k), mB);
      for (int f = 0; f < NMET; ++f) mf[f] = 0.5 * (mA[f] + mB[f]);
      Geom<Counted> G = make_geom(mf);
      State<Counted> SL = make_state(G, PL, o.gamma), SR = make_state(G, PR, o.gamma);
      g_phase = PH_FLUX;
      Counted FL[NCONS], FR[NCONS], UL[NCONS], UR[NCONS];
      flux(G, SL, d, o, FL);
      flux(G, SR, d, o, FR);
      prim2cons(G, SL, UL);
      prim2cons(G, SR, UR);
      g_phase = PH_SPEEDS;
      Counted lmL, lpL, lmR, lpR;
      speeds(G, SL, d, o.gamma, &lmL, &lpL);
      speeds(G, SR, d, o.gamma, &lmR, &lpR);
      g_phase = PH_HLLE;
      Counted sl = minv(Counted(0.0), minv(lmL, lmR));
      Counted sr = maxv(Counted(0.0), maxv(lpL, lpR));
      Counted* out = &Ff[(size_t)fidx * NCONS];
      for (int q = 0; q < NCONS; ++q) out[q] = hlle(sl, sr, FL[q], FR[q], UL[q], UR[q]);
      if (o.cleaning) {
        Counted cm, cp;
        clean_speeds(G, d, o.ch, &cm, &cp);
        Counted csl = minv(Counted(0.0), cm), csr = maxv(Counted(0.0), cp);
        out[CBX + d] = hlle(csl, csr, FL[CBX + d], FR[CBX + d], UL[CBX + d], UR[CBX + d]);
        out[CPSI] = hlle(csl, csr, FL[CPSI], FR[CPSI], UL[CPSI], UR[CPSI]);
      }
      for (int q = 0; q < NCONS; ++q) use(out[q]);
      flush();
    }
    counts_end();
    }
    const double idx = 1.0 / M.g.dx[d];
#pragma omp parallel
    {
    counts_begin();
    g_phase = PH_DIVERGENCE;
#pragma omp for schedule(static)
    for (long c = 0; c < nc; ++c) {
      const int i = (int)(c % n[0]);
      const int j = (int)((c / n[0]) % n[1]);
      const int k = (int)(c / ((long)n[0] * n[1]));
      const long fm = i + (long)nf[0] * (j + (long)nf[1] * k);
      const long fp = (i + e[0]) + (long)nf[0] * ((j + e[1]) + (long)nf[1] * (k + e[2]));
      for (int q = 0; q < NCONS; ++q) {
        Counted& l = L[(size_t)q * nc + c];
        l -= (Ff[(size_t)fp * NCONS + q] - Ff[(size_t)fm * NCONS + q]) * idx;
        use(l);
      }
      flush();
    }
    counts_end();
    }
  }
#pragma omp parallel
  {
  counts_begin();
  g_phase = PH_SOURCES;
#pragma omp for schedule(static)
  for (long c = 0; c < nc; ++c) {
    const int i = (int)(c % n[0]);
    const int j = (int)((c / n[0]) % n[1]);
    const int k = (int)(c / ((long)n[0] * n[1]));
    Counted m0[NMET];
    load_metric(M, met, M.mcell(i, j, k), m0);
    Geom<Counted> G = make_geom(m0);
    Counted P[NPRIM];
    for (int f = 0; f < NPRIM; ++f) P[f] = prim[(size_t)f * nc + c];
    State<Counted> S = make_state(G, P, o.gamma);
    for (int d = 0; d < 3; ++d) {
      if (!M.act[d]) continue;
      int e[3] = {0, 0, 0};
      e[d] = 1;
      Counted mp[NMET], mm[NMET];
      load_metric(M, met, M.mcell(i + e[0], j + e[1], k + e[2]), mp);
      load_metric(M, met, M.mcell(i - e[0], j - e[1], k - e[2]), mm);
      Geom<Counted> Gp = make_geom(mp), Gm = make_geom(mm);
      Counted src = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          Counted dg = (Gp.g4[a][b] - Gm.g4[a][b]) / (2.0 * M.g.dx[d]);
          src += Tup(G, S, a, b) * dg;
        }
      L[(size_t)(CTX + d) * nc + c] += 0.5 * G.sqrtmg * src;
      use(L[(size_t)(CTX + d) * nc + c]);
    }
    if (o.cleaning) {
      Counted Psi = G.sqrtgam * S.psi;
      L[(size_t)CPSI * nc + c] += -o.kappa * G.alp * Psi;
      use(L[(size_t)CPSI * nc + c]);
    }
    flush();
  }
  counts_end();
  }
}

// One RK3 step of the oracle from prim (field-major, n_cell each) with the step size dt and the
// CFL maximum at its start (as the oracle's evolve takes it), counted per phase.  raw and
// tally: NPH x NOP counts of the whole step (every operation; distinct operations per unit).
// With check_rhs, check[0..2]: per stage, the raw count of the phased right-hand side minus
// that of the oracle's rhs() (run on one thread); vdiff: largest |difference| of their values.
// iters: recovery iterations over the step; calls: recoveries that ran the root solve.
static void count_step(const Mesh& M, const hzo_opts& o, const double* met, const double* prim_in,
                       double dt, int check_rhs, long long* raw, long long* tally, long long* check,
                       double* vdiff, long* iters, long* calls) {
  const long nc = M.ncell;
  const int* n = M.g.n;
  const size_t N = (size_t)nc * NCONS;
  const SolveCost sc = solve_costs(o.gamma);
  std::vector<Counted> P((size_t)nc * NPRIM), U0(N), U1(N), L, Lref;
  for (size_t q = 0; q < P.size(); ++q) P[q] = counted_data(prim_in[q]);
  {
    OneThread one;
    g_dag = false;
    grid_prim2cons(M, o, met, P.data(), U0.data());  // the step's input: not counted
    g_dag = true;
  }
  for (size_t q = 0; q < N; ++q) U0[q] = counted_data(U0[q].v);
  flush();
  std::memset(s_raw, 0, sizeof(s_raw));
  std::memset(s_tally, 0, sizeof(s_tally));
  long it_sum = 0, call_sum = 0;
  *vdiff = 0.0;

  // CFL maximum at the start of the step, as the oracle's max_speed (unit: one cell)
#pragma omp parallel
  {
    counts_begin();
    g_phase = PH_CFL;
#pragma omp for schedule(static)
    for (long c = 0; c < nc; ++c) {
      const int i = (int)(c % n[0]);
      const int j = (int)((c / n[0]) % n[1]);
      const int k = (int)(c / ((long)n[0] * n[1]));
      Counted m[NMET], Pc[NPRIM];
      load_metric(M, met, M.mcell(i, j, k), m);
      for (int f = 0; f < NPRIM; ++f) Pc[f] = P[(size_t)f * nc + c];
      Geom<Counted> G = make_geom(m);
      State<Counted> S = make_state(G, Pc, o.gamma);
      for (int d = 0; d < 3; ++d) {
        if (!M.act[d]) continue;
        Counted lm, lp;
        speeds(G, S, d, o.gamma, &lm, &lp);
        Counted v = maxv(absv(lm), absv(lp));
        if (o.cleaning) {
          Counted cm, cp;
          clean_speeds(G, d, o.ch, &cm, &cp);
          v = maxv(v, maxv(absv(cm), absv(cp)));
        }
        v = v / M.g.dx[d];
        use(v);
      }
      flush();
    }
    counts_end();
  }

  for (int stage = 0; stage < 3; ++stage) {
    long long before = 0;
    for (int p = 0; p < NPH; ++p)
      for (int q = 0; q < NOP; ++q) before += s_raw[p][q];
    rhs_phased(M, o, met, P.data(), L);
    if (check_rhs) {
      long long phased = -before;
      for (int p = 0; p < NPH; ++p)
        for (int q = 0; q < NOP; ++q) phased += s_raw[p][q];
      OneThread one;
      counts_begin();
      g_dag = false;
      rhs(M, o, met, P.data(), Lref);
      g_dag = true;
      long long ref = 0;
      for (int p = 0; p < NPH; ++p)
        for (int q = 0; q < NOP; ++q) ref += g_raw[p][q];
      counts_begin();
      check[stage] = phased - ref;
      for (size_t q = 0; q < N; ++q) *vdiff = std::fmax(*vdiff, std::fabs(L[q].v - Lref[q].v));
    } else {
      check[stage] = 0;
    }
#pragma omp parallel reduction(+ : it_sum, call_sum)
    {
      counts_begin();
      // RK update (unit: one cell)
      g_phase = PH_UPDATE;
#pragma omp for schedule(static)
      for (long c = 0; c < nc; ++c) {
        for (int f = 0; f < NCONS; ++f) {
          const size_t q = (size_t)f * nc + c;
          if (stage == 0) U1[q] = U0[q] + dt * L[q];
          else if (stage == 1) U1[q] = 0.75 * U0[q] + 0.25 * (U1[q] + dt * L[q]);
          else U1[q] = (1.0 / 3.0) * U0[q] + (2.0 / 3.0) * (U1[q] + dt * L[q]);
          use(U1[q]);
        }
        flush();
      }
      // recovery (unit: one cell)
      g_phase = PH_C2P;
#pragma omp for schedule(dynamic, 64)
      for (long c = 0; c < nc; ++c) {
        const int i = (int)(c % n[0]);
        const int j = (int)((c / n[0]) % n[1]);
        const int k = (int)(c / ((long)n[0] * n[1]));
        Counted m[NMET], U[NCONS], Pg[NPRIM], Pn[NPRIM];
        load_metric(M, met, M.mcell(i, j, k), m);
        Geom<Counted> G = make_geom(m);
        for (int f = 0; f < NCONS; ++f) U[f] = U1[(size_t)f * nc + c];
        for (int f = 0; f < NPRIM; ++f) Pg[f] = P[(size_t)f * nc + c];
        int it = 0;
        recover_cell(G, U, Pg, o, Pn, &it);
        for (int f = 0; f < NCONS; ++f) use(U[f]);
        for (int f = 0; f < NPRIM; ++f) use(Pn[f]);
        flush();
        if (it > 0) {
          for (int q = 0; q < NOP; ++q) {
            g_raw[PH_C2P][q] += sc.raw_bracket[q] + (long long)it * sc.raw_iter[q];
            g_tally[PH_C2P][q] += sc.dag_bracket[q] + (long long)it * sc.dag_iter[q];
          }
          it_sum += it;
          call_sum += 1;
        }
        // the stored state is data for what follows, whatever the recovery assigned
        for (int f = 0; f < NCONS; ++f) U1[(size_t)f * nc + c] = counted_data(U[f].v);
        for (int f = 0; f < NPRIM; ++f) P[(size_t)f * nc + c] = counted_data(Pn[f].v);
      }
      counts_end();
    }
  }
  *iters = it_sum;
  *calls = call_sum;
  std::memcpy(raw, s_raw, sizeof(s_raw));
  std::memcpy(tally, s_tally, sizeof(s_tally));
}

}  // namespace hzo

extern "C" {

int hzo_opcount_nphase() { return hzo::NPH; }
int hzo_opcount_nop() { return hzo::NOP; }
long hzo_opcount_max_unit() { return (long)hzo::g_max_unit; }

// One counted RK3 step; see count_step.  raw, tally: NPH x NOP; check: 3.  Threads: OpenMP.
void hzo_opcount_step(const hzo_grid* g, const hzo_opts* o, const double* met, const double* prim,
                      double dt, int check_rhs, long long* raw, long long* tally, long long* check,
                      double* vdiff, long* iters, long* calls) {
  hzo::Mesh M(*g);
  hzo::count_step(M, *o, met, prim, dt, check_rhs, raw, tally, check, vdiff, iters, calls);
}

}  // extern "C"
