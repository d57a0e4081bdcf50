// flop_count.cpp -- TEST INFRASTRUCTURE ONLY (like hweno_oracle.c, which it compiles).
//
// Counts the floating-point operations of one oracle stage.  The oracle's C source is
// compiled unchanged as C++ with a counting scalar type in place of double: every value
// carries its double and a reference into a dataflow tape.  Values that do not depend on the
// stage input (literals, problem constants such as dx, gamma - 1 or the linear weights) are
// constants and cost nothing; an operation on a constant and a tracked value, or on two
// tracked values, adds a tape node.  Two counts are reported per operation kind:
//   executed   every tape node created while the stage runs;
//   dataflow   the distinct nodes from which a stage output is reachable, after merging
//              repeated identical operations (same operation on the same operands, e.g. a
//              face flux that the oracle forms once for each of the face's two cells) and
//              after the identities x*1, x*0, x+0, x-0, x/1 -- i.e. the arithmetic the
//              oracle's formulas need to produce the stage's outputs, once each.
// The wave speeds of the LF flux (max over all cells) are counted separately, as executed
// operations per cell: a maximum depends on every cell's speed although only one survives.
// Comparisons, negations and absolute values are not counted as flops.
#include <math.h>
#include <stdint.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <unordered_map>
#include <vector>

namespace fc {

enum Op : uint8_t { INPUT, ADD, SUB, MUL, DIV, SQRT, NEG, ABS, NOPS };

struct Node {
  Op op;
  int32_t a, b;  // operands: node index >= 0, constant index encoded as -2 - k, unused -1
};

struct Tape {
  std::vector<Node> nodes;
  std::vector<double> consts;
  std::unordered_map<uint64_t, int32_t> const_ix;
  std::unordered_map<uint64_t, int32_t> cse;  // (op, a, b) -> node
  uint64_t executed[NOPS] = {};

  void reset() {
    nodes.clear();
    consts.clear();
    const_ix.clear();
    cse.clear();
    memset(executed, 0, sizeof(executed));
  }
  int32_t constant(double v) {
    uint64_t bits;
    memcpy(&bits, &v, 8);
    auto it = const_ix.find(bits);
    if (it != const_ix.end()) return -2 - it->second;
    const int32_t k = (int32_t)consts.size();
    consts.push_back(v);
    const_ix.emplace(bits, k);
    return -2 - k;
  }
  int32_t input() {
    nodes.push_back({INPUT, -1, -1});
    return (int32_t)nodes.size() - 1;
  }
  int32_t node(Op op, int32_t a, int32_t b) {
    ++executed[op];
    if ((op == ADD || op == MUL) && a > b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    // exact key: 4 bits of operation, 30 bits per operand (nodes below 2^29, constants
    // from 2^29 on; the tapes counted here stay far below both limits)
    auto enc = [](int32_t x) -> uint64_t {
      if (x == -1) return (1ull << 30) - 1;   // no operand
      return x >= 0 ? (uint64_t)x : (1ull << 29) + (uint64_t)(-2 - x);
    };
    const uint64_t key = ((uint64_t)op << 60) | (enc(a) << 30) | enc(b);
    auto it = cse.find(key);
    if (it != cse.end()) return it->second;
    nodes.push_back({op, a, b});
    const int32_t id = (int32_t)nodes.size() - 1;
    cse[key] = id;
    return id;
  }
};

Tape tape;

}  // namespace fc

// The counting scalar.  id == -1: a constant (not derived from the stage input).
struct F {
  double v;
  int32_t id;
  F() : v(0.0), id(-1) {}
  F(double x) : v(x), id(-1) {}
};

static inline int32_t ref_of(const F& x) { return x.id >= 0 ? x.id : fc::tape.constant(x.v); }
static inline bool is_const(const F& x, double c) { return x.id < 0 && x.v == c; }

static inline F mk(double v, fc::Op op, const F& a, const F& b) {
  F r(v);
  if (a.id < 0 && b.id < 0) return r;  // constant folding
  r.id = fc::tape.node(op, ref_of(a), ref_of(b));
  return r;
}
static inline F mk1(double v, fc::Op op, const F& a) {
  F r(v);
  if (a.id < 0) return r;
  r.id = fc::tape.node(op, a.id, -1);
  return r;
}

static inline F operator+(const F& a, const F& b) {
  if (is_const(a, 0.0)) return b;
  if (is_const(b, 0.0)) return a;
  return mk(a.v + b.v, fc::ADD, a, b);
}
static inline F operator-(const F& a) { return mk1(-a.v, fc::NEG, a); }
static inline F operator-(const F& a, const F& b) {
  if (is_const(b, 0.0)) return a;
  if (is_const(a, 0.0)) return -b;
  return mk(a.v - b.v, fc::SUB, a, b);
}
static inline F operator*(const F& a, const F& b) {
  if (is_const(a, 1.0)) return b;
  if (is_const(b, 1.0)) return a;
  if (is_const(a, -1.0)) return -b;
  if (is_const(b, -1.0)) return -a;
  if (is_const(a, 0.0) || is_const(b, 0.0)) return F(a.v * b.v);
  return mk(a.v * b.v, fc::MUL, a, b);
}
static inline F operator/(const F& a, const F& b) {
  if (is_const(b, 1.0)) return a;
  return mk(a.v / b.v, fc::DIV, a, b);
}
static inline F& operator+=(F& a, const F& b) { return a = a + b; }
static inline F& operator-=(F& a, const F& b) { return a = a - b; }
static inline F& operator*=(F& a, const F& b) { return a = a * b; }
static inline F& operator/=(F& a, const F& b) { return a = a / b; }
static inline bool operator<(const F& a, const F& b) { return a.v < b.v; }
static inline bool operator>(const F& a, const F& b) { return a.v > b.v; }
static inline bool operator<=(const F& a, const F& b) { return a.v <= b.v; }
static inline bool operator>=(const F& a, const F& b) { return a.v >= b.v; }
static inline bool operator==(const F& a, const F& b) { return a.v == b.v; }
static inline bool operator!=(const F& a, const F& b) { return a.v != b.v; }
static inline F fabs(const F& a) { return mk1(fabs(a.v), fc::ABS, a); }
static inline F sqrt(const F& a) { return mk1(sqrt(a.v), fc::SQRT, a); }
static inline bool isfinite(const F& a) { return std::isfinite(a.v); }

// the oracle, with the counting scalar for every double
#define double F
#include "hweno_oracle.c"
#undef double

// ------------------------------------------------------------------------------------------
// Entry point.  P_plain: the oracle's problem with plain doubles (hweno_oracle.h layout).
// Uin, Un: NC*NM arrays of ny*nx; Vh: NC*(NM-1) arrays (read for k > 1).  The stage's LF
// speeds and dt are inputs.  counts[0..5] = dataflow add, sub, mul, div, sqrt, total;
// counts[6..11] = executed add, sub, mul, div, sqrt, total; counts[12..17] = executed add,
// sub, mul, div, sqrt, total of the wave-speed evaluation of all cells (orc_alpha).
// Returns the oracle's stage status, or -1.
struct plain_problem {
  int dim, eq, nx, ny;
  double x0, x1, y0, y1, ax, ay, gam;
  int bc[4];
  int characteristic, weights, rk;
  double gamma_lo, eps, cfl;
};

extern "C" int orc_count_stage_flops(const plain_problem* Pp, int k, const double* Uin,
                                     const double* Un, const double* Vh, const double* alpha,
                                     double dt, int64_t counts[18]) {
  orc_problem P;
  P.dim = Pp->dim;
  P.eq = Pp->eq;
  P.nx = Pp->nx;
  P.ny = Pp->ny;
  P.x0 = Pp->x0; P.x1 = Pp->x1; P.y0 = Pp->y0; P.y1 = Pp->y1;
  P.ax = Pp->ax; P.ay = Pp->ay; P.gam = Pp->gam;
  for (int s = 0; s < 4; ++s) P.bc[s] = Pp->bc[s];
  P.characteristic = Pp->characteristic;
  P.weights = Pp->weights;
  P.rk = Pp->rk;
  P.gamma_lo = Pp->gamma_lo; P.eps = Pp->eps; P.cfl = Pp->cfl;
  const int nc = orc_ncomp(&P), nm = orc_nmom(&P);
  const size_t ncell = (size_t)P.nx * P.ny;
  const size_t nU = (size_t)nc * nm * ncell, nV = (size_t)nc * (nm - 1) * ncell;
  std::vector<F> fUin(nU), fUn(nU), fVh(nV), fUout(nU);
  fc::tape.reset();
  for (size_t q = 0; q < nU; ++q) {
    fUin[q] = F(Uin[q]);
    fUin[q].id = fc::tape.input();
    fUn[q] = F(Un[q]);
    fUn[q].id = fc::tape.input();
  }
  for (size_t q = 0; q < nV; ++q) {
    fVh[q] = F(Vh ? Vh[q] : 0.0);
    fVh[q].id = fc::tape.input();
  }
  F fa[2] = {F(alpha[0]), F(alpha[1])};
  fa[0].id = fc::tape.input();
  fa[1].id = fc::tape.input();
  F fdt(dt);
  fdt.id = fc::tape.input();
  // k == 1: the stage reads U^n = its input (the oracle is called that way)
  const int rc = orc_stage(&P, k, fUin.data(), k == 1 ? fUin.data() : fUn.data(), fVh.data(),
                           fa, fdt, fUout.data());
  // reachability from the outputs
  std::vector<uint8_t> live(fc::tape.nodes.size(), 0);
  std::vector<int32_t> stack;
  auto mark = [&](const F& x) {
    if (x.id >= 0 && !live[x.id]) {
      live[x.id] = 1;
      stack.push_back(x.id);
    }
  };
  for (size_t q = 0; q < nU; ++q) mark(fUout[q]);
  if (k == 1)
    for (size_t q = 0; q < nV; ++q) mark(fVh[q]);
  while (!stack.empty()) {
    const fc::Node n = fc::tape.nodes[stack.back()];
    stack.pop_back();
    for (int32_t o : {n.a, n.b})
      if (o >= 0 && !live[o]) {
        live[o] = 1;
        stack.push_back(o);
      }
  }
  int64_t df[fc::NOPS] = {};
  for (size_t i = 0; i < fc::tape.nodes.size(); ++i)
    if (live[i]) ++df[fc::tape.nodes[i].op];
  const fc::Op kinds[5] = {fc::ADD, fc::SUB, fc::MUL, fc::DIV, fc::SQRT};
  int64_t tot = 0, tex = 0;
  for (int q = 0; q < 5; ++q) {
    counts[q] = df[kinds[q]];
    tot += df[kinds[q]];
    counts[6 + q] = (int64_t)fc::tape.executed[kinds[q]];
    tex += (int64_t)fc::tape.executed[kinds[q]];
  }
  counts[5] = tot;
  counts[11] = tex;
  // wave speeds of every cell (the LF speed of the next stage is their maximum)
  fc::tape.reset();
  for (size_t q = 0; q < nU; ++q) fUout[q].id = fc::tape.input();
  F am[2];
  orc_alpha(&P, fUout.data(), am);
  int64_t ta = 0;
  for (int q = 0; q < 5; ++q) {
    counts[12 + q] = (int64_t)fc::tape.executed[kinds[q]];
    ta += counts[12 + q];
  }
  counts[17] = ta;
  fc::tape.reset();
  return rc;
}
