// Operation-counting build of the oracle -- TEST INFRASTRUCTURE.
//
// This translation unit compiles mhd_oracle.c unchanged, as C++, with every
// `double` of the oracle replaced by `Real`: a value type that holds the same
// double and counts each arithmetic operation it takes part in.  The oracle's
// arithmetic therefore runs exactly as written (same values, same branches),
// and the counts are the algorithmic operation counts of the method as the
// oracle states it (Sec. 2.2 of the paper: primitive recovery, PLM-MC,
// HLLD/HLL, constrained-transport EMFs, flux divergence, RK stages, CFL).
//
// Categories: add (also subtract and negation-free sums), mul, div, sqrt
// (each one flop), and non-flop operations: compare, abs/min/max/copysign.
// Only the oracle package's tests and its measurement script use this build.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace opc {
enum { ADD, MUL, DIV, SQRT, CMP, MISC, NCAT };
static unsigned long long g_count[NCAT];
}  // namespace opc

struct Real {
  double v;
  Real() = default;
  Real(double x) : v(x) {}
  explicit operator float() const { return (float)v; }
  explicit operator int() const { return (int)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
  Real& operator+=(Real o) { ++opc::g_count[opc::ADD]; v += o.v; return *this; }
  Real& operator-=(Real o) { ++opc::g_count[opc::ADD]; v -= o.v; return *this; }
  Real& operator*=(Real o) { ++opc::g_count[opc::MUL]; v *= o.v; return *this; }
  Real& operator/=(Real o) { ++opc::g_count[opc::DIV]; v /= o.v; return *this; }
};
static_assert(sizeof(Real) == sizeof(double), "Real must share the layout of double");

static inline Real operator+(Real a, Real b) { ++opc::g_count[opc::ADD]; return Real(a.v + b.v); }
static inline Real operator-(Real a, Real b) { ++opc::g_count[opc::ADD]; return Real(a.v - b.v); }
static inline Real operator*(Real a, Real b) { ++opc::g_count[opc::MUL]; return Real(a.v * b.v); }
static inline Real operator/(Real a, Real b) { ++opc::g_count[opc::DIV]; return Real(a.v / b.v); }
static inline Real operator-(Real a) { return Real(-a.v); }   // sign flip: no arithmetic
static inline Real operator+(Real a) { return a; }
static inline bool operator<(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v < b.v; }
static inline bool operator>(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v > b.v; }
static inline bool operator<=(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v <= b.v; }
static inline bool operator>=(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v >= b.v; }
static inline bool operator==(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v == b.v; }
static inline bool operator!=(Real a, Real b) { ++opc::g_count[opc::CMP]; return a.v != b.v; }
static inline Real sqrt(Real a) { ++opc::g_count[opc::SQRT]; return Real(::sqrt(a.v)); }
static inline Real fabs(Real a) { ++opc::g_count[opc::MISC]; return Real(::fabs(a.v)); }
static inline Real fmax(Real a, Real b) { ++opc::g_count[opc::MISC]; return Real(::fmax(a.v, b.v)); }
static inline Real fmin(Real a, Real b) { ++opc::g_count[opc::MISC]; return Real(::fmin(a.v, b.v)); }
static inline Real copysign(Real a, Real b) { ++opc::g_count[opc::MISC]; return Real(::copysign(a.v, b.v)); }
static inline bool isfinite(Real a) { return ::isfinite(a.v); }
static inline bool isnan(Real a) { return ::isnan(a.v); }

#define double Real
extern "C" {
#include "mhd_oracle.c"
}
#undef double

extern "C" {

void orc_opcount_reset(void) {
  for (int i = 0; i < opc::NCAT; ++i) opc::g_count[i] = 0;
}

// counts so far: add, mul, div, sqrt, compare, abs/min/max/copysign
void orc_opcount_get(unsigned long long out[6]) {
  for (int i = 0; i < opc::NCAT; ++i) out[i] = opc::g_count[i];
}

// The primitive-recovery part of one operator evaluation alone (the same
// grid setup as the operator, then its primitive stage).
void orc_opcount_prims(const orc_cfg *c, Real *const cell[5], Real *const face[3]) {
  grid g;
  g.c = c;
  g.st = NULL;
  g.zout = NULL;
  g.n[0] = c->nx; g.n[1] = c->ny; g.n[2] = c->nz;
  for (int d = 0; d < 3; ++d) {
    g.N[d] = g.n[d] + 2 * NG;
    g.nf[d] = g.n[d] + (c->bc[d] == ORC_OUTFLOW ? 1 : 0);
  }
  g.ncell = (size_t)g.N[0] * g.N[1] * g.N[2];
  g.nedge = (size_t)(g.N[0] + 1) * (g.N[1] + 1) * (g.N[2] + 1);
  Real *W[8], *Bf[3];
  for (int v = 0; v < 8; ++v) W[v] = (Real *)calloc(g.ncell, sizeof(Real));
  for (int d = 0; d < 3; ++d) Bf[d] = (Real *)calloc(g.nedge, sizeof(Real));
  build_primitives(&g, cell, face, W, Bf, NULL);
  for (int v = 0; v < 8; ++v) free(W[v]);
  for (int d = 0; d < 3; ++d) free(Bf[d]);
}

}  // extern "C"
