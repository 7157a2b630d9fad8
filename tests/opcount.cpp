// Host tool: counts the floating-point operations of the model routines by
// instantiating them with a counting scalar.  Prints one line per routine:
//   name add mul div sincos
// These are the per-unit operation counts of the evaluation work used in the
// roofline model (the factorisation and solve counts are closed forms).
#include <cstdio>

#include "quad_model.cuh"

namespace {
long long g_add = 0, g_mul = 0, g_div = 0, g_sc = 0;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
Cnt operator+(Cnt a, Cnt b) { ++g_add; return Cnt(a.v + b.v); }
Cnt operator-(Cnt a, Cnt b) { ++g_add; return Cnt(a.v - b.v); }
Cnt operator-(Cnt a) { return Cnt(-a.v); }
Cnt operator*(Cnt a, Cnt b) { ++g_mul; return Cnt(a.v * b.v); }
Cnt operator/(Cnt a, Cnt b) { ++g_div; return Cnt(a.v / b.v); }
// found by argument-dependent lookup from the model templates
void sincos_s(Cnt a, Cnt* s, Cnt* c) {
  ++g_sc;
  *s = Cnt(::sin(a.v));
  *c = Cnt(::cos(a.v));
}
}  // namespace

using namespace bipm;

static void reset() { g_add = g_mul = g_div = g_sc = 0; }
static void report(const char* name) {
  std::printf("%s %lld %lld %lld %lld\n", name, g_add, g_mul, g_div, g_sc);
}

int main() {
  Cnt dt(0.05);
  {
    Cnt x[12], u[4], F[12];
    for (int i = 0; i < 12; ++i) x[i] = Cnt(0.1 * i);
    for (int i = 0; i < 4; ++i) u[i] = Cnt(1.2);
    reset();
    rk4_value<Cnt>(x, u, dt, F);
    report("rk4_value");
  }
  {
    Cnt x[12], u[4], F[12], gx[12], gu[4], lam[12];
    for (int i = 0; i < 12; ++i) { x[i] = Cnt(0.1 * i); lam[i] = Cnt(0.3); }
    for (int i = 0; i < 4; ++i) u[i] = Cnt(1.2);
    reset();
    rk4_fwd_rev<Cnt>(x, u, dt, lam, F, gx, gu);
    report("rk4_adjoint");
  }
  {
    typedef Dual<Cnt> D;
    D x[12], u[4], F[12], gx[12], gu[4];
    Cnt lam[12];
    for (int i = 0; i < 12; ++i) { x[i] = D{Cnt(0.1 * i), Cnt(0)}; lam[i] = Cnt(0.3); }
    for (int i = 0; i < 4; ++i) u[i] = D{Cnt(1.2), Cnt(0)};
    x[6].d = Cnt(1);
    reset();
    rk4_fwd_rev<D>(x, u, Dual<Cnt>{dt, Cnt(0)}.v, lam, F, gx, gu);
    report("rk4_dual_adjoint");
  }
  return 0;
}
