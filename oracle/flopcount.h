// flopcount.h -- operation-counting scalar for the oracle's flop-count build (-DORACLE_COUNT_FLOPS).
// TEST/MEASUREMENT INFRASTRUCTURE ONLY.  Every +, -, *, / and sqrt on a Counted value increments a
// global counter, so compiling the oracle's stage with `real` = Counted yields the exact number of
// floating-point operations its algorithm performs, phase by phase.
#pragma once
#include <cmath>
#include <cstdint>

struct OpCount {
  double add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
extern OpCount g_ops;

struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}  // NOLINT: implicit from double literals and inputs
  Counted& operator+=(Counted o) { g_ops.add++; v += o.v; return *this; }
  Counted& operator-=(Counted o) { g_ops.add++; v -= o.v; return *this; }
  Counted& operator*=(Counted o) { g_ops.mul++; v *= o.v; return *this; }
  Counted& operator/=(Counted o) { g_ops.div++; v /= o.v; return *this; }
};
inline Counted operator+(Counted a, Counted b) { g_ops.add++; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { g_ops.add++; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { g_ops.mul++; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { g_ops.div++; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { g_ops.cmp++; return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { g_ops.cmp++; return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { g_ops.cmp++; return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { g_ops.cmp++; return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { g_ops.cmp++; return a.v != b.v; }
namespace std {
inline Counted sqrt(Counted a) { g_ops.sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline bool isfinite(Counted a) { return std::isfinite(a.v); }
}  // namespace std
