// Forward-mode dual numbers for the oracle (test infrastructure only).
//
// A Dual carries a value and its derivatives with respect to up to
// kDualMax free parameters. Every operation applies the chain rule
// exactly (no step size, no truncation), so derivatives are exact up to
// floating-point rounding. The oracle instantiates its model code with
// both `double` and `Dual`; the `double` instantiation gives ln L and the
// `Dual` instantiation gives ln L together with its gradient.
#pragma once
#include <cmath>

namespace oracle {

constexpr int kDualMax = 11;

struct Dual {
  double v;
  double d[kDualMax];
  Dual() : v(0.0) { for (int i = 0; i < kDualMax; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < kDualMax; ++i) d[i] = 0.0; }
  static Dual variable(double x, int i) { Dual r(x); r.d[i] = 1.0; return r; }
};

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

// f(x) with f(x.v) = fv and f'(x.v) = fp.
inline Dual chain(const Dual& x, double fv, double fp) {
  Dual r(fv);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = fp * x.d[i];
  return r;
}

inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = -a.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) {
  Dual r(a.v * b);
  for (int i = 0; i < kDualMax; ++i) r.d[i] = a.d[i] * b;
  return r;
}
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }

inline Dual sqrt(const Dual& x) { double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
inline Dual log(const Dual& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
inline Dual exp(const Dual& x) { double e = std::exp(x.v); return chain(x, e, e); }
inline Dual sin(const Dual& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
inline Dual cos(const Dual& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
// x^p for a constant exponent p and x > 0.
inline Dual pow(const Dual& x, double p) {
  double y = std::pow(x.v, p);
  return chain(x, y, p * std::pow(x.v, p - 1.0));
}

using std::sqrt;
using std::log;
using std::exp;
using std::sin;
using std::cos;
using std::pow;

}  // namespace oracle
