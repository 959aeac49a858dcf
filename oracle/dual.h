// Forward-mode dual numbers for the oracle (test infrastructure only).
//
// A DualN<N> carries a value and its derivatives with respect to up to N free
// parameters. Every operation applies the chain rule exactly (no step size, no
// truncation), so derivatives are exact up to floating-point rounding. The
// oracle instantiates its model code with `double` (ln L) and DualN<N> (ln L
// and its gradient), N = 2, 4 or 11 depending on the model's dimension.
#pragma once
#include <cmath>

namespace oracle {

template <int N>
struct DualN {
  double v;
  double d[N];
  DualN() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  DualN(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  static DualN variable(double x, int i) { DualN r(x); r.d[i] = 1.0; return r; }
};

inline double val(double x) { return x; }
template <int N>
inline double val(const DualN<N>& x) { return x.v; }

// f(x) with f(x.v) = fv and f'(x.v) = fp.
template <int N>
inline DualN<N> chain(const DualN<N>& x, double fv, double fp) {
  DualN<N> r(fv);
  for (int i = 0; i < N; ++i) r.d[i] = fp * x.d[i];
  return r;
}

template <int N>
inline DualN<N> operator+(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v + b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
inline DualN<N> operator-(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v - b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
inline DualN<N> operator-(const DualN<N>& a) {
  DualN<N> r(-a.v);
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
inline DualN<N> operator*(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v * b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
inline DualN<N> operator/(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N>
inline DualN<N> operator*(const DualN<N>& a, double b) {
  DualN<N> r(a.v * b);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> inline DualN<N> operator+(const DualN<N>& a, double b) { return a + DualN<N>(b); }
template <int N> inline DualN<N> operator+(double a, const DualN<N>& b) { return DualN<N>(a) + b; }
template <int N> inline DualN<N> operator-(const DualN<N>& a, double b) { return a - DualN<N>(b); }
template <int N> inline DualN<N> operator-(double a, const DualN<N>& b) { return DualN<N>(a) - b; }
template <int N> inline DualN<N> operator*(double a, const DualN<N>& b) { return b * a; }
template <int N> inline DualN<N> operator/(const DualN<N>& a, double b) { return a / DualN<N>(b); }
template <int N> inline DualN<N> operator/(double a, const DualN<N>& b) { return DualN<N>(a) / b; }

template <int N>
inline DualN<N> sqrt(const DualN<N>& x) { double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
template <int N>
inline DualN<N> log(const DualN<N>& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
template <int N>
inline DualN<N> exp(const DualN<N>& x) { double e = std::exp(x.v); return chain(x, e, e); }
template <int N>
inline DualN<N> sin(const DualN<N>& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
template <int N>
inline DualN<N> cos(const DualN<N>& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
// x^p for a constant exponent p and x > 0.
template <int N>
inline DualN<N> pow(const DualN<N>& x, double p) {
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
