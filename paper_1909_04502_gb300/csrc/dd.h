// Double-double arithmetic (value = hi + lo, |lo| <= ulp(hi)/2) for the
// host-side table construction, built on error-free transformations
// (Knuth's two-sum, fma-based two-product).  Deterministic on any IEEE-754
// host with a correctly rounded std::fma.
#pragma once
#include <cmath>

namespace rlbm {

struct dd {
  double hi = 0.0, lo = 0.0;
  dd() = default;
  dd(double h) : hi(h), lo(0.0) {}
  dd(double h, double l) : hi(h), lo(l) {}
  double to_double() const { return hi + lo; }
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd(s, e);
}

inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return dd(s, b - (s - a));
}

inline dd two_prod(double a, double b) {
  double p = a * b;
  return dd(p, std::fma(a, b, -p));
}

inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }

inline dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}

inline dd operator/(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = a - b * dd(q1);
  double q2 = r.hi / b.hi;
  r = r - b * dd(q2);
  double q3 = r.hi / b.hi;
  return dd(q1) + dd(q2) + dd(q3);
}

inline dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd(0.0);
  double x = std::sqrt(a.hi);
  dd r = a - two_prod(x, x);
  return dd(x) + dd(r.hi / (2.0 * x));
}

}  // namespace rlbm
