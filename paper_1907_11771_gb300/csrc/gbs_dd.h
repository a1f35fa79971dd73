// Double-double ("dd") arithmetic on the host: a value is hi + lo with
// |lo| <= ulp(hi)/2, giving about 106 significant bits.  Built from the
// error-free transformations TwoSum (Knuth) and TwoProd via fused
// multiply-add, following Dekker (1971).  Used only for exact-enough weight
// solves and order-constraint checks in the scheme set-up.
#pragma once

#include <cmath>

namespace gbs {

struct dd {
  double hi, lo;
};

inline dd dd_from(double a) { return {a, 0.0}; }

inline dd two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

inline dd quick_two_sum(double a, double b) {
  const double s = a + b;
  return {s, b - (s - a)};
}

inline dd two_prod(double a, double b) {
  const double p = a * b;
  return {p, std::fma(a, b, -p)};
}

inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

inline dd operator-(dd a) { return {-a.hi, -a.lo}; }
inline dd operator-(dd a, dd b) { return a + (-b); }

inline dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}

inline dd operator/(dd a, dd b) {
  // long division: q1 = a/b, r = a - q1 b, q2 = r/b, ...
  const double q1 = a.hi / b.hi;
  dd r = a - b * dd_from(q1);
  const double q2 = r.hi / b.hi;
  r = r - b * dd_from(q2);
  const double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return q + dd_from(q3);
}

inline double dd_abs_hi(dd a) { return std::fabs(a.hi); }

}  // namespace gbs
