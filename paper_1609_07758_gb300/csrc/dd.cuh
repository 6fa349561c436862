// Double-double ("dd") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, giving
// about 106 bits.  Built from the error-free transformations of Knuth (TwoSum),
// Dekker (FastTwoSum) and the FMA form of TwoProduct, following the algorithm
// descriptions of Hida, Li & Bailey, "Library for double-double and quad-double
// arithmetic" (2001).  Used for the 1D eigen-data, whose smallest eigenvalues are
// O((k/K)^2) while the matrix entries are O(n^2): FP64 loses up to 8 digits there.
#pragma once
#include <cmath>

#if defined(__CUDACC__)
#define DD_HD __host__ __device__ __forceinline__
#else
#define DD_HD inline
#endif

struct dd {
  double hi, lo;
};

DD_HD dd dd_make(double a) { return dd{a, 0.0}; }

DD_HD dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

DD_HD dd fast_two_sum(double a, double b) {  // requires |a| >= |b| or a == 0
  double s = a + b;
  double e = b - (s - a);
  return dd{s, e};
}

DD_HD dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd{p, e};
}

DD_HD dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

DD_HD dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
DD_HD dd operator-(dd a, dd b) { return a + (-b); }

DD_HD dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = fma(a.hi, b.lo, p.lo);
  p.lo = fma(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

DD_HD dd operator*(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo = fma(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// Long division: three quotient digits q1 + q2 + q3, each from the hi parts.
DD_HD dd operator/(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = a - b * q1;
  double q2 = r.hi / b.hi;
  r = r - b * q2;
  double q3 = r.hi / b.hi;
  dd q = fast_two_sum(q1, q2);
  return q + dd_make(q3);
}

// One Newton step x + (a - x^2) / (2x) from the FP64 root (quadratic convergence).
DD_HD dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd{0.0, 0.0};
  double x = sqrt(a.hi);
  dd xx = two_prod(x, x);
  dd r = a - xx;
  double corr = r.hi / (2.0 * x);
  return fast_two_sum(x, corr);
}

DD_HD dd dd_abs(dd a) { return a.hi < 0.0 ? -a : a; }
DD_HD bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
DD_HD bool operator>(dd a, dd b) { return b < a; }
DD_HD double dd_to_double(dd a) { return a.hi + a.lo; }
