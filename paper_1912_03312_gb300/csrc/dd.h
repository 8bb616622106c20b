// Double-double ("dd", ~32 significant digits) real and complex arithmetic for
// the host-side plan construction.  Error-free transformations: TwoSum (Knuth),
// FastTwoSum and TwoProd via fused multiply-add (Dekker).  This file must be
// compiled with floating-point contraction disabled (-ffp-contract=off) so that
// the compiler does not fuse the compensation terms.
#pragma once

#include <cmath>

namespace rexi {

struct dd {
    double hi, lo;
    dd() : hi(0.0), lo(0.0) {}
    dd(double h) : hi(h), lo(0.0) {}
    dd(double h, double l) : hi(h), lo(l) {}
    explicit operator double() const { return hi + lo; }
};

inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return dd(s, e);
}
inline dd fast_two_sum(double a, double b) {  // requires |a| >= |b|
    double s = a + b;
    double e = b - (s - a);
    return dd(s, e);
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = std::fma(a, b, -p);
    return dd(p, e);
}

inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return q + dd(q3);
}
inline dd& operator+=(dd& a, dd b) { a = a + b; return a; }
inline dd& operator-=(dd& a, dd b) { a = a - b; return a; }
inline dd& operator*=(dd& a, dd b) { a = a * b; return a; }
inline dd& operator/=(dd& a, dd b) { a = a / b; return a; }
inline bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline bool operator>(dd a, dd b) { return b < a; }
inline dd dabs(dd a) { return a.hi < 0.0 ? -a : a; }
inline dd dsqrt(dd a) {
    if (a.hi <= 0.0) return dd(0.0);
    double x = 1.0 / std::sqrt(a.hi);
    double y = a.hi * x;                      // first approximation of sqrt(a)
    dd yy = two_prod(y, y);
    double corr = ((a - yy).hi) * (x * 0.5);  // one Newton correction (Karp)
    return two_sum(y, corr);
}

struct cdd {
    dd re, im;
    cdd() {}
    cdd(dd r) : re(r), im(0.0) {}
    cdd(dd r, dd i) : re(r), im(i) {}
    cdd(double r) : re(r), im(0.0) {}
};
inline cdd operator+(cdd a, cdd b) { return cdd(a.re + b.re, a.im + b.im); }
inline cdd operator-(cdd a, cdd b) { return cdd(a.re - b.re, a.im - b.im); }
inline cdd operator-(cdd a) { return cdd(-a.re, -a.im); }
inline cdd operator*(cdd a, cdd b) { return cdd(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
inline cdd operator*(cdd a, dd s) { return cdd(a.re * s, a.im * s); }
inline cdd conj(cdd a) { return cdd(a.re, -a.im); }
inline dd norm2(cdd a) { return a.re * a.re + a.im * a.im; }
inline dd cabs(cdd a) { return dsqrt(norm2(a)); }
inline cdd operator/(cdd a, cdd b) {
    dd d = norm2(b);
    cdd n = a * conj(b);
    return cdd(n.re / d, n.im / d);
}
inline cdd& operator+=(cdd& a, cdd b) { a = a + b; return a; }
inline cdd& operator-=(cdd& a, cdd b) { a = a - b; return a; }
inline cdd& operator*=(cdd& a, cdd b) { a = a * b; return a; }

}  // namespace rexi
