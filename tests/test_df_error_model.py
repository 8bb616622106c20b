"""Error model of the double-float arithmetic the Lanczos recurrence uses (CPU).

The kernel forms every result of the double-float recurrence the same way: the
leading parts of its terms summed by Knuth's two-sum (exact), products by
Dekker's method with a fused multiply-add (exact up to the lo*lo term), the
trailing parts and the rounding errors summed in FP32, one renormalisation.
The claim the design rests on: each result is within a few 2^-48 of the
magnitude of its largest term.  This test restates those steps in float32
(numpy, round to nearest, a fused multiply-add emulated exactly through
float64, which holds the product of two floats exactly) and measures the error
against exact rational arithmetic on random stencil-like and update-like
sums, including heavy cancellation.
"""

from fractions import Fraction

import numpy as np

F = np.float32


def f32(x):
    return F(x)


def fma32(a, b, c):
    # a*b is exact in float64 (24 + 24 bits); the sum then rounds once to float32
    # unless float64 already rounded it, which the exact check below rules out
    p = np.float64(a) * np.float64(b)
    s = p + np.float64(c)
    if Fraction(s) != Fraction(p) + Fraction(float(c)):
        # fall back to an exactly rounded result through fractions
        return F(float(Fraction(p) + Fraction(float(c))))
    return F(s)


def two_sum_acc(s, t, x):
    r = f32(s + x)
    z = f32(r - s)
    e = f32(f32(s - f32(r - z)) + f32(x - z))
    return r, f32(t + e)


def mul_acc(s, t, ah, al, bh, bl):
    p = f32(ah * bh)
    e = fma32(ah, bh, -p)
    e = fma32(ah, bl, e)
    e = fma32(al, bh, e)
    s, t = two_sum_acc(s, t, p)
    return s, f32(t + e)


def norm(s, t):
    h = f32(s + t)
    return h, f32(t - f32(h - s))


def split(x):
    h = F(x)
    return h, F(x - float(h))


def exact(*pairs_and_coefs):
    return sum(Fraction(float(c)) * (Fraction(float(h)) + Fraction(float(l))) for c, (h, l) in pairs_and_coefs)


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = F(rng.normal() * 10 ** rng.uniform(-5, 5)), F(rng.normal() * 10 ** rng.uniform(-5, 5))
        r, e = two_sum_acc(a, F(0.0), b)
        assert Fraction(float(r)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))


def test_stencil_result_within_a_few_2pow48_of_its_largest_term():
    # w = d c - (l + r + u + v): the shape of phase B with unit neighbour
    # weights, on smooth data (heavy cancellation) and on random data
    rng = np.random.default_rng(2)
    worst = 0.0
    for trial in range(1500):
        base = rng.normal()
        smooth = trial % 2 == 0
        vals = [base + (1e-6 if smooth else 1.0) * rng.normal() for _ in range(5)]
        c, l, r, u, v = (split(x) for x in vals)
        d = split(4.0 + (1e-7 if smooth else 1.0) * rng.normal())
        s, t = F(0.0), F(0.0)
        s, t = mul_acc(s, t, d[0], d[1], c[0], c[1])
        for nb in (l, r, u, v):
            s, t = two_sum_acc(s, t, -nb[0])
            t = f32(t - nb[1])
        wh, wl = norm(s, t)
        ex = (Fraction(float(d[0])) + Fraction(float(d[1]))) * (Fraction(float(c[0])) + Fraction(float(c[1])))
        for nb in (l, r, u, v):
            ex -= Fraction(float(nb[0])) + Fraction(float(nb[1]))
        big = max(abs(float(ex + 0)), *(abs(float(nb[0])) for nb in (l, r, u, v)),
                  abs(float(d[0]) * float(c[0])))
        err = abs(float(Fraction(float(wh)) + Fraction(float(wl)) - ex)) / big
        worst = max(worst, err)
    assert worst < 8 * 2.0 ** -48, worst


def test_update_result_within_a_few_2pow48_of_its_largest_term():
    # v = w - a u1 - b u2: the shape of phase A, the coefficients as pairs
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(1500):
        w, u1, u2 = (split(rng.normal()) for _ in range(3))
        a, b = split(rng.normal()), split(rng.uniform(0.1, 2.0))
        s, t = w
        s, t = mul_acc(s, t, -a[0], -a[1], u1[0], u1[1])
        s, t = mul_acc(s, t, -b[0], -b[1], u2[0], u2[1])
        vh, vl = norm(s, t)
        fr = lambda p: Fraction(float(p[0])) + Fraction(float(p[1]))
        ex = fr(w) - fr(a) * fr(u1) - fr(b) * fr(u2)
        big = max(abs(float(fr(w))), abs(float(fr(a) * fr(u1))), abs(float(fr(b) * fr(u2))))
        err = abs(float(Fraction(float(vh)) + Fraction(float(vl)) - ex)) / big
        worst = max(worst, err)
    assert worst < 8 * 2.0 ** -48, worst
