"""Sec. 3.4 (stability) beyond the statements pinned with Table 1's approximant:

* stabilised weights: scaling every beta_j by (1 - eps) with eps slightly above
  ||e||_inf makes |r(i w)| <= 1 on the whole approximation interval;
* the domain of absolute stability |r(w)| < 1 covers a box of the left
  half-plane (scan), and |r(i w)| stays within ||e|| of one beyond the interval
  for the default radii;
* the contrast Sec. 3.4 draws with polynomial approximation: the Chebyshev
  polynomial of Sec. 4 (degree 26 on i[-10, 10]) is within its error of one
  on the interval but grows without bound outside it.

Weights are stored in FP64 (as the library uses them); ||e||_inf is measured
on a dense grid of the interval.
"""

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle import tables


def _r(sigma, beta):
    s = np.array([complex(x) for x in sigma])
    b = np.array([complex(x) for x in beta])
    return lambda z: (b[None, :] / (np.atleast_1d(z)[:, None] - s[None, :])).sum(1)


@pytest.mark.parametrize("K,R1", [(16, 10.0), (16, 24.0), (32, 68.0)])
def test_stabilised_weights_bound_r_by_one(K, R1):
    sigma, beta, _ = tables.poles(K, R1)
    r = _r(sigma, beta)
    w = 1j * np.linspace(-R1, R1, 40001)
    rw = r(w)
    e = np.max(np.abs(rw - np.exp(w)))
    assert np.max(np.abs(rw)) > 1.0                       # unstabilised: |r| exceeds one on the interval
    eps = 1.01 * e
    assert np.max(np.abs((1.0 - eps) * rw)) <= 1.0       # (1 - eps) beta: bounded by one
    # the stabilisation costs at most eps more error
    assert np.max(np.abs((1.0 - eps) * rw - np.exp(w))) <= e + eps + 1e-15


@pytest.mark.parametrize("K,R1", [(16, 10.0), (16, 24.0), (32, 68.0)])
def test_stability_domain_scan(K, R1):
    sigma, beta, _ = tables.poles(K, R1)
    r = _r(sigma, beta)
    X, Y = np.meshgrid(np.linspace(-30.0, -0.5, 120), np.linspace(-2 * R1, 2 * R1, 240))
    Z = (X + 1j * Y).ravel()
    assert np.max(np.abs(r(Z))) < 1.0                   # the left half-plane box is stable
    w = 1j * np.linspace(-R1, R1, 40001)
    e = np.max(np.abs(r(w) - np.exp(w)))
    beyond = 1j * np.concatenate([np.linspace(R1, 6 * R1, 4000), -np.linspace(R1, 6 * R1, 4000)])
    assert np.max(np.abs(r(beyond))) <= 1.0 + e        # beyond the interval within ||e|| of one
    far = 1j * np.array([20.0, 50.0, 200.0]) * R1
    assert np.all(np.abs(r(far)) < 0.5)                # and decaying (strictly proper)


def test_chebyshev_polynomial_unstable_outside_interval():
    R, N = 10.0, 26
    a = ch.coefficients(R, N)
    k = np.arange(N + 1)
    x = np.linspace(-1.0, 1.0, 20001)
    p_in = a @ np.cos(np.outer(k, np.arccos(x)))
    e = np.max(np.abs(p_in - np.exp(-1j * R * x)))
    assert np.max(np.abs(p_in)) - 1.0 <= e * 1.0001     # on the interval: like the rational case
    # outside: T_k(x) = cosh(k arccosh x) grows like (x + sqrt(x^2 - 1))^k
    for xo, lo in ((1.5, 10.0), (2.0, 1e4), (3.0, 1e9)):
        p_out = np.sum(a * np.cosh(k * np.arccosh(xo)))
        assert abs(p_out) > lo
