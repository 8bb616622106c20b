"""Chebyshev propagator of the oracle (the comparison method of Sec. 4).

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

Sec. 4 approximates exp(z) on -i[-R, R] by p(z) = sum_{k<=N} a_k T_k(-i z / R),
computes the coefficients with the FFT and applies p(tau M) u_0 with the
Clenshaw algorithm.  For the Schroedinger operator M = -i H / hbar (B = hbar I)
and the centring of ``oracle.plan`` (H - c has its spectrum in [-W, W]):

    exp(-i dt H / hbar) = exp(-i dt c / hbar) exp(-i R Ht),   Ht = (H - c) / W,
    R = dt W / hbar,

and exp(-i R x) = sum_k a_k T_k(x) on x in [-1, 1].  The a_k are the Chebyshev
coefficients of f(x) = exp(-i R x): with x = cos(theta),
a_k = (2 - delta_k0) / pi * int_0^pi f(cos theta) cos(k theta) d theta, which
the FFT (trapezoid rule on a uniform theta grid) evaluates to machine
precision once the grid resolves the coefficients' decay.

Clenshaw: b_{N+1} = b_{N+2} = 0, b_k = a_k u + 2 Ht b_{k+1} - b_{k+2}
(k = N .. 1), p(Ht) u = a_0 u + Ht b_1 - b_2.
"""

from __future__ import annotations

import numpy as np

from . import operator as _op


def coefficients(R, N, M=None):
    """a_0 .. a_N of exp(-i R x) on [-1, 1] by the FFT (trapezoid rule in theta)."""
    if M is None:
        M = 4 * (N + 1) + 64
    theta = np.pi * np.arange(2 * M) / M            # full period, 2M nodes
    f = np.exp(-1j * R * np.cos(theta))
    c = np.fft.fft(f) / (2 * M)                      # c_k = mean of f(cos t) e^{-ik t}
    a = 2.0 * c[:N + 1]
    a[0] = c[0]
    return a


def degree(R, tol):
    """Smallest N >= R with sum_{k > N} |a_k| <= tol (then |p(x) - e^{-iRx}| <= tol on [-1, 1])."""
    Nmax = int(np.ceil(R)) + 200
    a = np.abs(coefficients(R, Nmax, M=4 * Nmax + 64))
    tail = np.cumsum(a[::-1])[::-1]                  # tail[k] = sum_{j >= k} |a_j|
    for N in range(int(np.ceil(R)), Nmax):
        if tail[N + 1] <= tol:
            return N
    raise ValueError("degree above %d" % Nmax)


def apply_scaled(u, V, h, c, W, hbar=1.0, mass=1.0):
    """Ht u = (H - c) u / W."""
    return (_op.apply_H(u, V, h, hbar, mass) - c * u) / W


def clenshaw(u, V, h, c, W, a, hbar=1.0, mass=1.0):
    """p(Ht) u = sum_k a_k T_k(Ht) u by the Clenshaw recurrence."""
    N = len(a) - 1
    b1 = np.zeros_like(u)
    b2 = np.zeros_like(u)
    for k in range(N, 0, -1):
        b0 = a[k] * u + 2.0 * apply_scaled(b1, V, h, c, W, hbar, mass) - b2
        b2, b1 = b1, b0
    return a[0] * u + apply_scaled(b1, V, h, c, W, hbar, mass) - b2


def step(u, V, h, dt, emin, emax, tol=1e-10, hbar=1.0, mass=1.0):
    """One step exp(-i dt H / hbar) u by the Chebyshev expansion on [emin, emax];
    returns (result, degree)."""
    c = 0.5 * (emin + emax)
    W = 0.5 * (emax - emin)
    R = dt * W / hbar
    N = degree(R, tol)
    a = coefficients(R, N) * np.exp(-1j * dt * c / hbar)
    return clenshaw(u, V, h, c, W, a, hbar, mass), N
