"""Pins of the oracle's Chebyshev propagator (the comparison method of Sec. 4).

* FFT coefficients == the closed form 2 (-i)^k J_k(R) (Jacobi-Anger expansion
  of exp(-i R cos theta)), a_0 = J_0(R);
* Sec. 4's setting: degree 26 on i[-10, 10] has an error of the order of the
  K = 16 Faber-CF approximant (Table 1: 2.38e-9);
* the truncation rule: max |p(x) - exp(-i R x)| <= tol on [-1, 1];
* Clenshaw == the forward three-term recurrence (a different evaluation);
* the propagator against exp(-i dt H) by dense eigendecomposition on tiny
  1D/2D/3D grids, and on a plane wave (an exact eigenvector) the scalar p.
"""

import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as ch
from oracle import operator as op
from oracle import plan
from oracle import step as ostep

special = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("R", [10.0, 38.9, 77.8])
def test_fft_coefficients_are_bessel(R):
    N = int(R) + 40
    a = ch.coefficients(R, N)
    k = np.arange(N + 1)
    ref = 2.0 * (-1j) ** k * special.jv(k, R)
    ref[0] = special.jv(0, R)
    assert np.max(np.abs(a - ref)) < 1e-14


def _max_err(R, N):
    a = ch.coefficients(R, N)
    x = np.cos(np.linspace(0.0, np.pi, 4001))
    T = np.cos(np.outer(np.arange(N + 1), np.arccos(x)))
    p = a @ T
    return np.max(np.abs(p - np.exp(-1j * R * x)))


def test_paper_degree_26_on_i10():
    err = _max_err(10.0, 26)
    assert 2.38e-9 / 10 < err < 2.38e-9 * 10, err


@pytest.mark.parametrize("R,tol", [(10.0, 1e-10), (38.9, 1e-12), (77.8, 1e-10)])
def test_degree_rule_meets_tolerance(R, tol):
    N = ch.degree(R, tol)
    assert N >= R
    assert _max_err(R, N) <= tol
    assert _max_err(R, N - 3) > tol * 1e-3          # not wildly over-resolved


def test_clenshaw_equals_forward_recurrence():
    g, V, psi = wl.random_problem(5, (24, 20), box=6.0)
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    emin, emax, c, W = plan.spectral_enclosure(V, h, g["hbar"], g["mass"])
    a = ch.coefficients(12.0, 40)
    got = ch.clenshaw(psi, V, h, c, W, a)
    t0, t1 = psi, ch.apply_scaled(psi, V, h, c, W)
    acc = a[0] * t0 + a[1] * t1
    for k in range(2, len(a)):
        t0, t1 = t1, 2.0 * ch.apply_scaled(t1, V, h, c, W) - t0
        acc = acc + a[k] * t1
    assert np.linalg.norm(got - acc) / np.linalg.norm(acc) < 1e-13


@pytest.mark.parametrize("n", [(48,), (8, 7), (5, 4, 4)])
def test_step_matches_dense_exponential(n):
    g, V, psi = wl.random_problem(6, n, box=4.0)
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    emin, emax, _, _ = plan.spectral_enclosure(V, h, g["hbar"], g["mass"])
    dt, tol = 0.3, 1e-11
    out, N = ch.step(psi, V, h, dt, emin, emax, tol=tol)
    ref = ostep.exact_propagator(V, h, psi, dt)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < tol + 1e-12


def test_plane_wave_gives_scalar_polynomial():
    n = (64, 48)
    g = wl.make_grid(n, (-5.0, -4.0), (5.0, 4.0))
    V = np.full(n[::-1], 0.7)
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    X = wl.coords(g)
    m = (3, -2)
    L = (10.0, 8.0)
    wave = np.exp(1j * sum(2 * np.pi * m[d] * (X[d] - g["lo"][d]) / L[d] for d in range(2)))
    lam = 0.7 + 0.5 * sum((2 - 2 * np.cos(2 * np.pi * m[d] / n[d])) / h[d] ** 2 for d in range(2))
    emin, emax, c, W = plan.spectral_enclosure(V, h, g["hbar"], g["mass"])
    dt = 0.05
    out, N = ch.step(wave, V, h, dt, emin, emax, tol=1e-12)
    R = dt * W
    a = ch.coefficients(R, N) * np.exp(-1j * dt * c)
    xt = (lam - c) / W
    p = np.sum(a * np.cos(np.arange(N + 1) * np.arccos(xt)))
    assert np.linalg.norm(out - p * wave) / np.linalg.norm(wave) < 1e-12
    assert abs(p - np.exp(-1j * dt * lam)) < 1e-11
