"""Plan arithmetic of the oracle: spectral enclosure, substeps, physical poles.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

Follows Sec. 3.1 (Eq. (3)-(5)) and Sec. 3.3 (Eq. (10)) of Rittich & Speck,
arXiv:1912.03312, for the finite-difference discretisation with B = hbar*I
(the B = I case named in Sec. 5):

* M = (iB)^{-1} A = -i H / hbar  (Eq. (3) with A = H, B = hbar I).
* A step u_1 = r(tau M) u_0 = sum_j beta_j (tau M - sigma_j I)^{-1} u_0, Eq. (5).
* Readings (the paper is silent): the spectrum of H is enclosed by
  [min V, max V + (hbar^2/2m) sum_d 4/h_d^2] (exact bound of the periodic
  second-order Laplacian plus a diagonal), and the exponential is centred at
  c = (E_min + E_max)/2:  exp(-i tau H/hbar) = e^{-i tau c/hbar}
  exp(-i tau (H - c)/hbar).  With half-width W, Eq. (10) becomes
  tau W / hbar <= R1, met by n_sub = ceil(dt W / (hbar R1)) substeps of
  tau = dt / n_sub.
* Expanding (tau M' - sigma_j)^{-1} with M' = -i (H - c)/hbar gives
  i hbar (tau H - z_j I)^{-1} with z_j = tau c + i hbar sigma_j, so
  psi' = alpha_0 psi + sum_j alpha_j (tau H - z_j I)^{-1} psi with
  alpha_j = i hbar beta_j e^{-i tau c / hbar} and alpha_0 = 0 (the FCF
  approximant is strictly proper, Eq. (4)).
"""

from __future__ import annotations

import math

import numpy as np


def grid_spacing(n, lo, hi):
    """h_d = (hi_d - lo_d) / N_d for a periodic grid whose points are
    x_j = lo + j h, j = 0..N-1 (the endpoint hi is the periodic image of lo)."""
    return [(float(b) - float(a)) / int(N) for N, a, b in zip(n, lo, hi)]


def spectral_enclosure(V, h, hbar=1.0, mass=1.0):
    """(E_min, E_max, c, W) enclosing the spectrum of H = -(hbar^2/2m) Lap_h + diag(V)."""
    V = np.asarray(V, dtype=np.float64)
    kin = hbar * hbar / (2.0 * mass) * sum(4.0 / (hd * hd) for hd in h)
    emin = float(V.min())
    emax = float(V.max()) + kin
    c = 0.5 * (emin + emax)
    W = 0.5 * (emax - emin)
    return emin, emax, c, W


def substeps(dt, W, R1, hbar=1.0):
    """Smallest n_sub with (dt/n_sub) W / hbar <= R1 (Eq. (10) after centring)."""
    x = dt * W / (hbar * R1)
    return max(1, int(math.ceil(x - 1e-12 * max(1.0, x))))


def physical_poles(sigma, beta, tau, c, hbar=1.0):
    """Map FCF poles/weights (sigma_j, beta_j) of exp on i[-R1,R1] to the
    (z_j, alpha_j, alpha_0) of psi' = alpha_0 psi + sum alpha_j (tau H - z_j)^{-1} psi."""
    sigma = np.asarray(sigma, dtype=np.complex128)
    beta = np.asarray(beta, dtype=np.complex128)
    phase = np.exp(-1j * tau * c / hbar)
    z = tau * c + 1j * hbar * sigma
    alpha = 1j * hbar * beta * phase
    return z, alpha, 0.0 + 0.0j


def amplification(sigma, beta, R1, samples=4001):
    """A = max over w in i[-R1,R1] of sum_j |beta_j| / |w - sigma_j|: the factor by
    which per-pole solve errors can grow in the pole sum of Eq. (5)."""
    sigma = np.asarray(sigma, dtype=np.complex128)
    beta = np.asarray(beta, dtype=np.complex128)
    w = 1j * np.linspace(-R1, R1, samples)
    return float(np.max(np.sum(np.abs(beta)[None, :] / np.abs(w[:, None] - sigma[None, :]), axis=1)))
