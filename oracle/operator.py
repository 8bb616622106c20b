"""Discrete Hamiltonian of the oracle.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

H = -(hbar^2 / 2m) Lap_h + diag(V), Eq. (1) discretised by second-order central
differences on a periodic grid (reading: the paper names finite differences
only as the B = I case of Sec. 5 and gives no order).  Arrays are numpy arrays
of shape (N_z, N_y, N_x) / (N_y, N_x) / (N_x,), x fastest in memory.
"""

from __future__ import annotations

import numpy as np


def laplacian(psi, h):
    """(Lap_h psi)_i = sum_d (psi_{i+e_d} - 2 psi_i + psi_{i-e_d}) / h_d^2, periodic.

    ``h`` is ordered (h_x, h_y, h_z) like the grid; numpy axes are reversed.
    """
    nd = psi.ndim
    out = np.zeros_like(psi)
    for d in range(nd):
        ax = nd - 1 - d
        out += (np.roll(psi, -1, axis=ax) - 2.0 * psi + np.roll(psi, 1, axis=ax)) / (h[d] * h[d])
    return out


def apply_H(psi, V, h, hbar=1.0, mass=1.0):
    """H psi."""
    return -(hbar * hbar / (2.0 * mass)) * laplacian(psi, h) + V * psi


def apply_shifted(psi, V, h, tau, z, hbar=1.0, mass=1.0):
    """(tau H - z I) psi, the matrix of one pole's system in Eq. (5)."""
    return tau * apply_H(psi, V, h, hbar, mass) - z * psi


def dense_H(V, h, hbar=1.0, mass=1.0):
    """H as a dense real symmetric matrix (tiny grids only), built column by
    column from ``apply_H`` on unit vectors."""
    shape = V.shape
    n = V.size
    Hm = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        Hm[:, j] = apply_H(e.reshape(shape), V, h, hbar, mass).ravel()
    return Hm

