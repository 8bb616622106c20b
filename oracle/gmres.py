"""Restarted GMRES(m) of the oracle, complex FP64.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

The paper solves the shifted systems of Eq. (5) with GMRES (Sec. 4.2, the
double-slit runs) without giving its parameters.  This is the textbook
algorithm of Saad & Schultz (1986): Arnoldi with modified Gram-Schmidt,
complex Givens rotations on the Hessenberg matrix, least squares by back
substitution at the end of each cycle.  Readings: x_0 = 0, restart length m,
stop when the true relative residual ||b - A x|| / ||b|| <= tol (checked at
every restart; inside a cycle the Givens estimate |g_{j+1}| decides when the
cycle ends early).
"""

from __future__ import annotations

import numpy as np


def gmres(apply_A, b, tol=1e-13, m=30, max_iters=5000):
    """Solve A x = b.  Returns (x, info) with info = dict(iters, cycles,
    relres, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    shape = b.shape
    bf = b.ravel()
    n = bf.size
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(bf)
    info = {"iters": 0, "cycles": 0, "relres": 0.0, "converged": True}
    if bnorm == 0.0:
        return x.reshape(shape), info
    total = 0
    while True:
        r = bf - apply_A(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        info["relres"] = beta / bnorm
        if beta <= tol * bnorm:
            info["converged"] = True
            break
        if total >= max_iters:
            info["converged"] = False
            break
        info["cycles"] += 1
        Vb = np.zeros((m + 1, n), dtype=np.complex128)
        Hh = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        Vb[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            w = apply_A(Vb[j].reshape(shape)).ravel()
            for i in range(j + 1):                      # modified Gram-Schmidt
                Hh[i, j] = np.vdot(Vb[i], w)
                w = w - Hh[i, j] * Vb[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                          # previous rotations
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -np.conj(sn[i]) * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            a = Hh[j, j]
            bb = Hh[j + 1, j]
            rr = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / rr
                sn[j] = (a / abs(a)) * np.conj(bb) / rr
            Hh[j, j] = cs[j] * a + sn[j] * bb
            Hh[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k = j + 1
            breakdown = abs(bb) == 0.0
            if abs(g[j + 1]) <= tol * bnorm or breakdown or total >= max_iters:
                break
            Vb[j + 1] = w / bb
        y = np.zeros(k, dtype=np.complex128)             # back substitution R y = g
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(Hh[i, i + 1:k], y[i + 1:k])) / Hh[i, i]
        x = x + y @ Vb[:k]
    info["iters"] = total
    return x.reshape(shape), info
