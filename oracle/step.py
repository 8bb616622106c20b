"""REXI step, adjoint step and gradient of the oracle, complex FP64.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

* ``substep``: one rational evaluation, Eq. (5) in the form
  psi' = alpha_0 psi + sum_k alpha_k (tau H - z_k I)^{-1} psi,
  each system solved independently by GMRES (Sec. 3.1: the K solves are
  independent tasks) and summed in FP64.
* ``step``: n_sub substeps (Eq. (10) after centring, see ``oracle.plan``).
* ``substep_adjoint``: vector-Jacobian product of ``substep`` (derived from
  Eq. (5); the paper has no adjoint).  H is real symmetric, so
  (tau H - z_k I)^H = tau H - conj(z_k) I.  For a real loss L and
  G = 2 dL/dconj(psi') (the gradient convention of torch.autograd):
      grad_psi = conj(alpha_0) G + sum_k conj(alpha_k) Y_k,
      Y_k = (tau H - conj(z_k) I)^{-1} G,
      dL/dV_i += -tau Re sum_k alpha_k conj(Y_{k,i}) X_{k,i},
      X_k = (tau H - z_k I)^{-1} psi.
* Dense references for tiny grids: direct solves and exp(-i dt H / hbar) by
  the symmetric eigendecomposition (f(G) = X f(Omega) X^{-1}, Sec. 3.1).
"""

from __future__ import annotations

import numpy as np

from . import gmres as _gmres
from . import operator as _op


def solve_pole(V, h, psi, tau, z, hbar=1.0, mass=1.0, tol=1e-13, m=30, max_iters=5000):
    """x = (tau H - z I)^{-1} psi by GMRES(m)."""
    A = lambda v: _op.apply_shifted(v, V, h, tau, z, hbar, mass)
    return _gmres.gmres(A, psi, tol=tol, m=m, max_iters=max_iters)


def substep(V, h, psi, tau, z, alpha, alpha0=0.0, hbar=1.0, mass=1.0,
            tol=1e-13, m=30, max_iters=5000, return_solutions=False):
    """One rational evaluation of Eq. (5)."""
    psi = np.asarray(psi, dtype=np.complex128)
    out = alpha0 * psi
    xs, infos = [], []
    for zk, ak in zip(z, alpha):
        x, info = solve_pole(V, h, psi, tau, zk, hbar, mass, tol, m, max_iters)
        out = out + ak * x
        xs.append(x)
        infos.append(info)
    if return_solutions:
        return out, xs, infos
    return out, infos


def step(V, h, psi, tau, n_sub, z, alpha, alpha0=0.0, hbar=1.0, mass=1.0,
         tol=1e-13, m=30, max_iters=5000):
    """One user step dt = n_sub * tau."""
    infos = []
    for _ in range(n_sub):
        psi, inf = substep(V, h, psi, tau, z, alpha, alpha0, hbar, mass, tol, m, max_iters)
        infos.append(inf)
    return psi, infos


def substep_adjoint(V, h, psi, G, tau, z, alpha, alpha0=0.0, hbar=1.0, mass=1.0,
                    tol=1e-13, m=30, max_iters=5000):
    """(grad_psi, dLdV) of one substep applied to ``psi``, given G at its output."""
    G = np.asarray(G, dtype=np.complex128)
    grad_psi = np.conj(alpha0) * G
    dV = np.zeros(np.shape(V))
    for zk, ak in zip(z, alpha):
        X, _ = solve_pole(V, h, psi, tau, zk, hbar, mass, tol, m, max_iters)
        Y, _ = solve_pole(V, h, G, tau, np.conj(zk), hbar, mass, tol, m, max_iters)
        grad_psi = grad_psi + np.conj(ak) * Y
        dV += -tau * np.real(ak * np.conj(Y) * X)
    return grad_psi, dV


def evolve(V, h, psi0, tau, n_sub, nsteps, z, alpha, alpha0=0.0, hbar=1.0, mass=1.0,
           tol=1e-13, m=30, max_iters=5000):
    """nsteps user steps; returns the list of states after every substep,
    starting with psi0 (the checkpoints the adjoint needs)."""
    states = [np.asarray(psi0, dtype=np.complex128)]
    for _ in range(nsteps * n_sub):
        nxt, _ = substep(V, h, states[-1], tau, z, alpha, alpha0, hbar, mass, tol, m, max_iters)
        states.append(nxt)
    return states


def loss_and_grad(V, h, psi0, target, tau, n_sub, nsteps, z, alpha, alpha0=0.0,
                  hbar=1.0, mass=1.0, tol=1e-13, m=30, max_iters=5000):
    """L = sum |psi(T) - target|^2 and dL/dV by the adjoint recursion."""
    states = evolve(V, h, psi0, tau, n_sub, nsteps, z, alpha, alpha0, hbar, mass, tol, m, max_iters)
    diff = states[-1] - target
    L = float(np.sum(np.abs(diff) ** 2))
    G = 2.0 * diff
    dV = np.zeros(np.shape(V))
    for s in range(len(states) - 2, -1, -1):
        G, dvs = substep_adjoint(V, h, states[s], G, tau, z, alpha, alpha0, hbar, mass, tol, m, max_iters)
        dV += dvs
    return L, dV, G, states


def direct_substep(V, h, psi, tau, z, alpha, alpha0=0.0, hbar=1.0, mass=1.0):
    """Eq. (5) with dense LU solves instead of GMRES (tiny grids)."""
    Hm = _op.dense_H(V, h, hbar, mass)
    n = Hm.shape[0]
    b = np.asarray(psi, dtype=np.complex128).ravel()
    out = alpha0 * b
    for zk, ak in zip(z, alpha):
        out = out + ak * np.linalg.solve(tau * Hm - zk * np.eye(n), b)
    return out.reshape(np.shape(psi))


def exact_propagator(V, h, psi, dt, hbar=1.0, mass=1.0):
    """exp(-i dt H / hbar) psi by the eigendecomposition of the dense H (Eq. (3))."""
    Hm = _op.dense_H(V, h, hbar, mass)
    lam, Q = np.linalg.eigh(Hm)
    b = np.asarray(psi, dtype=np.complex128).ravel()
    out = Q @ (np.exp(-1j * dt * lam / hbar) * (Q.T @ b))
    return out.reshape(np.shape(psi))
