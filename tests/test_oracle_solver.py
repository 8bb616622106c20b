"""Pins of the oracle's operator, GMRES, REXI step and adjoint.

Each check compares the oracle with something other than itself:
* plane waves e^{i k.x} are exact eigenvectors of the periodic second-order
  Laplacian, eigenvalue (hbar^2/2m) sum_d (2 - 2 cos(k_d h_d)) / h_d^2 + V0;
* GMRES against numpy.linalg.solve on the dense shifted matrix;
* the REXI step against scipy.linalg.expm of the dense -i dt H / hbar
  (Proposition 1 with cond(X) = 1 for the symmetric H);
* a plane-wave step equals the scalar r(-i tau (lambda - c)) e^{-i tau c} of
  Eq. (4)-(5), evaluated here directly from (sigma, beta);
* norm conservation within the approximation error (Sec. 3.4);
* adjoint: <phi, S psi> = <S^H phi, psi>; dL/dV against central differences.
"""

import numpy as np
import pytest

import workloads as wl
from oracle import operator as op
from oracle import plan, step, tables
from oracle.gmres import gmres


def eig_plane_wave(modes, n, h, V0):
    lam = V0
    for m, N, hd in zip(modes, n, h):
        k = 2 * np.pi * m / (N * hd)
        lam += 0.5 * (2 - 2 * np.cos(k * hd)) / hd ** 2
    return lam


def plane_wave(g, modes):
    X = wl.coords(g)
    ph = np.zeros(X[0].shape)
    for d, m in enumerate(modes):
        L = g["hi"][d] - g["lo"][d]
        ph = ph + 2 * np.pi * m * (X[d] - g["lo"][d]) / L
    return np.exp(1j * ph)


@pytest.mark.parametrize("n,modes", [((16,), (3,)), ((7,), (2,)), ((1,), (0,)), ((2,), (1,)),
                                     ((8, 6), (1, -2)), ((5, 4, 3), (2, 1, 1)), ((4, 1, 2), (1, 0, 1))])
def test_plane_wave_eigenvectors(n, modes):
    g = wl.make_grid(n, [-3.0] * len(n), [4.0] * len(n))
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    V0 = 0.7
    V = np.full(tuple(reversed(n)), V0)
    psi = plane_wave(g, modes)
    Hpsi = op.apply_H(psi, V, h)
    lam = eig_plane_wave(modes, n, h, V0)
    assert np.max(np.abs(Hpsi - lam * psi)) < 1e-11 * max(1.0, abs(lam))


def test_dense_H_symmetric_and_enclosed():
    g, V, _ = wl.random_problem(3, (6, 5))
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    Hm = op.dense_H(V, h)
    assert np.allclose(Hm, Hm.T, atol=1e-13)
    lam = np.linalg.eigvalsh(Hm)
    emin, emax, c, W = plan.spectral_enclosure(V, h)
    assert lam.min() >= emin - 1e-10 and lam.max() <= emax + 1e-10
    # with constant V and even N the checkerboard mode attains E_max exactly
    g2 = wl.make_grid((6, 4), (0.0, 0.0), (3.0, 2.0))
    h2 = plan.grid_spacing(g2["n"], g2["lo"], g2["hi"])
    V2 = np.full((4, 6), -1.5)
    lam2 = np.linalg.eigvalsh(op.dense_H(V2, h2))
    assert abs(lam2.max() - plan.spectral_enclosure(V2, h2)[1]) < 1e-10


def test_substep_rule():
    for dt, W, R1 in [(1.0, 140.96, 24.0), (0.5, 155.6, 64.0), (0.1, 10.0, 24.0), (2.0, 12.0, 24.0)]:
        ns = plan.substeps(dt, W, R1)
        assert (dt / ns) * W <= R1 * (1 + 1e-12)
        assert ns == 1 or (dt / (ns - 1)) * W > R1


def test_gmres_matches_dense_solve():
    g, V, psi = wl.random_problem(7, (10, 9))
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    Hm = op.dense_H(V, h)
    tau, z = 0.4, 1.0 + 0.5j
    A = lambda v: op.apply_shifted(v, V, h, tau, z)
    x, info = gmres(A, psi, tol=1e-13, m=5)
    ref = np.linalg.solve(tau * Hm - z * np.eye(Hm.shape[0]), psi.ravel())
    assert info["converged"] and info["cycles"] > 1
    assert np.linalg.norm(x.ravel() - ref) / np.linalg.norm(ref) < 1e-11


def test_gmres_zero_rhs():
    x, info = gmres(lambda v: 2.0 * v, np.zeros(5, dtype=complex))
    assert info["iters"] == 0 and np.all(x == 0)


def _plan_for(g, V, dt, K, R1):
    h = plan.grid_spacing(g["n"], g["lo"], g["hi"])
    emin, emax, c, W = plan.spectral_enclosure(V, h)
    ns = plan.substeps(dt, W, R1)
    tau = dt / ns
    sig, bet, _ = tables.poles(K, R1)
    z, alpha, a0 = plan.physical_poles(sig, bet, tau, c)
    return h, tau, ns, z, alpha, a0, c, sig, bet


@pytest.mark.parametrize("n", [(24,), (6, 5), (4, 3, 4)])
def test_step_matches_dense_exponential(n):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    g, V, psi = wl.random_problem(11, n, box=6.0)
    K, R1, dt = 16, 24.0, 0.4
    h, tau, ns, z, alpha, a0, c, sig, bet = _plan_for(g, V, dt, K, R1)
    out = psi
    for _ in range(ns):
        out, _ = step.substep(V, h, out, tau, z, alpha, a0, tol=1e-14, m=30)
    Hm = op.dense_H(V, h)
    ref = scipy_linalg.expm(-1j * dt * Hm) @ psi.ravel()
    err = np.linalg.norm(out.ravel() - ref) / np.linalg.norm(ref)
    A = plan.amplification(sig, bet, R1)
    # approximation error (2 sigma_{K+1} ~ 8e-10 per substep) plus solve error A*delta
    assert err < ns * 2e-9 + A * 1e-14 * 0.5, (err, A)


def test_direct_and_gmres_substeps_agree():
    g, V, psi = wl.random_problem(5, (8, 7), box=6.0)
    h, tau, ns, z, alpha, a0, *_ = _plan_for(g, V, 0.3, 16, 24.0)
    a, _ = step.substep(V, h, psi, tau, z, alpha, a0, tol=1e-14)
    b = step.direct_substep(V, h, psi, tau, z, alpha, a0)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8


def test_plane_wave_step_is_scalar_rational():
    n = (32, 16)
    g = wl.make_grid(n, (-5.0, -4.0), (5.0, 4.0))
    V0 = 0.4
    V = np.full(tuple(reversed(n)), V0)
    psi = plane_wave(g, (3, -2))
    K, R1, dt = 16, 24.0, 0.05
    h, tau, ns, z, alpha, a0, c, sig, bet = _plan_for(g, V, dt, K, R1)
    out, _ = step.substep(V, h, psi, tau, z, alpha, a0, tol=1e-14)
    lam = eig_plane_wave((3, -2), n, h, V0)
    w = -1j * tau * (lam - c)
    r = np.sum(bet / (w - sig)) * np.exp(-1j * tau * c)
    assert np.max(np.abs(out - r * psi)) < 1e-9
    assert abs(r - np.exp(-1j * tau * lam)) < 2e-9


def test_norm_conservation():
    g, V, psi = wl.random_problem(13, (12, 10), box=6.0)
    h, tau, ns, z, alpha, a0, c, sig, bet = _plan_for(g, V, 0.5, 16, 24.0)
    out = psi
    for _ in range(ns):
        out, _ = step.substep(V, h, out, tau, z, alpha, a0, tol=1e-14)
    drift = abs(np.linalg.norm(out) - np.linalg.norm(psi)) / np.linalg.norm(psi)
    assert drift < ns * 2e-9 + plan.amplification(sig, bet, 24.0) * 1e-14


def test_linearity_and_composition():
    g, V, psi = wl.random_problem(17, (10,), box=5.0)
    _, _, phi = wl.random_problem(18, (10,), box=5.0)
    h, tau, ns, z, alpha, a0, *_ = _plan_for(g, V, 0.1, 16, 24.0)
    s_psi, _ = step.substep(V, h, psi, tau, z, alpha, a0, tol=1e-14)
    s_phi, _ = step.substep(V, h, phi, tau, z, alpha, a0, tol=1e-14)
    s_lin, _ = step.substep(V, h, 2.0 * psi - 1j * phi, tau, z, alpha, a0, tol=1e-14)
    assert np.linalg.norm(s_lin - (2.0 * s_psi - 1j * s_phi)) < 1e-9


def test_adjoint_dot_product():
    g, V, psi = wl.random_problem(19, (9, 8), box=5.0)
    rng = np.random.default_rng(0)
    phi = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    h, tau, ns, z, alpha, a0, *_ = _plan_for(g, V, 0.2, 16, 24.0)
    s_psi, _ = step.substep(V, h, psi, tau, z, alpha, a0, tol=1e-14)
    sh_phi, _ = step.substep_adjoint(V, h, psi, phi, tau, z, alpha, a0, tol=1e-14)
    lhs = np.vdot(phi, s_psi)
    rhs = np.vdot(sh_phi, psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-9


def test_gradient_matches_finite_differences():
    # The finite-difference loss uses dense direct solves so that its noise is
    # at the rounding level; the oracle gradient uses GMRES and the adjoint.
    g, V, psi = wl.random_problem(23, (8, 6), box=5.0)
    _, _, target = wl.random_problem(24, (8, 6), box=5.0)
    K, R1, dt = 16, 24.0, 0.3
    h, tau, ns, z, alpha, a0, *_ = _plan_for(g, V, dt, K, R1)
    L, dV, _, _ = step.loss_and_grad(V, h, psi, target, tau, ns, 2, z, alpha, a0, tol=1e-14)

    def loss(Vp):
        st = psi
        for _ in range(2 * ns):
            st = step.direct_substep(Vp, h, st, tau, z, alpha, a0)
        return np.sum(np.abs(st - target) ** 2)

    assert abs(loss(V) - L) < 1e-8 * L
    # rounding noise of the loss is ~A * 1e-16 ~ 1e-10, truncation is O(eps^2)
    eps = 2e-3
    scale = np.max(np.abs(dV))
    for idx in [(0, 0), (3, 4), (5, 7), (2, 1), (4, 3)]:
        Vp = V.copy(); Vp[idx] += eps
        Vm = V.copy(); Vm[idx] -= eps
        fd = (loss(Vp) - loss(Vm)) / (2 * eps)
        assert abs(fd - dV[idx]) < 1e-5 * scale, (idx, fd, dV[idx], scale)
