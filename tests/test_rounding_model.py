"""How rounding in the Krylov recurrence reaches a REXI substep (CPU model, no GPU).

The Lanczos kernel can run its recurrence in double-float pairs (a unit
roundoff about 2^5 larger than FP64's) because that rounding reaches
psi' = alpha_0 psi + Q r(T) e_1 ||psi|| only through Q and T, i.e. through the
combined coefficients sum_k alpha_k y_k, whose magnitudes sum to O(10) -- not
through the individual weights alpha_k, whose cancellation (the pole-sum
amplification A) happens in FP64 on the small matrix T.

This model runs the three-term recurrence of tau H (the oracle's operator and
poles) on a small grid, perturbs every vector it forms by eps times the
magnitude of that vector's terms (the error model of floating-point sums and
products with unit roundoff eps), forms psi' from Q and T as the kernel does,
and checks that psi' moves by O(10) eps -- orders of magnitude below A eps --
for eps from 2^-40 to 2^-24.
"""

import numpy as np

import workloads as wl
from oracle import operator as op
from oracle import step as ostep

from _common import OraclePlan


def _substep(psi, V, h, tau, orc, m, eps, rng):
    def pert(x, scale):
        if eps == 0.0:
            return x
        return x + eps * scale * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))

    def abs_terms(u):
        # sum over the stencil's terms of |coefficient| |u|, per component
        s = np.zeros(u.shape)
        for d in range(u.ndim):
            ax = u.ndim - 1 - d
            s += (np.abs(np.roll(u, -1, axis=ax)) + 2.0 * np.abs(u) + np.abs(np.roll(u, 1, axis=ax))) / h[d] ** 2
        return abs(tau) * (0.5 * s + np.abs(V) * np.abs(u))

    nrm = np.linalg.norm(psi)
    Q = [psi / nrm]
    a, b = [], []
    qprev, bprev = np.zeros_like(psi), 0.0
    for _ in range(m):
        q = Q[-1]
        w = pert(tau * op.apply_H(q, V, h), abs_terms(q.real) + abs_terms(q.imag))
        al = np.vdot(q, w).real * (1.0 + eps * rng.standard_normal())
        r = pert(w - al * q - bprev * qprev, np.abs(w) + abs(al) * np.abs(q) + bprev * np.abs(qprev))
        be = np.linalg.norm(r) * (1.0 + eps * rng.standard_normal())
        a.append(al)
        b.append(be)
        qprev, bprev = q, be
        Q.append(r / be)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    e1 = np.zeros(m, complex)
    e1[0] = nrm
    c = sum(ak * np.linalg.solve(T - zk * np.eye(m), e1) for zk, ak in zip(orc.z, orc.alpha))
    out = orc.alpha0 * psi + np.tensordot(c, np.array(Q[:m]), axes=(0, 0))
    return out, c


def test_recurrence_rounding_enters_through_the_combined_coefficients():
    g, V, psi = wl.random_problem(31, (48, 40), box=8.0)
    K, R1, dt = 16, 24.0, 0.5
    orc = OraclePlan(g, V, dt, K, R1)
    h, tau = orc.h, orc.tau
    m = 60
    rng = np.random.default_rng(5)
    ref, c = _substep(psi, V, h, tau, orc, m, 0.0, rng)
    # the unperturbed model is the rational evaluation the oracle computes
    want, _ = ostep.substep(V, h, psi, tau, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
    floor = np.linalg.norm(ref - want) / np.linalg.norm(want)
    assert floor < 1e-8, floor
    csum = np.abs(c).sum() / np.linalg.norm(psi)
    assert csum < 100.0 and orc.A > 1e5                 # O(10) combined coefficients, A ~ 4.5e5
    # the FP64 evaluation of sum_k alpha_k (T - z_k)^{-1} e_1 on a T that differs
    # in its last digits moves psi' by up to about A u_64 by itself
    fp64_floor = 2.0 * orc.A * 2.0 ** -53
    for eps in (2.0 ** -40, 2.0 ** -32, 2.0 ** -24):
        worst = 0.0
        for seed in (1, 2):
            out, _ = _substep(psi, V, h, tau, orc, m, eps, np.random.default_rng(seed))
            worst = max(worst, np.linalg.norm(out - ref) / np.linalg.norm(ref))
        # the effect scales with the combined coefficients, far below what A eps
        # would allow
        assert worst < 20.0 * csum * eps + fp64_floor, (eps, worst, csum)
        assert worst < 1e-3 * orc.A * eps + fp64_floor, (eps, worst, orc.A)
