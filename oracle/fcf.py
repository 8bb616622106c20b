"""Faber-Caratheodory-Fejer (FCF) poles and weights for exp on i[-R1, R1].

ORACLE -- test infrastructure only.  Nothing on the product path may import
this module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use the oracle.

This is a plain, slow, arbitrary-precision (mpmath) restatement of the
construction of Sec. 3.2 of Rittich & Speck, "Time-parallel simulation of the
Schroedinger equation" (arXiv:1912.03312):

* ``faber_sequence_exp``  -- Algorithm 2, first step ("FaberSequence" of f=exp):
  the Faber coefficients a_n of Eq. (8) for the conformal map of Eq. (9),
  eta(z) = (R1/2)(z - 1/z), computed as the contour integral of Eq. (8) by the
  trapezoid rule on |z| = 1.
* ``cf``                  -- Algorithm 1 (Caratheodory-Fejer approximation of
  the truncated series h(z) = sum_{j<=L} a_j z^j, with n = m+1), built on
  Theorem 1 (Trefethen): Hankel matrix, (n+1)-st singular pair, the error
  formula Eq. (7), outer roots of q, Laurent sequence of q_out * r~*.
* ``faber_cf``            -- Algorithm 2: sigma_j = eta(z_j), the Faber
  sequences b^{(k)} of w -> 1/(w - sigma_k) (again by the trapezoid rule of
  Eq. (8)), the Maclaurin coefficients c_j of r^cf, and the K x K linear system
  for beta.

Readings of garbled or silent passages:

* In Algorithm 1 the polynomial q is v_{L+1} + v_L z + ... + v_1 z^L and p is
  u_1 + u_2 z + ... + u_{L+1} z^L (the printed indices K+1 / k+1 are typos,
  the vectors have L+1 entries).
* The Hankel matrix of Algorithm 1 is real symmetric (the a_j are real), so its
  SVD is taken from the symmetric eigendecomposition: singular values |lambda|,
  v = eigenvector, u = sign(lambda) v.
* The Laurent sequence is taken on a circle of radius rho strictly between the
  largest inner and the smallest outer root of q, with enough trapezoid nodes
  that the aliased tail is below the working precision.
* The last row of the linear system of Algorithm 2 is b_{K-1}^{(K)}.
* The number of outer roots must equal K = n; otherwise the construction is
  rejected (Sec. 3.2.1 says K <= n with equality "for all practical purposes").
"""

from __future__ import annotations

import mpmath as mp

DEFAULT_DPS = 60


def faber_sequence_exp(R1, L, N=None):
    """a_n, n = 0..L, of Eq. (8) for f = exp and eta of Eq. (9).

    The contour integral (1/2 pi i) \\oint_{|z|=1} f(eta(z)) z^{-n-1} dz is
    evaluated with the N-point trapezoid rule on the unit circle (exp is
    entire, so the radius 1 + eps of Eq. (8) may be taken as 1).
    """
    R1 = mp.mpf(R1)
    if N is None:
        N = 4 * (L + 1) + 64
    half = R1 / 2
    vals = []
    for k in range(N):
        w = mp.expjpi(mp.mpf(2 * k) / N)          # e^{2 pi i k / N}
        vals.append(mp.exp(half * (w - 1 / w)))    # f(eta(w))
    a = []
    for n in range(L + 1):
        s = mp.mpc(0)
        for k in range(N):
            s += vals[k] * mp.expjpi(mp.mpf(-2 * k * n) / N)
        a.append(mp.re(s) / N)                     # a_n is real for this eta
    return a


def _poly_eval(coeffs_low_first, z):
    """Horner evaluation of sum_i c_i z^i."""
    acc = mp.mpc(0)
    for c in reversed(coeffs_low_first):
        acc = acc * z + c
    return acc


def cf(a, n, laurent_nodes=None):
    """Algorithm 1 (CF) for the polynomial h(z) = sum_{j=0}^L a_j z^j.

    Returns a dict with the CF error sigma_{n+1} (Theorem 1), the outer roots
    z_1..z_K of q, the numerator coefficients d_0..d_{n-1} of r^cf and the
    coefficients of q_out (lowest degree first).
    """
    L = len(a) - 1
    if n < 1 or n > L:
        raise ValueError("need 1 <= n <= L")
    # Hankel matrix H_{ij} = a_{i+j} (zero below the anti-diagonal), size L+1.
    H = mp.matrix(L + 1, L + 1)
    for i in range(L + 1):
        for j in range(L + 1):
            if i + j <= L:
                H[i, j] = a[i + j]
    # SVD of a real symmetric matrix from its eigendecomposition.
    E, Q = mp.eigsy(H)
    order = sorted(range(L + 1), key=lambda i: -abs(E[i]))
    sing = [abs(E[i]) for i in order]
    idx = order[n]                                   # (n+1)-st singular value
    s = abs(E[idx])
    if n + 1 < len(sing) and abs(sing[n - 1] - sing[n]) <= mp.mpf(10) ** (-mp.mp.dps // 2) * sing[0]:
        raise ArithmeticError("sigma_n == sigma_{n+1}: CF approximant not unique")
    sgn = 1 if E[idx] >= 0 else -1
    v = [Q[i, idx] for i in range(L + 1)]
    u = [sgn * vi for vi in v]
    # p(z) = u_1 + u_2 z + ... + u_{L+1} z^L
    p = list(u)
    # q(z) = v_{L+1} + v_L z + ... + v_1 z^L   (lowest degree first)
    q = [v[L - i] for i in range(L + 1)]

    def rtilde(z):
        # r~*(z) = h(z) - sigma_{n+1} z^L p(z) / q(z)
        return _poly_eval(a, z) - s * z ** L * _poly_eval(p, z) / _poly_eval(q, z)

    # Roots of q (mpmath wants the highest-degree coefficient first).
    roots = mp.polyroots(list(reversed(q)), maxsteps=2000, extraprec=4 * mp.mp.dps)
    outer = sorted([r for r in roots if abs(r) > 1], key=lambda r: (mp.im(r), mp.re(r)))
    inner = [r for r in roots if abs(r) <= 1]
    K = len(outer)
    if K != n:
        raise ArithmeticError("q has %d outer roots, expected %d" % (K, n))

    # q_out(z) = prod (z - z_k), lowest degree first.
    qout = [mp.mpc(1)]
    for zk in outer:
        nxt = [mp.mpc(0)] * (len(qout) + 1)
        for i, c in enumerate(qout):
            nxt[i + 1] += c
            nxt[i] -= zk * c
        qout = nxt

    # Laurent sequence of q_out * r~* on |z| = rho, max|inner| < rho < min|outer|.
    rin = max([abs(r) for r in inner]) if inner else mp.mpf(0)
    rout = min(abs(r) for r in outer)
    rho = mp.sqrt(max(rin, mp.mpf("1e-3")) * rout) if rin > 0 else (1 + rout) / 2
    if laurent_nodes is None:
        ratio = max(rin / rho, rho / rout)
        need = int(mp.ceil((mp.mp.dps + 10) * mp.log(10) / (-mp.log(ratio)))) + 8
        laurent_nodes = max(4 * (L + 1), need)
    N = laurent_nodes
    g = []
    for k in range(N):
        w = rho * mp.expjpi(mp.mpf(2 * k) / N)
        g.append(_poly_eval(qout, w) * rtilde(w))
    d = []
    # d_j for j = 0..n-1 (the terms that r^cf keeps) and a few beyond for checks.
    for j in range(n + 4):
        acc = mp.mpc(0)
        for k in range(N):
            acc += g[k] * mp.expjpi(mp.mpf(-2 * k * j) / N)
        d.append(acc / (N * rho ** j))
    return {
        "sigma": s,
        "singular_values": sing,
        "outer_roots": outer,
        "inner_roots": inner,
        "numerator": d[:n],
        "numerator_tail": d[n:],
        "qout": qout,
        "L": L,
        "n": n,
        "rho": rho,
        "laurent_nodes": N,
    }


def eta(z, R1):
    """Conformal map of Eq. (9): exterior of the unit disc -> exterior of i[-R1, R1]."""
    return mp.mpf(R1) / 2 * (z - 1 / z)


def faber_sequence_resolvent(sigma_k, z_k, R1, J, N=None):
    """b_j^{(k)}, j = 0..J-1: Faber coefficients of w -> 1/(w - sigma_k).

    Eq. (8) with f(w) = 1/(w - sigma_k).  f(eta(z)) is analytic on the annulus
    1/|z_k| < |z| < |z_k| (its poles are z_k and -1/z_k), which contains the
    unit circle, so the trapezoid rule on |z| = 1 converges like |z_k|^{-N}.
    """
    if N is None:
        r = abs(z_k)
        N = int(mp.ceil((mp.mp.dps + 10) * mp.log(10) / mp.log(r))) + J + 8
    vals = []
    for k in range(N):
        w = mp.expjpi(mp.mpf(2 * k) / N)
        vals.append(1 / (eta(w, R1) - sigma_k))
    b = []
    for j in range(J):
        acc = mp.mpc(0)
        for k in range(N):
            acc += vals[k] * mp.expjpi(mp.mpf(-2 * k * j) / N)
        b.append(acc / N)
    return b


def maclaurin(num_low_first, den_low_first, J):
    """First J Maclaurin coefficients of num(z)/den(z) (power-series division)."""
    c = []
    for j in range(J):
        acc = num_low_first[j] if j < len(num_low_first) else mp.mpc(0)
        for i in range(1, min(j, len(den_low_first) - 1) + 1):
            acc -= den_low_first[i] * c[j - i]
        c.append(acc / den_low_first[0])
    return c


def truncation_length(R1, tol_exp=None):
    """Smallest L with |J_j(R1)| below 10^-tol_exp for all j > L (Sec. 3.2.1:
    the Maclaurin series is truncated where the remaining terms are negligible).
    Uses the closed form a_j = J_j(R1) only to pick L; the coefficients
    themselves come from the contour integral."""
    if tol_exp is None:
        tol_exp = mp.mp.dps // 2 + 5
    R1 = mp.mpf(R1)
    L = int(mp.ceil(R1))
    thr = mp.mpf(10) ** (-tol_exp)
    while abs(mp.besselj(L + 1, R1)) > thr or abs(mp.besselj(L + 2, R1)) > thr:
        L += 1
    return L


def faber_cf(R1, K, L=None, dps=DEFAULT_DPS):
    """Algorithm 2 (FaberCF) for f = exp, eta of Eq. (9), n = K.

    Returns (sigma, beta, info): f(w) ~ sum_j beta_j / (w - sigma_j) on
    w in i[-R1, R1], with sigma and beta as lists of mpc.
    """
    with mp.workdps(dps):
        if L is None:
            L = truncation_length(R1)
        a = faber_sequence_exp(R1, L)
        res = cf(a, K)
        zs = res["outer_roots"]
        sig = [eta(z, R1) for z in zs]
        # Faber sequences of the resolvents, one column per pole.
        B = mp.matrix(K, K)
        for k in range(K):
            bk = faber_sequence_resolvent(sig[k], zs[k], R1, K)
            for j in range(K):
                B[j, k] = bk[j]
        c = maclaurin(res["numerator"], res["qout"], K)
        beta_vec = mp.lu_solve(B, mp.matrix(c))
        beta = [beta_vec[k] for k in range(K)]
        info = dict(res)
        info.update({"a": a, "z": zs, "R1": mp.mpf(R1), "K": K})
        return sig, beta, info


def rational_eval(sigma, beta, w):
    """r(w) = sum_j beta_j / (w - sigma_j), Eq. (4), at working precision."""
    acc = mp.mpc(0)
    for s, b in zip(sigma, beta):
        acc += b / (w - s)
    return acc
