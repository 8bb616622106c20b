"""The per-pole stop of the shared-basis Lanczos kernel (CPU, no GPU).

Each pole solves min ||beta e_1 - (T_k - s [I; 0]) y|| by complex Givens
rotations G_i = [c_i s_i; -conj(s_i) c_i] (c_i real) on the shared basis Q,
whose columns have unit norm but are orthogonal only locally.  The residual
is r_k = Q_{k+1} z with z = G_0^H ... G_k^H (g_{k+1} e_{k+1}), so

    ||r_k|| <= ||z||_1 = |g_{k+1}| L_k,  L_k = c_k + |s_k| L_{k-1},  L_{-1} = 1,

and L_k <= sqrt(k+2) (the bound for unit columns without orthogonality).
The kernel stops a pole on |g_{k+1}| L_k <= tol.  These tests check the
identity ||z||_1 = |g| L_k on random rotations, the inequality against the
true residual of a Lanczos basis that has lost orthogonality, and that L_k
stays near c / (1 - |s|) while GMRES converges.
"""

import numpy as np


def _rotation(x, h):
    """G [x; h] = [r; 0] for complex x and real h >= 0 (the kernel's convention)."""
    nu = np.hypot(abs(x), h)
    if h == 0.0:
        return 1.0, 0.0j, x
    if x == 0:
        return 0.0, 1.0 + 0j, h
    ph = x / abs(x)
    return abs(x) / nu, ph * h / nu, ph * nu


def _z_of(cs, ss, g):
    """G_0^H ... G_k^H (g e_{k+1}) for rotations (c_i, s_i) on rows (i, i+1)."""
    k = len(cs)
    z = np.zeros(k + 1, complex)
    z[k] = g
    for i in range(k - 1, -1, -1):
        c, s = cs[i], ss[i]
        a, b = z[i], z[i + 1]
        # G^H = [c -s; conj(s) c] on rows (i, i+1)
        z[i], z[i + 1] = c * a - s * b, np.conj(s) * a + c * b
    return z


def _L(cs, ss):
    L = 1.0
    for c, s in zip(cs, ss):
        L = c + abs(s) * L
    return L


def test_one_norm_identity_on_random_rotations():
    rng = np.random.default_rng(11)
    for k in (1, 2, 5, 17, 60):
        for _ in range(20):
            cs = rng.uniform(0.0, 1.0, k)
            ph = np.exp(2j * np.pi * rng.uniform(size=k))
            ss = ph * np.sqrt(1.0 - cs * cs)
            g = complex(rng.normal(), rng.normal())
            z = _z_of(cs, ss, g)
            L = _L(cs, ss)
            assert np.isclose(np.abs(z).sum(), abs(g) * L, rtol=1e-12)
            assert np.isclose(np.linalg.norm(z), abs(g), rtol=1e-12)      # the rotations are unitary
            assert L <= np.sqrt(k + 1) * (1 + 1e-12)


def test_bound_holds_for_a_lanczos_basis_without_reorthogonalisation():
    # B = tau H (1D periodic Laplacian + potential with three spikes, whose
    # isolated eigenvalues the recurrence finds within ~20 steps: from then on
    # the basis loses orthogonality), a complex shift s as a pole's, the
    # three-term recurrence without reorthogonalisation
    rng = np.random.default_rng(12)
    n, tau = 400, 0.05
    h = 0.1
    V = 4.0 * rng.uniform(size=n)
    V[[50, 170, 300]] += 500.0
    main = 1.0 / h ** 2 + V
    off = -0.5 / h ** 2 * np.ones(n)

    def B(v):
        return tau * (main * v + off * np.roll(v, 1) + off * np.roll(v, -1))

    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    beta0 = np.linalg.norm(b)
    m = 80
    Q = np.zeros((n, m + 1), complex)
    alpha = np.zeros(m)
    betas = np.zeros(m)
    Q[:, 0] = b / beta0
    for j in range(m):
        w = B(Q[:, j])
        alpha[j] = np.vdot(Q[:, j], w).real
        w = w - alpha[j] * Q[:, j] - (betas[j - 1] * Q[:, j - 1] if j else 0)
        betas[j] = np.linalg.norm(w)
        Q[:, j + 1] = w / betas[j]
    loss = np.abs(Q[:, :m].conj().T @ Q[:, :m] - np.eye(m)).max()
    assert loss > 0.1                        # orthogonality is lost
    s = 2.0 + 3.0j                           # a pole's shift (B - s I is nonsingular)
    # Givens QR of the (k+2) x (k+1) matrix T~_k - s [I; 0], column by column
    Tt = np.zeros((m + 1, m), complex)
    for j in range(m):
        Tt[j, j] = alpha[j] - s
        Tt[j + 1, j] = betas[j]
        if j:
            Tt[j - 1, j] = betas[j - 1]
    R = Tt.copy()
    gvec = np.zeros(m + 1, complex)
    gvec[0] = beta0
    cs, ss = [], []
    Ls = []
    for k in range(m):
        for i in range(k):                   # the earlier rotations on the new column
            c, sn = cs[i], ss[i]
            a, d = R[i, k], R[i + 1, k]
            R[i, k], R[i + 1, k] = c * a + sn * d, -np.conj(sn) * a + c * d
        c, sn, r = _rotation(R[k, k], R[k + 1, k].real)
        R[k, k], R[k + 1, k] = r, 0.0
        cs.append(c)
        ss.append(sn)
        gvec[k], gvec[k + 1] = c * gvec[k], -np.conj(sn) * gvec[k]
        L = _L(cs, ss)
        Ls.append(L)
        y = np.linalg.solve(np.triu(R[:k + 1, :k + 1]), gvec[:k + 1])
        x = Q[:, :k + 1] @ y
        true = np.linalg.norm(b - (B(x) - s * x))
        bound = abs(gvec[k + 1]) * L
        # the recurrence's own rounding (a few eps ||B|| per column) is the slack
        assert true <= bound * (1 + 1e-8) + 1e-11 * beta0, (k, true, bound)
        assert bound <= abs(gvec[k + 1]) * np.sqrt(k + 2) * (1 + 1e-12)
        if true < 1e-12 * beta0:
            break
    # while the pole converges L settles far below sqrt(k+2)
    assert Ls[-1] < 0.5 * np.sqrt(len(Ls) + 1)
