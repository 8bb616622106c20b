"""Long-horizon behaviour (Sec. 3.4) on the GPU: 10^4 REXI steps of the 1D
harmonic oscillator, against the exact propagator exp(-i n dt H) (dense
eigendecomposition of the 256-point H).

|r(i w)| <= 1 + ||e|| on the interval, so without stabilisation the norm may
grow by up to n (||e|| + solve error); with the weights scaled by (1 - eps),
eps slightly above ||e||, |r| <= 1 and only the solve error can raise the
norm.  The error against the exact evolution grows at most linearly,
~ n (||e|| + solve error) over these n (the (1 + 1e-9)^n growth of Sec. 3.4 is
indistinguishable from linear for n << 1e9).
"""

import numpy as np
import pytest

import workloads as wl
from oracle import operator as op
from oracle import plan as oplan

from _common import library_plan, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STEPS = 10000
EVERY = 1000


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


def _approx_error(lp):
    sigma, beta = lp.fcf()
    R1 = lp.info()["R1"]
    w = 1j * np.linspace(-R1, R1, 40001)
    r = (beta[None, :] / (w[:, None] - sigma[None, :])).sum(1)
    return float(np.max(np.abs(r - np.exp(w))))


def _run(lp, psi0, lam, Q, dt):
    cur = to_dev(psi0)
    nxt = torch.empty_like(cur)
    c0 = Q.T @ psi0
    rec = []
    for n in range(1, STEPS + 1):
        lp.step(cur, out=nxt)
        cur, nxt = nxt, cur
        if n % EVERY == 0:
            psi = cur.cpu().numpy()
            exact = Q @ (np.exp(-1j * n * dt * lam) * c0)
            rec.append((n, np.linalg.norm(psi) / np.linalg.norm(psi0),
                        np.linalg.norm(psi - exact) / np.linalg.norm(exact)))
    assert lp.last_status() == 0
    return rec


def test_ten_thousand_steps_norm_drift_and_error():
    cfg = wl.config_1d_harmonic()
    g, V, psi0 = cfg["grid"], cfg["V"], cfg["psi0"]
    dt, K, R1, tol = 0.2, 16, 24.0, 1e-13
    h = oplan.grid_spacing(g["n"], g["lo"], g["hi"])
    lam, Q = np.linalg.eigh(op.dense_H(V, h))
    plain = library_plan(g, V, dt, K, R1, precision="fp64", tol=tol, window=2, restart=64)
    e = _approx_error(plain)
    A = plain.info()["amplification"]
    stab = library_plan(g, V, dt, K, R1, precision="fp64", tol=tol, window=2, restart=64,
                        stabilize_eps=1.01 * e)
    ns = plain.info()["n_sub"]
    r_plain = _run(plain, psi0, lam, Q, dt)
    r_stab = _run(stab, psi0, lam, Q, dt)
    per_sub = e + 2.0 * A * tol                             # approximation + solve error per rational step
    for (n, nrm, err), (_, nrm_s, err_s) in zip(r_plain, r_stab):
        bound = n * ns * per_sub
        assert abs(nrm - 1.0) <= bound, (n, nrm, bound)
        assert err <= bound, (n, err, bound)
        assert nrm_s <= 1.0 + n * ns * 2.0 * A * tol + 1e-12, (n, nrm_s)   # no growth from the approximant
        assert err_s <= n * ns * (2.02 * e + 2.0 * A * tol), (n, err_s)
    n, nrm, err = r_plain[-1]
    _, nrm_s, err_s = r_stab[-1]
    print("\n%d steps (n_sub %d, ||e|| %.2e, A %.2e): plain |norm-1| %.2e err %.2e; stabilised norm-1 %.2e err %.2e"
          % (n, ns, e, A, abs(nrm - 1.0), err, nrm_s - 1.0, err_s))
