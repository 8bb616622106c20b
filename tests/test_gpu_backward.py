"""GPU parity of the adjoint step (rexi_step_backward) and the autograd wrapper.

* dot-product test <phi, S psi> = <S^H phi, psi> on the GPU;
* grad_in and dL/dV of one step against the oracle's adjoint substeps;
* dL/dV of a multi-step loss through RexiEvolve against the oracle's adjoint
  recursion (which is itself pinned to finite differences on the CPU).
"""

import numpy as np
import pytest

import workloads as wl
from oracle import step as ostep

from _common import OraclePlan, library_plan, relerr, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


@pytest.mark.parametrize("precision,K,R1", [("fp64", 8, 8.0), ("mixed", 16, 24.0)])
def test_adjoint_dot_product(precision, K, R1):
    g, V, psi = wl.random_problem(60, (70, 64), box=8.0)
    rng = np.random.default_rng(3)
    phi = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    tol = 1e-13
    lp = library_plan(g, V, 0.6, K, R1, precision=precision, tol=tol)
    spsi = lp.step(to_dev(psi)).cpu().numpy()
    dV = torch.zeros(psi.size, dtype=torch.float64, device="cuda")
    shphi = lp.step_backward(to_dev(psi), to_dev(phi), dV).cpu().numpy()
    lhs = np.vdot(phi, spsi)
    rhs = np.vdot(shphi, psi)
    A = lp.info()["amplification"]
    # forward and adjoint solves are independent, each to relative residual tol
    assert abs(lhs - rhs) / abs(lhs) < max(1e-9, 2.0 * A * tol * lp.info()["n_sub"])


@pytest.mark.parametrize("precision,K,R1", [("fp64", 8, 8.0), ("mixed", 16, 24.0)])
def test_backward_matches_oracle(precision, K, R1):
    g, V, psi = wl.random_problem(61, (48, 40), box=8.0)
    rng = np.random.default_rng(4)
    G = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    dt = 0.5
    tol = 1e-13
    lp = library_plan(g, V, dt, K, R1, precision=precision, tol=tol)
    orc = OraclePlan(g, V, dt, K, R1)
    # oracle: states of the substeps, then adjoint substeps in reverse
    states = [psi]
    for _ in range(orc.n_sub - 1):
        states.append(ostep.substep(V, orc.h, states[-1], orc.tau, orc.z, orc.alpha, orc.alpha0, tol=1e-14)[0])
    Go = G.copy()
    dVo = np.zeros(V.shape)
    for s in range(orc.n_sub - 1, -1, -1):
        Go, dv = ostep.substep_adjoint(V, orc.h, states[s], Go, orc.tau, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
        dVo += dv
    dV = torch.zeros(psi.size, dtype=torch.float64, device="cuda")
    gin, st = lp.step_backward(to_dev(psi), to_dev(G), dV, stats=True)
    assert st["status"] == 0
    A = orc.A
    bound = max(1e-9 if precision == "fp64" else 1e-6, 2.0 * A * tol * orc.n_sub)
    assert relerr(gin.cpu().numpy(), Go) < bound
    assert relerr(dV.cpu().numpy().reshape(V.shape), dVo) < bound * 10


def test_autograd_gradient_matches_oracle():
    n = (40, 32)
    g, V, psi = wl.random_problem(62, n, box=8.0)
    _, _, target = wl.random_problem(63, n, box=8.0)
    K, R1, dt, nsteps = 16, 24.0, 0.4, 3
    from paper_1912_03312_gb300 import RexiEvolve
    lp = library_plan(g, V, dt, K, R1, precision="fp64", tol=1e-13)
    Vt = torch.tensor(V, dtype=torch.float64, device="cuda", requires_grad=True)
    psiT = RexiEvolve.apply(Vt, to_dev(psi), lp, nsteps)
    loss = (psiT - to_dev(target)).abs().pow(2).sum()
    loss.backward()
    orc = OraclePlan(g, V, dt, K, R1)
    L, dVo, _, _ = ostep.loss_and_grad(V, orc.h, psi, target, orc.tau, orc.n_sub, nsteps, orc.z, orc.alpha,
                                       orc.alpha0, tol=1e-14)
    assert abs(float(loss) - L) / L < 1e-8
    assert relerr(Vt.grad.cpu().numpy(), dVo) < max(1e-7, orc.A * 1e-13)
