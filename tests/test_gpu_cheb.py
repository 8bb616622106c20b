"""GPU parity of the Chebyshev propagator (rexi_cheb_step, the comparison method
of Sec. 4) against the oracle's Clenshaw evaluation, at small sizes in 1D/2D/3D
and at the benchmark size, plus the plane-wave property on the 3D 128^3 grid,
in-place use, tiny R, and agreement with the REXI step within the two
approximations' errors."""

import numpy as np
import pytest

import workloads as wl
from oracle import chebyshev as och
from oracle import plan as oplan

from _common import library_plan, relerr, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


def _oracle(g, V, psi, dt, N):
    h = oplan.grid_spacing(g["n"], g["lo"], g["hi"])
    emin, emax, c, W = oplan.spectral_enclosure(V, h, g["hbar"], g["mass"])
    R = dt * W / g["hbar"]
    a = och.coefficients(R, N) * np.exp(-1j * dt * c / g["hbar"])
    return och.clenshaw(psi, V, h, c, W, a, g["hbar"], g["mass"]), R


@pytest.mark.parametrize("n,dt", [((300,), 1.0), ((130, 101), 0.5), ((20, 18, 14), 0.3)])
def test_cheb_matches_oracle(n, dt):
    g, V, psi = wl.random_problem(90, n, box=8.0)
    lp = library_plan(g, V, dt, 16, 24.0)
    out, N = lp.cheb_step(to_dev(psi), tol=1e-12)
    ref, R = _oracle(g, V, psi, dt, N)
    assert N >= R
    assert relerr(out.cpu().numpy(), ref) < 1e-12


def test_cheb_full_size_and_against_rexi():
    cfg = wl.config_2d_wells()
    g = cfg["grid"]
    lp = library_plan(g, cfg["V"], cfg["dt"], cfg["K"], 0.0, precision="fp64")
    psi = to_dev(cfg["psi0"])
    out, N = lp.cheb_step(psi, tol=1e-10)
    ref, R = _oracle(g, cfg["V"], cfg["psi0"], cfg["dt"], N)
    assert relerr(out.cpu().numpy(), ref) < 1e-12
    # both approximate exp(-i dt H): Chebyshev to 1e-10, REXI to 2 sigma_{K+1} + A tol
    rexi = lp.step(psi).cpu().numpy()
    assert relerr(out.cpu().numpy(), rexi) < 1e-6


def test_cheb_in_place_tiny_R_and_plane_wave_3d():
    g, V, psi = wl.random_problem(91, (64, 48), box=8.0)
    lp = library_plan(g, V, 1e-4, 8, 8.0)            # R < 1: degree 1
    x = to_dev(psi)
    ref, _ = lp.cheb_step(x, tol=1e-12)
    ref = ref.clone()
    out, N = lp.cheb_step(x, out=x, tol=1e-12)        # in place
    assert N >= 1 and torch.equal(out, ref)
    o2, R = _oracle(g, V, psi, 1e-4, N)
    assert relerr(ref.cpu().numpy(), o2) < 1e-13
    # 3D 128^3 plane wave on a constant potential: p(lambda_t) times the wave
    n = (128, 128, 128)
    g3 = wl.make_grid(n, (-15.0,) * 3, (15.0,) * 3)
    V0 = -0.3
    lw = library_plan(g3, np.full(n, V0), 0.25, 16, 24.0)
    X = wl.coords(g3)
    m = (2, -1, 3)
    wave = np.exp(1j * sum(2 * np.pi * m[d] * (X[d] + 15.0) / 30.0 for d in range(3)))
    ow, N3 = lw.cheb_step(to_dev(wave), tol=1e-12)
    h = 30.0 / 128
    lam = V0 + 0.5 * sum(2 - 2 * np.cos(2 * np.pi * m[d] / 128) for d in range(3)) / h ** 2
    info = lw.info()
    c, W = info["c"], info["W"]
    a = och.coefficients(0.25 * W, N3) * np.exp(-1j * 0.25 * c)
    p = np.sum(a * np.cos(np.arange(N3 + 1) * np.arccos((lam - c) / W)))
    assert relerr(ow.cpu().numpy(), p * wave) < 1e-12
    assert abs(p - np.exp(-1j * 0.25 * lam)) < 1e-11
