"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds input data only -- grids, potentials, wave packets and the
workload definitions -- and none of the REXI method's arithmetic.  Both the
oracle and the CUDA library are fed from here; neither is imported.

The paper's own workloads (FEM meshes of the tunnelling and double-slit runs,
Sec. 4) are not available, so seeded stand-ins with the same kind of content
are used: a periodic grid, a smooth potential and the Gaussian wave packet of
Eq. (12) in Hartree atomic units (hbar = m = 1, Sec. 4).

Arrays are numpy, shape (N_z, N_y, N_x) / (N_y, N_x) / (N_x,), x fastest in
memory; psi is complex128, V is float64.
"""

from __future__ import annotations

import numpy as np


def make_grid(n, lo, hi, hbar=1.0, mass=1.0):
    """Periodic grid description; points x_j = lo + j (hi - lo) / N, j < N."""
    n = tuple(int(v) for v in n)
    return {"ndim": len(n), "n": n, "lo": tuple(float(v) for v in lo),
            "hi": tuple(float(v) for v in hi), "hbar": float(hbar), "mass": float(mass)}


def coords(g):
    """Coordinate arrays (x, y, z order) broadcast to the grid's numpy shape."""
    axes = []
    for N, a, b in zip(g["n"], g["lo"], g["hi"]):
        axes.append(a + (b - a) / N * np.arange(N))
    mesh = np.meshgrid(*reversed(axes), indexing="ij")      # numpy order z, y, x
    return list(reversed(mesh))


def cell_volume(g):
    v = 1.0
    for N, a, b in zip(g["n"], g["lo"], g["hi"]):
        v *= (b - a) / N
    return v


def wave_packet(g, r0, sigma, p0):
    """Gaussian wave packet of Eq. (12) with Sigma = sigma I, normalised so that
    (cell volume) * sum |psi|^2 = 1 (the discrete form of the integral in Sec. 4)."""
    X = coords(g)
    hbar = g["hbar"]
    q = np.zeros(X[0].shape)
    ph = np.zeros(X[0].shape)
    for d in range(g["ndim"]):
        dx = X[d] - r0[d]
        q += dx * dx / sigma
        ph += p0[d] * dx / hbar
    psi = np.exp(-0.5 * q) * np.exp(1j * ph)
    psi /= np.sqrt(cell_volume(g) * np.sum(np.abs(psi) ** 2))
    return psi.astype(np.complex128)


def harmonic(g, omega=1.0):
    X = coords(g)
    return 0.5 * omega * omega * sum(x * x for x in X)


def gaussian_wells(g, rng, count=4, depth=(1.0, 5.0), centre_box=20.0, width=2.0):
    """V = sum_i -D_i exp(-|r - c_i|^2 / (2 w^2)), D_i ~ U[depth], c_i ~ U[-box, box]^d."""
    X = coords(g)
    V = np.zeros(X[0].shape)
    for _ in range(count):
        D = rng.uniform(*depth)
        c = rng.uniform(-centre_box, centre_box, size=g["ndim"])
        r2 = sum((X[d] - c[d]) ** 2 for d in range(g["ndim"]))
        V -= D * np.exp(-r2 / (2.0 * width * width))
    return V


def softened_coulomb(g, soft=0.5):
    X = coords(g)
    return -1.0 / np.sqrt(sum(x * x for x in X) + soft)


FOURIER_MODES_2D = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 0), (0, 2), (1, 2), (2, 1)]


def fourier_field(g, rng, scale=0.5, modes=FOURIER_MODES_2D):
    """Smooth periodic field sum_m a_m cos(k_m.r) + b_m sin(k_m.r), a, b ~ N(0, scale^2)."""
    X = coords(g)
    L = [b - a for a, b in zip(g["lo"], g["hi"])]
    V = np.zeros(X[0].shape)
    for m in modes:
        a, b = rng.normal(0.0, scale, size=2)
        ph = sum(2.0 * np.pi * m[d] * (X[d] - g["lo"][d]) / L[d] for d in range(g["ndim"]))
        V += a * np.cos(ph) + b * np.sin(ph)
    return V


def random_problem(seed, n, box=10.0, potential="wells"):
    """Small random problem for parity tests: grid, V, psi0."""
    rng = np.random.default_rng(seed)
    nd = len(n)
    g = make_grid(n, [-box] * nd, [box] * nd)
    if potential == "wells":
        V = gaussian_wells(g, rng, centre_box=0.6 * box, width=0.15 * box)
    elif potential == "harmonic":
        V = harmonic(g, omega=rng.uniform(0.2, 0.5))
    else:
        V = np.full(tuple(reversed(g["n"])), float(potential))
    r0 = rng.uniform(-0.3 * box, 0.3 * box, size=nd)
    p0 = rng.uniform(-2.0, 2.0, size=nd)
    psi = wave_packet(g, r0, 1.0, p0)
    return g, V, psi


# ---------------------------------------------------------------------------
# Benchmark workloads (the configurations the engine is measured on)
# ---------------------------------------------------------------------------

def config_1d_harmonic():
    """1D, N=256 on [-20, 20), V = x^2/2, packet x0=-5, width 1, k0=2; K=16, one
    step dt=1.0, plain FP64, GMRES tol 1e-12."""
    g = make_grid((256,), (-20.0,), (20.0,))
    return {"name": "1d_harmonic_N256_K16", "grid": g, "V": harmonic(g),
            "psi0": wave_packet(g, (-5.0,), 1.0, (2.0,)), "K": 16, "dt": 1.0, "nsteps": 1,
            "precision": "fp64", "tol": 1e-12}


def config_2d_wells(seed=2):
    """2D 512^2 on [-30, 30)^2, four Gaussian wells (depth U[1,5], centres
    U[-20,20]^2, width 2), packet at (-10, 0), width 1, k0=(3,0); K=32, 20 steps
    of dt=0.5, complex FP32 Krylov + FP64 refinement."""
    rng = np.random.default_rng(seed)
    g = make_grid((512, 512), (-30.0, -30.0), (30.0, 30.0))
    return {"name": "2d_wells_512x512_K32", "grid": g, "V": gaussian_wells(g, rng),
            "psi0": wave_packet(g, (-10.0, 0.0), 1.0, (3.0, 0.0)), "K": 32, "dt": 0.5,
            "nsteps": 20, "precision": "mixed", "tol": 1e-6}


def config_3d_coulomb():
    """3D 128^3 on [-15, 15)^3, V = -1/sqrt(r^2 + 0.5), packet at (3, 0, 0), width
    1, p0 = 0; K=64, 10 steps of dt=0.25, mixed precision, restart 30."""
    g = make_grid((128, 128, 128), (-15.0,) * 3, (15.0,) * 3)
    return {"name": "3d_coulomb_128cube_K64", "grid": g, "V": softened_coulomb(g),
            "psi0": wave_packet(g, (3.0, 0.0, 0.0), 1.0, (0.0, 0.0, 0.0)), "K": 64,
            "dt": 0.25, "nsteps": 10, "precision": "mixed", "tol": 1e-6}


def config_batched(seed=4, count=64, sides=(128, 192, 256, 384)):
    """count independent 2D problems on [-30, 30)^2, N_x and N_y drawn
    independently from ``sides``; Gaussian-well potentials, packets with random
    centre in [-15,15]^2 and |p0| <= 3; K=32 each, one step dt=0.5."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        nx, ny = (int(rng.choice(sides)), int(rng.choice(sides)))
        g = make_grid((nx, ny), (-30.0, -30.0), (30.0, 30.0))
        V = gaussian_wells(g, rng)
        r0 = rng.uniform(-15.0, 15.0, size=2)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        pm = rng.uniform(0.0, 3.0)
        probs.append({"grid": g, "V": V,
                      "psi0": wave_packet(g, r0, 1.0, (pm * np.cos(ang), pm * np.sin(ang)))})
    return {"name": "batched_64x2d_K32", "problems": probs, "K": 32, "dt": 0.5, "nsteps": 1,
            "precision": "mixed", "tol": 1e-6}


def config_learnable(seed=5, target_seed=105, n=256):
    """2D n^2 on [-30, 30)^2, V = 8-mode Fourier field (seed), target state from
    the same evolution under a second field (target_seed); K=32, 10 steps dt=0.5."""
    g = make_grid((n, n), (-30.0, -30.0), (30.0, 30.0))
    V = fourier_field(g, np.random.default_rng(seed))
    Vt = fourier_field(g, np.random.default_rng(target_seed))
    return {"name": "learnable_V_256x256_K32", "grid": g, "V": V, "V_target": Vt,
            "psi0": wave_packet(g, (-10.0, 0.0), 1.0, (3.0, 0.0)), "K": 32, "dt": 0.5,
            "nsteps": 10, "precision": "mixed", "tol": 1e-6}
