"""Shared set-up for the GPU parity tests: the same seeded problem handed to the
CUDA library (through the C ABI) and to the oracle (each with its own plan
arithmetic; only the inputs are shared)."""

import numpy as np

import workloads as wl
from oracle import plan as oplan
from oracle import tables


class OraclePlan:
    """The oracle's version of a plan: spacing, enclosure, substeps, poles."""

    def __init__(self, g, V, dt, K, R1):
        self.h = oplan.grid_spacing(g["n"], g["lo"], g["hi"])
        self.emin, self.emax, self.c, self.W = oplan.spectral_enclosure(V, self.h, g["hbar"], g["mass"])
        self.n_sub = oplan.substeps(dt, self.W, R1, g["hbar"])
        self.tau = dt / self.n_sub
        self.sigma, self.beta, _ = tables.poles(K, R1)
        self.z, self.alpha, self.alpha0 = oplan.physical_poles(self.sigma, self.beta, self.tau, self.c, g["hbar"])
        self.A = oplan.amplification(self.sigma, self.beta, R1)
        self.V = V
        self.g = g


def library_plan(g, V, dt, K, R1, **opts):
    from paper_1912_03312_gb300 import Plan
    return Plan(g["n"], g["lo"], g["hi"], V, dt, K, hbar=g["hbar"], mass=g["mass"], R1=R1, **opts)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


METRIC_TOL = 1e-6     # the step error the benchmark metric allows against FP64


def solve_tol(A, cap=1e-13):
    """Per-pole relative residual for a step parity case: `cap`, or less where
    the pole-sum amplification A would otherwise let two solvers that each stop
    at that residual differ by more than the metric's 1e-6 (2 A tol <= 0.95e-6;
    for K = 32, R1 = 68: A = 2.5e7, tol = 1.9e-14)."""
    return min(cap, 0.475 * METRIC_TOL / A)


def step_bound(A, tol, precision):
    """Step tolerance of two solvers at relative residual tol: the precision's
    floor (1e-10 FP64, 1e-6 mixed) or 2 A tol, whichever is larger."""
    return max(1e-10 if precision == "fp64" else METRIC_TOL, 2.0 * A * tol)


def log_parity(name, err, bound, **extra):
    """Append one measured parity error to $REXI_PARITY_LOG (JSON lines) when
    that variable is set; a no-op otherwise."""
    import json
    import os
    path = os.environ.get("REXI_PARITY_LOG")
    if not path:
        return
    rec = dict(name=name, err=float(err), bound=float(bound))
    rec.update({k: (float(v) if isinstance(v, (int, float, np.floating)) else str(v)) for k, v in extra.items()})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")
