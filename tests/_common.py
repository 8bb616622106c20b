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
