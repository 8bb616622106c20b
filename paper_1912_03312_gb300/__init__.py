"""GB300-native engine for the Faber-Caratheodory-Fejer REXI time step of
Rittich & Speck, "Time-parallel simulation of the Schroedinger equation"
(arXiv:1912.03312).

The compute path is the CUDA library ``librexi.so`` (C ABI in include/rexi.h);
this package only marshals arguments to it.
"""

from . import _native
from .rexi import Plan, RexiEvolve, fcf, options, step_batched

__all__ = ["Plan", "RexiEvolve", "fcf", "options", "step_batched", "_native"]
