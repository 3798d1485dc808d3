"""Plain FP64 CPU oracle for the McMurchie-Davidson RHF hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline / reference leg, never by the product package.  It
shares no code with the CUDA library; both read the same seeded inputs from
``fsim_synth``.
"""
from .oracle import (OracleBasis, build, boys, hermite_E, hermite_R, jacobi_eigh)
from .scf import rhf, core_guess_density
from .spherical import SphericalOracleBasis

__all__ = ["OracleBasis", "build", "boys", "hermite_E", "hermite_R", "jacobi_eigh",
           "rhf", "core_guess_density", "SphericalOracleBasis"]
