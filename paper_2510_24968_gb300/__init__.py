"""GB300 (sm_103a) McMurchie-Davidson RHF hot path: C-ABI libfsim + thin binding."""
from .fsim import (Basis, Batch, scf_batched, load, FsimError, FSIM_FP64, FSIM_MIXED, FSIM_DFLOAT, FSIM_PTR_HOST,
                   FSIM_PTR_DEVICE, FSIM_GUESS_CORE, FSIM_GUESS_DENSITY, EXPORTS, LIB_PATH)

__all__ = ["Basis", "Batch", "scf_batched", "load", "FsimError", "FSIM_FP64", "FSIM_MIXED", "FSIM_DFLOAT",
           "FSIM_PTR_HOST", "FSIM_PTR_DEVICE", "FSIM_GUESS_CORE", "FSIM_GUESS_DENSITY", "EXPORTS", "LIB_PATH"]
