"""GB300-native FP64 WENO5/WENO7 + RK3 solver for 3+1D ideal relativistic
hydrodynamics (after Sikorski et al., arXiv:1604.03360).

The hot path runs in hand-written sm_103a CUDA kernels behind the C ABI of
include/hydro.h (libhydro.so, built in-tree by build.py).  This package is the
thin Python binding over that ABI.
"""
from ._binding import (BC_HALO, BC_OUTFLOW, BC_PERIODIC, MEM_DEVICE, MEM_HOST, MUSTA_FORCE, WENO5, WENO7, Hydro, HydroBatch, HydroConfig,
                       HydroError, LIB_PATH, as_buffer, eval_rcp, lib, make_config, measure_fp64_peak)

from . import autograd  # noqa: E402  (torch.autograd.Function wrappers of the adjoint)

__all__ = ["autograd", "Hydro", "HydroBatch", "HydroConfig", "HydroError", "lib", "make_config", "measure_fp64_peak", "eval_rcp", "as_buffer", "LIB_PATH",
           "WENO5", "WENO7", "MUSTA_FORCE", "BC_OUTFLOW", "BC_PERIODIC", "BC_HALO", "MEM_HOST", "MEM_DEVICE"]
