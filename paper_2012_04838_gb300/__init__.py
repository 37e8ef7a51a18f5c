"""GB300-native pseudo-spectral solver for forced homogeneous isotropic
turbulence with a passive scalar (arXiv:2012.04838, section 2).

The compute path is the CUDA library ``libpsc.so`` (C ABI in ``include/psc.h``);
``binding`` is its ctypes wrapper and ``build`` compiles it with nvcc.
"""
from .binding import (FP32_MIXED, FP64, FORCE_CONST_POWER, FORCE_HOLD_ENERGY, FORCE_NONE, IC_PAPER_EQ9, NL_CONVECTIVE,
                      NL_ROTATIONAL, DEALIAS_TWO_THIRDS, DEALIAS_PHASE_SHIFT,
                      IC_SPECTRUM_K4, IC_TAYLOR_GREEN_NOISE, INTEG_IFRK4, INTEG_RK4, Params,
                      Batch, PersistentBatch, PscError, Simulation, XPassProbe, PERSISTENT_SIZES, compact_shape, load, supported_sizes, workspace_size)

__all__ = ["Params", "Simulation", "Batch", "PersistentBatch", "PERSISTENT_SIZES", "XPassProbe", "PscError", "load", "supported_sizes", "workspace_size",
           "compact_shape", "FP64", "FP32_MIXED", "IC_SPECTRUM_K4", "IC_TAYLOR_GREEN_NOISE",
           "IC_PAPER_EQ9", "FORCE_NONE", "FORCE_CONST_POWER", "FORCE_HOLD_ENERGY", "INTEG_IFRK4", "INTEG_RK4",
           "NL_ROTATIONAL", "NL_CONVECTIVE", "DEALIAS_TWO_THIRDS", "DEALIAS_PHASE_SHIFT"]
