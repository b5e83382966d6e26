"""GB300-native (sm_103a) recursive regularised lattice Boltzmann solver for
2-D incompressible MHD (De Rosis, "Recursive regularised lattice Boltzmann
method for magnetohydrodynamics").

The solver is the CUDA library ``libmhdlbm.so`` behind the C ABI of
``include/mhd.h``; this package is its thin Python binding.
"""
from ._abi import (MHD_BGK, MHD_FP16S, MHD_FP32, MHD_FP64, MHD_HALO, MHD_IN_PLACE, MHD_MAG_BGK,
                   MHD_MAG_REGULARISED, MHD_PERIODIC, MHD_RR, MHD_TWO_BUFFERS, MHD_WALL, Batch, Lattice,
                   MhdError, check, lib)


def tau_from_viscosity(nu: float) -> float:
    """tau = 1/2 + nu / cs^2 with cs^2 = 1/3 (the paper's transport relation
    with the cs^2 factor it omits; the same holds for eta and tau_m)."""
    return 0.5 + 3.0 * nu


__all__ = ["Lattice", "Batch", "MhdError", "lib", "check", "tau_from_viscosity", "MHD_FP64", "MHD_FP32",
           "MHD_FP16S", "MHD_PERIODIC", "MHD_WALL", "MHD_RR", "MHD_BGK",
           "MHD_MAG_BGK", "MHD_MAG_REGULARISED", "MHD_TWO_BUFFERS", "MHD_IN_PLACE", "MHD_HALO"]
