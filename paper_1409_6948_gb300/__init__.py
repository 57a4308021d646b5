"""GB300 (sm_103a) parallel event-chain Monte Carlo for two-dimensional hard
disks and three-dimensional hard spheres (Kampmann, Boltz, Kierfeld,
arXiv:1409.6948), with the striped decomposition the paper compares against.

The computation lives in the CUDA library libecmc.so (C ABI in
include/ecmc.h, include/ecmc3.h and include/ecmc_stripes.h); this package only loads it and marshals
arguments.
"""
from .ecmc import (DIR_PM_AXIS_ALT, DIR_POS_ONLY, PREC_FP32_GEOM, PREC_FP64, Ecmc, Ecmc3,
                   EcmcError, EcmcStripes, load, version)

__all__ = ["Ecmc", "Ecmc3", "EcmcStripes", "EcmcError", "load", "version", "DIR_PM_AXIS_ALT", "DIR_POS_ONLY",
           "PREC_FP64", "PREC_FP32_GEOM"]
