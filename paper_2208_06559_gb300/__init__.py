"""GB300 (sm_103a) library for the per-timestep hot path of bead-rod Brownian
dynamics with hydrodynamic interaction (arXiv 2208.06559).

The compute lives in libbd.so (CUDA kernels behind the C ABI of include/bd.h);
``binding`` marshals torch tensors into it and ``build`` compiles it.
"""
from .binding import (FLOW_NONE, FLOW_SHEAR, FLOW_UNIAXIAL, FP64, FRAENKEL, MIXED_BF16, MIXED_TF32,
                      OBS_MAXDEV, OBS_NEWTON, OBS_R2, OBS_REE_X, OBS_RG2, OBS_STRETCH, OBS_STRIDE,
                      OBS_TAU_XX, OBS_TAU_XY, OBS_TAU_YY, OBS_TAU_ZZ, RIGID, SCHEME_EULER, SCHEME_MIDPOINT,
                      BDError, Context, lib)

__all__ = ["Context", "BDError", "lib", "FLOW_NONE", "FLOW_SHEAR", "FLOW_UNIAXIAL", "FP64",
           "MIXED_TF32", "MIXED_BF16", "OBS_STRIDE", "OBS_REE_X", "OBS_R2", "OBS_RG2", "OBS_STRETCH",
           "OBS_MAXDEV", "OBS_NEWTON", "OBS_TAU_XX", "OBS_TAU_YY", "OBS_TAU_ZZ", "OBS_TAU_XY", "RIGID",
           "FRAENKEL", "SCHEME_MIDPOINT", "SCHEME_EULER"]
