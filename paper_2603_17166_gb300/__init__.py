"""GB300 (sm_103a) partial-sky spin-s spherical harmonic transforms.

Synthesis general and its adjoint at arbitrary points inside one sky patch, by the partial-sky
Fourier-sphere route of Carron & Reinecke (Wigner-d recursion onto apodised rings, FFTs onto a
reduced oversampled grid, ES-kernel interpolation), as a C-ABI CUDA library with a thin binding.
"""
from .psht import (Plan, PshtError, Rotator, Server, adjoint_synthesis, estimate_bytes, estimate_points,  # noqa: F401
                   lib, nalm, patch_rotation, plan_params, predict_error, rotate_alm, rotate_points,
                   synthesis)
