"""GB300-native matrix-free high-order nonlinear Stokes operator.

The compute path is the CUDA library libstokes_gb300.so (C-ABI in
include/stokes.h); this package only marshals arguments to it.
"""
from . import capi
from .capi import (STOKES_F32, STOKES_F64, StokesError, stokes_jacobian_apply,
                   stokes_jacobian_apply_transpose, stokes_linearize, stokes_mesh_create,
                   stokes_mesh_destroy, stokes_mesh_sizes, stokes_param_grad, stokes_residual,
                   stokes_state_apply, stokes_state_apply_transpose, stokes_state_create,
                   stokes_state_destroy)
from .mesh import Mesh, State, params

__all__ = [
    "capi", "Mesh", "State", "params", "StokesError", "STOKES_F32", "STOKES_F64",
    "stokes_mesh_create", "stokes_mesh_destroy", "stokes_mesh_sizes", "stokes_residual",
    "stokes_jacobian_apply", "stokes_jacobian_apply_transpose", "stokes_param_grad",
    "stokes_state_create", "stokes_state_destroy", "stokes_linearize", "stokes_state_apply",
    "stokes_state_apply_transpose",
]
