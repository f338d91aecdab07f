"""Numbering and par_loop over extruded meshes on one GB300 GPU.

The method is Bercea et al.'s vertical-innermost numbering (Algorithm 1),
vertical offsets (Algorithm 2) and layered stencil iteration (Algorithm 3);
the compute path is the CUDA library libextmesh.so behind the C ABI in
include/extmesh.h.  This package is its binding: ``_abi`` mirrors the C
functions by name, ``api`` adds meshes, spaces and torch fields.
"""
from ._abi import *  # noqa: F401,F403  (ext_* functions and constants)
from ._abi import ExtError, LIB_PATH  # noqa: F401
from .api import (DELTA, Batch, Mesh, ResidualFn, Space, extrude_coords, par_loop,  # noqa: F401
                  residual_u2v, residual_u2v_adjoint)
