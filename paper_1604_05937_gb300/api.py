"""Object layer over the C ABI: meshes, function spaces, fields as torch
tensors, par_loop, batched plans and the autograd Function of the u^2 v
residual.  PyTorch provides device memory and streams; every kernel is the
library's."""
from __future__ import annotations

import numpy as np

from . import _abi as A

# delta((d1,d2)) at index 2*d1+d2 for the spaces the kernels know
DELTA = {
    "CG1xCG1": (1, 0, 0, 0, 0, 0),
    "DG0xDG0": (0, 0, 0, 0, 0, 1),
    "DG1xDG1": (0, 0, 0, 0, 0, 6),
    "Q2xP2": (1, 1, 1, 1, 1, 1),
    "DG2": (0, 0, 0, 0, 0, 27),
    # the nine prism spaces of Sec. 4.1.2 (CG1xCG1 and DG0xDG0, DG1xDG1 above)
    "CG1xDG0": (0, 1, 0, 0, 0, 0),
    "CG1xDG1": (0, 2, 0, 0, 0, 0),
    "DG0xCG1": (0, 0, 0, 0, 1, 0),
    "DG0xDG1": (0, 0, 0, 0, 0, 2),
    "DG1xCG1": (0, 0, 0, 0, 3, 0),
    "DG1xDG0": (0, 0, 0, 0, 0, 3),
}


def _torch():
    import torch
    return torch


class Mesh:
    """Extruded mesh: base cells (C, 3|4) int32, optional base coordinates
    (V, 2) float64, and the number of layers: an int, or per-column
    ``cell_first``/``cell_layers`` arrays for variable layers (then
    ``layers`` is ignored and reports the highest level)."""

    def __init__(self, cells, xy=None, layers: int = 1, nverts: int | None = None, cell_first=None,
                 cell_layers=None):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        if cells.ndim != 2 or cells.shape[1] not in (3, 4):
            raise ValueError("cells must be (C, 3) or (C, 4)")
        nv = int(xy.shape[0]) if xy is not None else int(nverts if nverts is not None else cells.max() + 1)
        if cell_layers is not None:
            first = np.zeros(cells.shape[0], np.int32) if cell_first is None else cell_first
            self.handle = A.ext_mesh_create_var(cells.shape[1], nv, cells.shape[0], cells, xy, first, cell_layers)
            self.variable = True
        else:
            self.handle = A.ext_mesh_create(cells.shape[1], nv, cells.shape[0], cells, xy, layers)
            self.variable = False
        self.kind, self.N, self.layers = A.ext_mesh_info(self.handle)

    @property
    def ncells(self) -> int:
        return self.N[2]

    def close(self):
        if getattr(self, "handle", None):
            A.ext_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Space:
    """A function space numbered by Algorithm 1 on `mesh`: one delta table
    for every entity type, or per-entity counts ``dent`` ((V + E + C) x 2,
    dimension-major; ragged lists)."""

    def __init__(self, mesh: Mesh, delta=None, ncomp: int = 1, stream=None, dent=None):
        self.mesh = mesh
        if dent is not None:
            self.delta = None
            self.handle = A.ext_number_dofs_ragged(mesh.handle, dent, ncomp, stream)
        else:
            if isinstance(delta, str):
                delta = DELTA[delta]
            self.delta = tuple(int(d) for d in delta)
            self.handle = A.ext_number_dofs(mesh.handle, self.delta, ncomp, stream)
        self.ndofs, self.k, self.ncomp, _, _ = A.ext_space_info(self.handle)
        self.ragged = dent is not None

    def stencil_map(self):
        """(C, k) layer-0 stencil lists and (k,) offsets, copied to the host;
        for per-entity counts (rowptr, entries, per-entry offsets)."""
        if self.ragged:
            return A.ext_space_copy_ragged_to_host(self.handle, self.mesh.ncells)
        return A.ext_space_copy_map_to_host(self.handle, self.mesh.ncells)

    def zeros(self, device="cuda"):
        torch = _torch()
        return torch.zeros(self.ndofs * self.ncomp, dtype=torch.float64, device=device)

    def close(self):
        if getattr(self, "handle", None):
            A.ext_space_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_field(space: Space, t) -> None:
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("fields are torch tensors")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("fields must be contiguous float64 CUDA tensors")
    if t.numel() != space.ndofs * space.ncomp:
        raise ValueError(f"field has {t.numel()} values, space needs {space.ndofs * space.ncomp}")


def par_loop(mesh: Mesh, kernel_id: int, *args, stream=None) -> None:
    """Algorithm 3 with local kernel `kernel_id`; args are (Space, tensor, access)."""
    for sp, t, _ in args:
        _check_field(sp, t)
    A.ext_par_loop(mesh.handle, kernel_id, [(sp.handle, t, acc) for sp, t, acc in args], stream)


def extrude_coords(mesh: Mesh, coords: Space, stream=None):
    X = coords.zeros()
    par_loop(mesh, A.EXT_K_EXTRUDE, (coords, X, A.EXT_WRITE), stream=stream)
    return X


class Batch:
    """Captured batched persistent launch of a u^2 v kernel over many meshes.

    per_mesh: list of argument lists [(Space, tensor, access), ...] (one per
    mesh, the kernel's argument order).  params=None autotunes."""

    def __init__(self, meshes, kernel_id: int, per_mesh, params=None, stream=None):
        self.meshes = list(meshes)
        self.keep = per_mesh
        nargs = len(per_mesh[0])
        flat = []
        for m, args in zip(self.meshes, per_mesh):
            for sp, t, acc in args:
                _check_field(sp, t)
                flat.append((sp.handle, t, acc))
        self.handle = A.ext_batch_create([m.handle for m in self.meshes], kernel_id, nargs, flat, params, stream)

    @property
    def params(self) -> dict:
        return A.ext_batch_params(self.handle)

    @property
    def plan_info(self) -> dict:
        """{"source": "given" | "autotuned" | "cache", "setup_seconds": host time of the creation}."""
        return A.ext_batch_plan_info(self.handle)

    def launch(self, stream=None) -> None:
        A.ext_batch_launch(self.handle, stream)

    def launch_params(self, params, stream=None) -> None:
        A.ext_batch_launch_params(self.handle, params, stream)

    def close(self):
        if getattr(self, "handle", None):
            A.ext_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _out_access(space: Space) -> int:
    # continuous spaces accumulate (INC); DG2 is written (WRITE)
    return A.EXT_WRITE if space.delta == DELTA["DG2"] else A.EXT_INC


def residual_u2v(mesh: Mesh, coords: Space, X, space: Space, u):
    """F(u)_i = int u_h^2 phi_i dx."""
    F = space.zeros()
    par_loop(mesh, A.EXT_K_U2V_FWD, (coords, X, A.EXT_READ), (space, u, A.EXT_READ),
             (space, F, _out_access(space)))
    return F


def residual_u2v_adjoint(mesh: Mesh, coords: Space, X, space: Space, u, w):
    """g = (dF/du)^T w, the hand-written adjoint par_loop."""
    g = space.zeros()
    par_loop(mesh, A.EXT_K_U2V_ADJ, (coords, X, A.EXT_READ), (space, u, A.EXT_READ), (space, w, A.EXT_READ),
             (space, g, _out_access(space)))
    return g


def _make_residual_fn():
    torch = _torch()

    class ResidualFn(torch.autograd.Function):
        """F = ResidualFn.apply(u, mesh, coords, X, space): the u^2 v residual as
        a differentiable function of u; backward runs the adjoint par_loop."""

        @staticmethod
        def forward(ctx, u, mesh, coords, X, space):
            u = u.contiguous()
            ctx.save_for_backward(u)
            ctx.meta = (mesh, coords, X, space)
            return residual_u2v(mesh, coords, X, space, u)

        @staticmethod
        def backward(ctx, gF):
            (u,) = ctx.saved_tensors
            mesh, coords, X, space = ctx.meta
            g = residual_u2v_adjoint(mesh, coords, X, space, u, gF.contiguous())
            return g, None, None, None, None

    return ResidualFn


_residual_fn = None


def ResidualFn():
    """The torch.autograd.Function class (created on first use, importing torch lazily)."""
    global _residual_fn
    if _residual_fn is None:
        _residual_fn = _make_residual_fn()
    return _residual_fn
