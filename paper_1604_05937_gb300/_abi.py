"""ctypes binding of the extmesh C ABI (include/extmesh.h), same names.

Argument marshalling only: every computation happens in libextmesh.so.  The
import fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# EXTMESH_CHECKED=1 loads the checked build (stencil indices range-checked on
# the device before every launch)
LIB_PATH = os.path.join(_HERE, "libextmesh_checked.so" if os.environ.get("EXTMESH_CHECKED") == "1"
                        else "libextmesh.so")

EXT_OK, EXT_EINVAL, EXT_ENOMEM, EXT_ECUDA, EXT_EOVERFLOW, EXT_ETIMEOUT, EXT_EDEVICE, EXT_EUNSUPPORTED = range(8)
STATUS_NAMES = ["EXT_OK", "EXT_EINVAL", "EXT_ENOMEM", "EXT_ECUDA", "EXT_EOVERFLOW", "EXT_ETIMEOUT",
                "EXT_EDEVICE", "EXT_EUNSUPPORTED"]
EXT_TRI, EXT_QUAD = 3, 4
EXT_READ, EXT_WRITE, EXT_INC = 0, 1, 2
(EXT_K_EXTRUDE, EXT_K_COPY_DG, EXT_K_RHS_P1P1, EXT_K_MASS_P1P1, EXT_K_INTERP_DG1, EXT_K_U2V_FWD,
 EXT_K_U2V_ADJ, EXT_K_U2V_FWDADJ, EXT_K_MASS_TP, EXT_K_HFACET_MASS, EXT_K_HFACET_JUMP, EXT_K_MASS_DGP) = range(12)


class ExtError(RuntimeError):
    """A non-zero ext_status, with the library's message."""

    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class ext_arg(ctypes.Structure):
    _fields_ = [("space", ctypes.c_void_p), ("data", ctypes.c_void_p), ("access", ctypes.c_int32)]


class ext_tune_params(ctypes.Structure):
    _fields_ = [("cols_per_item", ctypes.c_int32), ("layer_tile", ctypes.c_int32),
                ("use_atomics", ctypes.c_int32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"extmesh CUDA library not built ({LIB_PATH} missing); "
                          "run paper_1604_05937_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "ext_abi_version": (i32, []),
        "ext_last_error": (ctypes.c_char_p, []),
        "ext_mesh_create": (ctypes.c_int, [i32, i64, i64, vp, vp, i32, ctypes.POINTER(vp)]),
        "ext_mesh_create_var": (ctypes.c_int, [i32, i64, i64, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "ext_mesh_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        "ext_mesh_destroy": (None, [vp]),
        "ext_number_dofs": (ctypes.c_int, [vp, vp, i32, vp, ctypes.POINTER(vp)]),
        "ext_number_dofs_ragged": (ctypes.c_int, [vp, vp, i32, vp, ctypes.POINTER(vp)]),
        "ext_space_ragged_info": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                 ctypes.POINTER(vp)]),
        "ext_space_copy_ragged_to_host": (ctypes.c_int, [vp, vp, vp, vp]),
        "ext_space_info": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "ext_space_copy_map_to_host": (ctypes.c_int, [vp, vp, vp]),
        "ext_space_destroy": (None, [vp]),
        "ext_par_loop": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(ext_arg), vp]),
        "ext_batch_create": (ctypes.c_int, [i32, ctypes.POINTER(vp), i32, i32, ctypes.POINTER(ext_arg),
                                            ctypes.POINTER(ext_tune_params), vp, ctypes.POINTER(vp)]),
        "ext_batch_launch": (ctypes.c_int, [vp, vp]),
        "ext_batch_launch_params": (ctypes.c_int, [vp, ctypes.POINTER(ext_tune_params), vp]),
        "ext_batch_params": (ctypes.c_int, [vp, ctypes.POINTER(ext_tune_params)]),
        "ext_batch_destroy": (None, [vp]),
        "ext_sync_check": (ctypes.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(st: int) -> None:
    if st != EXT_OK:
        raise ExtError(st, lib.ext_last_error().decode())


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    """cudaStream_t handle of a torch stream / int; None = torch's current stream."""
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def ext_abi_version() -> int:
    return lib.ext_abi_version()


def ext_last_error() -> str:
    return lib.ext_last_error().decode()


def ext_mesh_create(kind: int, nverts: int, ncells: int, cell_verts, base_xy, layers: int) -> int:
    cv = np.ascontiguousarray(cell_verts, dtype=np.int32)
    xy = None if base_xy is None else np.ascontiguousarray(base_xy, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib.ext_mesh_create(kind, nverts, ncells, _ptr(cv) if cv.size else None,
                               None if xy is None else _ptr(xy), layers, ctypes.byref(out)))
    return out.value


def ext_mesh_create_var(kind: int, nverts: int, ncells: int, cell_verts, base_xy, cell_first,
                        cell_layers) -> int:
    cv = np.ascontiguousarray(cell_verts, dtype=np.int32)
    xy = None if base_xy is None else np.ascontiguousarray(base_xy, dtype=np.float64)
    cf = np.ascontiguousarray(cell_first, dtype=np.int32)
    cl = np.ascontiguousarray(cell_layers, dtype=np.int32)
    if cf.shape != (ncells,) or cl.shape != (ncells,):
        raise ValueError("cell_first and cell_layers need one entry per base cell")
    out = ctypes.c_void_p()
    _check(lib.ext_mesh_create_var(kind, nverts, ncells, _ptr(cv) if cv.size else None,
                                   None if xy is None else _ptr(xy), _ptr(cf) if cf.size else None,
                                   _ptr(cl) if cl.size else None, ctypes.byref(out)))
    return out.value


def ext_mesh_info(mesh: int):
    kind = ctypes.c_int32()
    n = (ctypes.c_int64 * 3)()
    layers = ctypes.c_int32()
    _check(lib.ext_mesh_info(mesh, ctypes.byref(kind), n, ctypes.byref(layers)))
    return kind.value, (n[0], n[1], n[2]), layers.value


def ext_mesh_destroy(mesh: int) -> None:
    lib.ext_mesh_destroy(mesh)


def ext_number_dofs(mesh: int, delta, ncomp: int = 1, stream=None) -> int:
    d = np.ascontiguousarray(delta, dtype=np.int32)
    if d.size != 6:
        raise ValueError("delta has 6 entries: delta((d1,d2)) at 2*d1+d2")
    out = ctypes.c_void_p()
    _check(lib.ext_number_dofs(mesh, _ptr(d), ncomp, _stream(stream), ctypes.byref(out)))
    return out.value


def ext_space_info(space: int):
    nd = ctypes.c_int64()
    k = ctypes.c_int32()
    nc = ctypes.c_int32()
    mp = ctypes.c_void_p()
    op = ctypes.c_void_p()
    _check(lib.ext_space_info(space, ctypes.byref(nd), ctypes.byref(k), ctypes.byref(nc), ctypes.byref(mp),
                              ctypes.byref(op)))
    return nd.value, k.value, nc.value, mp.value, op.value


def ext_space_copy_map_to_host(space: int, ncells: int):
    _, k, _, _, _ = ext_space_info(space)
    m = np.empty((ncells, k), dtype=np.int32)
    o = np.empty(k, dtype=np.int32)
    _check(lib.ext_space_copy_map_to_host(space, _ptr(m) if m.size else None, _ptr(o)))
    return m, o


def ext_number_dofs_ragged(mesh: int, dent, ncomp: int = 1, stream=None) -> int:
    d = np.ascontiguousarray(dent, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib.ext_number_dofs_ragged(mesh, _ptr(d) if d.size else None, ncomp, _stream(stream), ctypes.byref(out)))
    return out.value


def ext_space_ragged_info(space: int):
    n = ctypes.c_int64()
    rp, mp, op = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.ext_space_ragged_info(space, ctypes.byref(n), ctypes.byref(rp), ctypes.byref(mp), ctypes.byref(op)))
    return n.value, rp.value, mp.value, op.value


def ext_space_copy_ragged_to_host(space: int, ncells: int):
    n, _, _, _ = ext_space_ragged_info(space)
    rowptr = np.empty(ncells + 1, dtype=np.int64)
    m = np.empty(n, dtype=np.int32)
    o = np.empty(n, dtype=np.int32)
    _check(lib.ext_space_copy_ragged_to_host(space, _ptr(rowptr), _ptr(m) if n else None, _ptr(o) if n else None))
    return rowptr, m, o


def ext_space_destroy(space: int) -> None:
    lib.ext_space_destroy(space)


def _args(args) -> ctypes.Array:
    arr = (ext_arg * max(1, len(args)))()
    for i, (space, data, access) in enumerate(args):
        arr[i].space = space
        arr[i].data = _ptr(data)
        arr[i].access = access
    return arr


def ext_par_loop(mesh: int, kernel_id: int, args, stream=None) -> None:
    """args: sequence of (space handle, data tensor/pointer, access)."""
    _check(lib.ext_par_loop(mesh, kernel_id, len(args), _args(args), _stream(stream)))


def _params(p):
    if p is None:
        return None
    if isinstance(p, ext_tune_params):
        return ctypes.byref(p)
    q = ext_tune_params(**p)
    return ctypes.byref(q)


def ext_batch_create(meshes, kernel_id: int, nargs: int, args, params=None, stream=None) -> int:
    """args: flat mesh-major list of nmesh * nargs (space, data, access)."""
    ms = (ctypes.c_void_p * len(meshes))(*meshes)
    out = ctypes.c_void_p()
    _check(lib.ext_batch_create(len(meshes), ms, kernel_id, nargs, _args(args), _params(params),
                                _stream(stream), ctypes.byref(out)))
    return out.value


def ext_batch_launch(batch: int, stream=None) -> None:
    _check(lib.ext_batch_launch(batch, _stream(stream)))


def ext_batch_launch_params(batch: int, params, stream=None) -> None:
    _check(lib.ext_batch_launch_params(batch, _params(params), _stream(stream)))


def ext_batch_params(batch: int) -> dict:
    p = ext_tune_params()
    _check(lib.ext_batch_params(batch, ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in ext_tune_params._fields_}


lib.ext_batch_plan_info.restype = ctypes.c_int
lib.ext_batch_plan_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
TUNE_SOURCES = {0: "given", 1: "autotuned", 2: "cache"}


def ext_batch_plan_info(batch: int) -> dict:
    """Origin of the batch's parameters and the host time of its creation."""
    src, sec = ctypes.c_int32(0), ctypes.c_double(0.0)
    _check(lib.ext_batch_plan_info(batch, ctypes.byref(src), ctypes.byref(sec)))
    return {"source": TUNE_SOURCES.get(int(src.value), str(src.value)), "setup_seconds": float(sec.value)}


def ext_batch_destroy(batch: int) -> None:
    lib.ext_batch_destroy(batch)


def ext_sync_check(stream=None) -> None:
    _check(lib.ext_sync_check(_stream(stream)))


# ---- batched launch without allocation (ext_batch_run_noalloc)
lib.ext_batch_run_noalloc.restype = ctypes.c_int
lib.ext_batch_run_noalloc.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                      ctypes.c_int32, ctypes.POINTER(ext_arg), ctypes.POINTER(ext_tune_params),
                                      ctypes.c_void_p]
EXT_NOALLOC_MAX_MESHES = 256


def ext_batch_run_noalloc(meshes, kernel_id: int, nargs: int, args, params=None, stream=None) -> None:
    """Batched u^2 v launch that allocates no device memory, for callers that
    cannot call cudaMalloc; args is the flat mesh-major list of (space, data,
    access).  Calls that overlap on the GPU share one scratch array and race."""
    ms = (ctypes.c_void_p * len(meshes))(*meshes)
    _check(lib.ext_batch_run_noalloc(len(meshes), ms, kernel_id, nargs, _args(args), _params(params),
                                     _stream(stream)))


# ---- FP64 issue rates (roofline denominator of the FP64-bound kernels)
lib.ext_fp64_rates.restype = ctypes.c_int
lib.ext_fp64_rates.argtypes = [ctypes.c_void_p, ctypes.c_void_p]


def ext_fp64_rates(stream=None) -> dict:
    """Measured DFMA, DADD, DMUL issue rates and L2 FP64 atomic-add rate (G/s)."""
    out = np.zeros(4)
    _check(lib.ext_fp64_rates(_ptr(out), _stream(stream)))
    return {"dfma": float(out[0]), "dadd": float(out[1]), "dmul": float(out[2]), "l2_atomic_add": float(out[3])}


# ---- process-wide options (ext_set_option / ext_get_option)
EXT_OPT_P1_FORM = 1
EXT_OPT_P1_FLAT = 2
EXT_P1_FLAT_FUSED, EXT_P1_FLAT_SPLIT, EXT_P1_FLAT_OPTIMISTIC = 0, 1, 2
(EXT_P1_AUTO, EXT_P1_SPLIT, EXT_P1_GATHER, EXT_P1_FACTORED, EXT_P1_UNFACTORED, EXT_P1_CELLS,
 EXT_P1_SINGLE) = range(7)
P1_FORMS = {"auto": EXT_P1_AUTO, "split": EXT_P1_SPLIT, "gather": EXT_P1_GATHER, "factored": EXT_P1_FACTORED,
            "unfactored": EXT_P1_UNFACTORED, "cells": EXT_P1_CELLS, "single": EXT_P1_SINGLE}
lib.ext_set_option.restype = ctypes.c_int
lib.ext_set_option.argtypes = [ctypes.c_int32, ctypes.c_int32]
lib.ext_get_option.restype = ctypes.c_int
lib.ext_get_option.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]


def ext_set_option(option: int, value: int) -> None:
    _check(lib.ext_set_option(option, value))


def ext_get_option(option: int) -> int:
    v = ctypes.c_int32(0)
    _check(lib.ext_get_option(option, ctypes.byref(v)))
    return int(v.value)


# ---- range check of a space's stencil lists (ext_space_check)
lib.ext_space_check.restype = ctypes.c_int
lib.ext_space_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]


def ext_space_check(space: int, stream=None) -> None:
    _check(lib.ext_space_check(space, _stream(stream)))
