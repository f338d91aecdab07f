"""ctypes wrapper of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg.  The CUDA library and its binding
never import this package.  Everything here marshals arguments; the
arithmetic lives in oracle.c (Algorithms 1-3 of Sec. 3, the local kernels of
Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

READ, WRITE, INC = 0, 1, 2
K_EXTRUDE, K_COPY, K_MASS, K_INTERP, K_U2V, K_U2V_ADJ, K_MASS_TP = range(7)
CG1, DG0, DG1 = 0, 1, 2

# delta((d1,d2)) flattened as [d(0,0), d(0,1), d(1,0), d(1,1), d(2,0), d(2,1)]
DELTA = {
    "CG1xCG1": (1, 0, 0, 0, 0, 0),
    "CG1xDG0": (0, 1, 0, 0, 0, 0),
    "CG1xDG1": (0, 2, 0, 0, 0, 0),
    "DG0xCG1": (0, 0, 0, 0, 1, 0),
    "DG0xDG0": (0, 0, 0, 0, 0, 1),
    "DG0xDG1": (0, 0, 0, 0, 0, 2),
    "DG1xCG1": (0, 0, 0, 0, 3, 0),
    "DG1xDG0": (0, 0, 0, 0, 0, 3),
    "DG1xDG1": (0, 0, 0, 0, 0, 6),
    "Q2xP2": (1, 1, 1, 1, 1, 1),
    "DG2hex": (0, 0, 0, 0, 0, 27),
}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no fused multiply-add)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Arg(ctypes.Structure):
    _fields_ = [
        ("map", ctypes.c_void_p),
        ("offset", ctypes.c_void_p),
        ("k", ctypes.c_int32),
        ("ncomp", ctypes.c_int32),
        ("data", ctypes.c_void_p),
        ("absdata", ctypes.c_void_p),
        ("access", ctypes.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB lets the mutation test load a deliberately broken copy
        override = os.environ.get("ORACLE_LIB")
        if override:
            path = override
        else:
            path = build()
        L = ctypes.CDLL(path)
        L.oracle_derive_edges.restype = ctypes.c_int64
        L.oracle_derive_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p]
        L.oracle_alg1.restype = ctypes.c_int64
        L.oracle_alg1.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_stencil_size.restype = ctypes.c_int32
        L.oracle_stencil_size.argtypes = [ctypes.c_int32, ctypes.c_void_p]
        L.oracle_base_map.restype = ctypes.c_int
        L.oracle_base_map.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_alg2.restype = None
        L.oracle_alg2.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_par_loop.restype = ctypes.c_int
        L.oracle_par_loop.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        L.oracle_gauss_legendre.restype = None
        L.oracle_gauss_legendre.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_set_hex_rule.restype = None
        L.oracle_set_hex_rule.argtypes = [ctypes.c_int32]
        L.oracle_set_tp_element.restype = None
        L.oracle_set_tp_element.argtypes = [ctypes.c_int32, ctypes.c_int32]
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def derive_edges(cells: np.ndarray, nverts: int) -> tuple[np.ndarray, int]:
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.empty_like(cells)
    n = lib().oracle_derive_edges(cells.shape[1], cells.shape[0], _p(cells), nverts, _p(out))
    if n < 0:
        raise ValueError("invalid cell-vertex list")
    return out, int(n)


@dataclass
class Space:
    """Oracle numbering of one function space on an extruded mesh."""

    delta: tuple
    layers: int
    ndofs: int
    k: int
    map: np.ndarray       # (C, k) int32, layer-0 explicit lists
    offset: np.ndarray    # (k,) int32, Algorithm 2
    first: dict = field(default_factory=dict)  # t=2*d1+d2 -> (N_d1, layers+1-d2) int64


def entity_counts(cells: np.ndarray, nverts: int) -> tuple[int, int, int, np.ndarray]:
    ce, ne = derive_edges(cells, nverts)
    return nverts, ne, cells.shape[0], ce


def number(cells: np.ndarray, nverts: int, layers: int, delta, keep_tables: bool = False) -> Space:
    """Algorithm 1 + explicit lists + Algorithm 2 for one space."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    delta = tuple(int(x) for x in delta)
    d = np.array(delta, dtype=np.int32)
    nvc = cells.shape[1]
    ce, ne = derive_edges(cells, nverts)
    N = np.array([nverts, ne, cells.shape[0]], dtype=np.int64)
    L = lib()
    nul = (ctypes.c_void_p * 6)()
    if L.oracle_alg1(_p(N), layers, _p(d), nul) >= 2**31:
        raise OverflowError("DoF count does not fit int32")
    tabs = []
    ptrs = (ctypes.c_void_p * 6)()
    for t in range(6):
        d1, d2 = divmod(t, 2)
        if delta[t] > 0:
            a = np.full((int(N[d1]), layers + 1 - d2), -1, dtype=np.int64)
            tabs.append(a)
            ptrs[t] = a.ctypes.data
        else:
            tabs.append(None)
            ptrs[t] = None
    ndofs = L.oracle_alg1(_p(N), layers, _p(d), ptrs)
    k = L.oracle_stencil_size(nvc, _p(d))
    m = np.empty((cells.shape[0], k), dtype=np.int32)
    rc = L.oracle_base_map(nvc, cells.shape[0], _p(cells), _p(ce), layers, _p(d), ptrs, _p(m))
    if rc != 0:
        raise ValueError("oracle_base_map failed")
    off = np.empty(k, dtype=np.int32)
    L.oracle_alg2(nvc, _p(d), _p(off))
    first = {t: tabs[t] for t in range(6) if tabs[t] is not None} if keep_tables else {}
    return Space(delta=delta, layers=layers, ndofs=int(ndofs), k=int(k), map=m, offset=off, first=first)


def par_loop(kernel: int, cells: np.ndarray, layers: int, args, base_xy: np.ndarray | None = None,
             ncells: int | None = None) -> None:
    """Algorithm 3 over the first ``ncells`` cells (all by default).

    ``args`` is a list of (Space, data ndarray float64, ncomp, access[, absdata]).
    Data arrays are updated in place.
    """
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    n = cells.shape[0] if ncells is None else int(ncells)
    arr = (_Arg * len(args))()
    keep = []
    for i, a in enumerate(args):
        sp, data, ncomp, acc = a[:4]
        absd = a[4] if len(a) > 4 else None
        assert data.dtype == np.float64 and data.flags.c_contiguous
        assert data.size == sp.ndofs * ncomp, (data.size, sp.ndofs, ncomp)
        if absd is not None:
            assert absd.dtype == np.float64 and absd.size == data.size and absd.flags.c_contiguous
        keep += [sp.map, sp.offset]
        arr[i].map = sp.map.ctypes.data
        arr[i].offset = sp.offset.ctypes.data
        arr[i].k = sp.k
        arr[i].ncomp = ncomp
        arr[i].data = data.ctypes.data
        arr[i].absdata = None if absd is None else absd.ctypes.data
        arr[i].access = acc
    xy = None if base_xy is None else np.ascontiguousarray(base_xy, dtype=np.float64)
    rc = lib().oracle_par_loop(kernel, cells.shape[1], n, layers, _p(cells), _p(xy), len(args), arr)
    if rc != 0:
        raise RuntimeError(f"oracle_par_loop failed: {rc}")


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    x = np.empty(n)
    w = np.empty(n)
    lib().oracle_gauss_legendre(n, _p(x), _p(w))
    return x, w


def set_hex_rule(n: int) -> None:
    lib().oracle_set_hex_rule(n)


def set_tp_element(h: int, v: int) -> None:
    """Horizontal and vertical element (CG1, DG0, DG1) of K_MASS_TP."""
    lib().oracle_set_tp_element(h, v)


# the nine prism spaces of the paper's Sec. 4.1.2 as (name, h, v)
TP_PAIRS = [(f"{a}x{b}", ha, vb) for a, ha in (("CG1", CG1), ("DG0", DG0), ("DG1", DG1))
            for b, vb in (("CG1", CG1), ("DG0", DG0), ("DG1", DG1))]


# ---------------------------------------------------------------------------
# Convenience: whole workloads as the tests and the CPU baseline use them.
# ---------------------------------------------------------------------------

def coords(cells: np.ndarray, xy: np.ndarray, layers: int) -> tuple[Space, np.ndarray]:
    """Coordinate space (CG1xCG1, 3 values per DoF) and its extruded field."""
    sp = number(cells, xy.shape[0], layers, DELTA["CG1xCG1"])
    X = np.zeros(sp.ndofs * 3)
    par_loop(K_EXTRUDE, cells, layers, [(sp, X, 3, WRITE)], base_xy=xy)
    return sp, X
