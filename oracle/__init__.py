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
(K_EXTRUDE, K_COPY, K_MASS, K_INTERP, K_U2V, K_U2V_ADJ, K_MASS_TP, K_HFACET_MASS, K_HFACET_JUMP,
 K_MASS_DGP) = range(10)
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
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    # OpenMP only spreads the coloured CPU-baseline loop over cores; without
    # it that loop runs on one thread and everything else is unchanged
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.check_call(base)
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
        ("rowptr", ctypes.c_void_p),
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
        L.oracle_color_cells.restype = ctypes.c_int32
        L.oracle_color_cells.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p]
        L.oracle_max_threads.restype = ctypes.c_int32
        L.oracle_max_threads.argtypes = []
        L.oracle_par_loop_colored.restype = ctypes.c_int
        L.oracle_par_loop_colored.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        L.oracle_par_loop.restype = ctypes.c_int
        L.oracle_par_loop.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        L.oracle_gauss_legendre.restype = None
        L.oracle_gauss_legendre.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_set_hex_rule.restype = None
        L.oracle_set_hex_rule.argtypes = [ctypes.c_int32]
        L.oracle_set_tp_element.restype = None
        L.oracle_set_tp_element.argtypes = [ctypes.c_int32, ctypes.c_int32]
        L.oracle_var_ranges.restype = ctypes.c_int
        L.oracle_var_ranges.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_alg1_var.restype = ctypes.c_int64
        L.oracle_alg1_var.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_base_map_var.restype = ctypes.c_int
        L.oracle_base_map_var.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
        L.oracle_hfacet_size.restype = ctypes.c_int32
        L.oracle_hfacet_size.argtypes = [ctypes.c_int32, ctypes.c_void_p]
        L.oracle_hfacet_map.restype = ctypes.c_int
        L.oracle_hfacet_map.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.oracle_hfacet_alg2.restype = None
        L.oracle_hfacet_alg2.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_alg1_ragged.restype = ctypes.c_int64
        L.oracle_alg1_ragged.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_ragged_map.restype = ctypes.c_int
        L.oracle_ragged_map.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_par_loop_var.restype = ctypes.c_int
        L.oracle_par_loop_var.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p]
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
    hmap: np.ndarray | None = None     # (C, hk) horizontal-facet lists (closure DoFs), if any
    hoffset: np.ndarray | None = None  # (hk,) their offsets
    cell_first: np.ndarray | None = None   # variable layers: first level of each column
    cell_layers: np.ndarray | None = None  # variable layers: layers of each column
    rowptr: np.ndarray | None = None       # ragged lists: cell c's entries are map[rowptr[c]:rowptr[c+1]]

    def facet(self) -> "Space":
        """The same numbering seen through the horizontal-facet lists."""
        if self.hmap is None:
            raise ValueError("the space has no DoFs on horizontal facets")
        return Space(delta=self.delta, layers=self.layers, ndofs=self.ndofs, k=int(self.hmap.shape[1]),
                     map=self.hmap, offset=self.hoffset, cell_first=self.cell_first,
                     cell_layers=self.cell_layers)


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
    hmap, hoff = _facet_lists(cells, ce, layers, None, d, ptrs)
    return Space(delta=delta, layers=layers, ndofs=int(ndofs), k=int(k), map=m, offset=off, first=first,
                 hmap=hmap, hoffset=hoff)


def _facet_lists(cells, ce, maxlevel, cell_first, d, ptrs):
    nvc = cells.shape[1]
    L = lib()
    hk = L.oracle_hfacet_size(nvc, _p(d))
    if hk == 0:
        return None, None
    hm = np.empty((cells.shape[0], hk), dtype=np.int32)
    if L.oracle_hfacet_map(nvc, cells.shape[0], _p(cells), _p(ce), maxlevel, _p(cell_first), _p(d), ptrs,
                           _p(hm)) != 0:
        raise ValueError("oracle_hfacet_map failed")
    ho = np.empty(hk, dtype=np.int32)
    L.oracle_hfacet_alg2(nvc, _p(d), _p(ho))
    return hm, ho


def var_ranges(cells: np.ndarray, nverts: int, cell_first, cell_layers):
    """Level ranges (lo, hi) of every base entity, dimension-major."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    ce, ne = derive_edges(cells, nverts)
    cf = np.ascontiguousarray(cell_first, dtype=np.int32)
    cl = np.ascontiguousarray(cell_layers, dtype=np.int32)
    N = np.array([nverts, ne, cells.shape[0]], dtype=np.int64)
    lo = np.empty(int(N.sum()), dtype=np.int32)
    hi = np.empty_like(lo)
    rc = lib().oracle_var_ranges(cells.shape[1], _p(N), _p(cells), _p(ce), _p(cf), _p(cl), _p(lo), _p(hi))
    if rc != 0:
        raise ValueError(f"oracle_var_ranges failed: {rc}")
    return lo, hi, N, ce


def number_var(cells: np.ndarray, nverts: int, cell_first, cell_layers, delta,
               keep_tables: bool = False) -> Space:
    """Algorithm 1 with a variable number of layers per column."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    delta = tuple(int(x) for x in delta)
    d = np.array(delta, dtype=np.int32)
    cf = np.ascontiguousarray(cell_first, dtype=np.int32)
    cl = np.ascontiguousarray(cell_layers, dtype=np.int32)
    lo, hi, N, ce = var_ranges(cells, nverts, cf, cl)
    maxlevel = int((cf + cl).max())
    nvc = cells.shape[1]
    L = lib()
    nul = (ctypes.c_void_p * 6)()
    if L.oracle_alg1_var(_p(N), maxlevel, _p(lo), _p(hi), _p(d), nul) >= 2**31:
        raise OverflowError("DoF count does not fit int32")
    tabs = []
    ptrs = (ctypes.c_void_p * 6)()
    for t in range(6):
        d1, d2 = divmod(t, 2)
        if delta[t] > 0:
            a = np.full((int(N[d1]), maxlevel + 1 - d2), -1, dtype=np.int64)
            tabs.append(a)
            ptrs[t] = a.ctypes.data
        else:
            tabs.append(None)
            ptrs[t] = None
    ndofs = L.oracle_alg1_var(_p(N), maxlevel, _p(lo), _p(hi), _p(d), ptrs)
    k = L.oracle_stencil_size(nvc, _p(d))
    m = np.empty((cells.shape[0], k), dtype=np.int32)
    if L.oracle_base_map_var(nvc, cells.shape[0], _p(cells), _p(ce), maxlevel, _p(cf), _p(d), ptrs, _p(m)) != 0:
        raise ValueError("oracle_base_map_var failed")
    off = np.empty(k, dtype=np.int32)
    L.oracle_alg2(nvc, _p(d), _p(off))
    first = {t: tabs[t] for t in range(6) if tabs[t] is not None} if keep_tables else {}
    hmap, hoff = _facet_lists(cells, ce, maxlevel, cf, d, ptrs)
    return Space(delta=delta, layers=maxlevel, ndofs=int(ndofs), k=int(k), map=m, offset=off, first=first,
                 hmap=hmap, hoffset=hoff, cell_first=cf, cell_layers=cl)


def par_loop(kernel: int, cells: np.ndarray, layers: int, args, base_xy: np.ndarray | None = None,
             ncells: int | None = None, cell_first=None, cell_layers=None) -> None:
    """Algorithm 3 over the first ``ncells`` cells (all by default).

    ``args`` is a list of (Space, data ndarray float64, ncomp, access[, absdata]).
    Data arrays are updated in place.  With ``cell_first``/``cell_layers``
    the columns have variable layers and ``layers`` is the highest level.
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
        keep += [sp.map, sp.offset, sp.rowptr]
        arr[i].map = sp.map.ctypes.data
        arr[i].offset = sp.offset.ctypes.data
        arr[i].rowptr = None if sp.rowptr is None else sp.rowptr.ctypes.data
        arr[i].k = sp.k
        arr[i].ncomp = ncomp
        arr[i].data = data.ctypes.data
        arr[i].absdata = None if absd is None else absd.ctypes.data
        arr[i].access = acc
    xy = None if base_xy is None else np.ascontiguousarray(base_xy, dtype=np.float64)
    if cell_first is None:
        rc = lib().oracle_par_loop(kernel, cells.shape[1], n, layers, _p(cells), _p(xy), len(args), arr)
    else:
        cf = np.ascontiguousarray(cell_first, dtype=np.int32)
        cl = np.ascontiguousarray(cell_layers, dtype=np.int32)
        rc = lib().oracle_par_loop_var(kernel, cells.shape[1], n, _p(cf), _p(cl), layers, _p(cells), _p(xy),
                                       len(args), arr)
    if rc != 0:
        raise RuntimeError(f"oracle_par_loop failed: {rc}")


def _args_array(args):
    arr = (_Arg * len(args))()
    keep = []
    for i, a in enumerate(args):
        sp, data, ncomp, acc = a[:4]
        absd = a[4] if len(a) > 4 else None
        assert data.dtype == np.float64 and data.flags.c_contiguous
        assert data.size == sp.ndofs * ncomp, (data.size, sp.ndofs, ncomp)
        keep += [sp.map, sp.offset]
        arr[i].map = sp.map.ctypes.data
        arr[i].offset = sp.offset.ctypes.data
        arr[i].rowptr = None
        arr[i].k = sp.k
        arr[i].ncomp = ncomp
        arr[i].data = data.ctypes.data
        arr[i].absdata = None if absd is None else absd.ctypes.data
        arr[i].access = acc
    return arr, keep


def color_cells(cells: np.ndarray, nverts: int) -> tuple[np.ndarray, np.ndarray]:
    """Greedy vertex-disjoint colouring of base cells (in cell order):
    (color_ptr of ncolors + 1 offsets, cells grouped by colour, ascending)."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    col = np.empty(cells.shape[0], dtype=np.int32)
    nc = lib().oracle_color_cells(cells.shape[1], cells.shape[0], _p(cells), nverts, _p(col))
    if nc < 0:
        raise RuntimeError(f"oracle_color_cells failed: {nc}")
    order = np.argsort(col, kind="stable").astype(np.int64)
    ptr = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(np.bincount(col, minlength=nc), out=ptr[1:])
    return ptr, np.ascontiguousarray(order)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def par_loop_colored(kernel: int, cells: np.ndarray, layers: int, args, color_ptr, color_cells_,
                     nthreads: int | None = None) -> None:
    """Algorithm 3 over the listed cells on several host cores: colours in
    sequence, the cells of one colour (no shared vertex) split over threads.
    A CPU baseline; the checks use the serial par_loop."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    arr, keep = _args_array(args)
    ptr = np.ascontiguousarray(color_ptr, dtype=np.int64)
    ids = np.ascontiguousarray(color_cells_, dtype=np.int64)
    rc = lib().oracle_par_loop_colored(kernel, cells.shape[1], layers, _p(cells), None, len(args), arr,
                                       ptr.size - 1, _p(ptr), _p(ids), nthreads or max_threads())
    if rc != 0:
        raise RuntimeError(f"oracle_par_loop_colored failed: {rc}")


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


def coords_var(cells: np.ndarray, xy: np.ndarray, cell_first, cell_layers) -> tuple[Space, np.ndarray]:
    """Coordinate space and field of a mesh with variable layers per column
    (z = level / highest level)."""
    sp = number_var(cells, xy.shape[0], cell_first, cell_layers, DELTA["CG1xCG1"])
    X = np.zeros(sp.ndofs * 3)
    par_loop(K_EXTRUDE, cells, sp.layers, [(sp, X, 3, WRITE)], base_xy=xy,
             cell_first=sp.cell_first, cell_layers=sp.cell_layers)
    return sp, X


def number_ragged(cells: np.ndarray, nverts: int, dent, layers: int | None = None, cell_first=None,
                  cell_layers=None, keep_tables: bool = False) -> Space:
    """Algorithm 1 with per-entity DoF counts dent ((V + E + C) x 2:
    horizontal, vertical; entities dimension-major), on constant layers or
    per-column layer ranges.  The lists are ragged (Space.rowptr)."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    dent = np.ascontiguousarray(dent, dtype=np.int32).reshape(-1)
    ce, ne = derive_edges(cells, nverts)
    N = np.array([nverts, ne, cells.shape[0]], dtype=np.int64)
    nent = int(N.sum())
    if dent.size != 2 * nent:
        raise ValueError(f"dent needs {nent} x 2 entries")
    if cell_layers is None:
        cf = np.zeros(cells.shape[0], np.int32)
        cl = np.full(cells.shape[0], int(layers), np.int32)
    else:
        cf = np.ascontiguousarray(cell_first, dtype=np.int32)
        cl = np.ascontiguousarray(cell_layers, dtype=np.int32)
    lo, hi, _, _ = var_ranges(cells, nverts, cf, cl)
    maxlevel = int((cf + cl).max())
    L = lib()
    tabs, ptrs = [], (ctypes.c_void_p * 6)()
    for t in range(6):
        d1, d2 = divmod(t, 2)
        a = np.full((int(N[d1]), maxlevel + 1 - d2), -1, dtype=np.int64)
        tabs.append(a)
        ptrs[t] = a.ctypes.data
    ndofs = L.oracle_alg1_ragged(_p(N), maxlevel, _p(lo), _p(hi), _p(dent), ptrs)
    if ndofs >= 2**31:
        raise OverflowError("DoF count does not fit int32")
    rowptr = np.zeros(cells.shape[0] + 1, dtype=np.int64)
    if L.oracle_ragged_map(cells.shape[1], cells.shape[0], _p(cells), _p(ce), maxlevel, _p(cf), _p(N), _p(dent),
                           ptrs, _p(rowptr), None, None) != 0:
        raise ValueError("oracle_ragged_map failed")
    m = np.empty(int(rowptr[-1]), dtype=np.int32)
    off = np.empty(int(rowptr[-1]), dtype=np.int32)
    L.oracle_ragged_map(cells.shape[1], cells.shape[0], _p(cells), _p(ce), maxlevel, _p(cf), _p(N), _p(dent),
                        ptrs, _p(rowptr), _p(m), _p(off))
    first = {t: tabs[t] for t in range(6)} if keep_tables else {}
    return Space(delta=None, layers=maxlevel, ndofs=int(ndofs), k=0, map=m, offset=off, first=first,
                 cell_first=None if cell_layers is None else cf, cell_layers=None if cell_layers is None else cl,
                 rowptr=rowptr)


def dent_of(cells: np.ndarray, nverts: int, delta) -> np.ndarray:
    """Per-entity counts of a constant-delta space (for comparisons)."""
    _, ne = derive_edges(cells, nverts)
    N = [nverts, ne, cells.shape[0]]
    return np.concatenate([np.tile(np.array([delta[2 * d], delta[2 * d + 1]], np.int32), (N[d], 1))
                           for d in range(3)])
