"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds input generation only: base meshes (perturbed structured
triangulations and quadrilateral grids of the unit square), their vertex/cell
orderings, uniform random fields and the per-mesh parameters of the batched
workload.  It contains none of the method's arithmetic (no numbering, no
stencil maps, no quadrature): every array it returns is consumed by both the
oracle and the CUDA library, which each apply their own implementation of the
method to it.

The paper's meshes were unstructured Gmsh meshes of the unit square extruded
to the unit cube (Sec. 4.1.1); they are not available, so a structured grid
with randomly flipped diagonals and jittered interior vertices stands in for
them.  The ordering experiment of Sec. 4.1.4 (reverse Cuthill-McKee versus a
random permutation) is reproduced by the ``order`` argument.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "BaseMesh",
    "tri_mesh",
    "quad_mesh",
    "uniform_field",
    "batched_params",
    "BatchedParams",
]


@dataclass
class BaseMesh:
    """A 2-D base mesh: ``xy`` is (V, 2) float64, ``cells`` is (C, nv) int32 CCW."""

    xy: np.ndarray
    cells: np.ndarray
    n: int
    order: str
    seed: int

    @property
    def nverts(self) -> int:
        return int(self.xy.shape[0])

    @property
    def ncells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def kind(self) -> int:
        """Vertices per cell: 3 (triangle) or 4 (quadrilateral)."""
        return int(self.cells.shape[1])


def _grid_vertices(n: int, rng: np.random.Generator, jitter: float) -> np.ndarray:
    """(n+1)^2 vertices of the unit square, interior ones jittered by
    U(-1,1)*jitter*spacing in x and y; boundary vertices stay on the boundary
    so the extruded domain is exactly the unit cube."""
    s = 1.0 / n
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    x = (i * s).astype(np.float64).ravel()
    y = (j * s).astype(np.float64).ravel()
    d = rng.uniform(-1.0, 1.0, size=(2, (n + 1) * (n + 1))) * (jitter * s)
    interior = ((i > 0) & (i < n) & (j > 0) & (j < n)).ravel()
    x[interior] += d[0, interior]
    y[interior] += d[1, interior]
    return np.stack([x, y], axis=1)


def _reorder(xy: np.ndarray, cells: np.ndarray, order: str,
             rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Renumber vertices and cells.

    ``rcm``: reverse Cuthill-McKee over the vertex adjacency graph, then cells
    sorted lexicographically by their sorted (new) vertex ids.
    ``random``: seeded random permutations of vertices and of cells.
    ``natural``: generation order.
    The local vertex order inside each cell (its orientation) is never changed.
    """
    nv = xy.shape[0]
    if order == "natural":
        return xy, cells
    if order == "rcm":
        from scipy.sparse import coo_matrix
        from scipy.sparse.csgraph import reverse_cuthill_mckee

        k = cells.shape[1]
        rows, cols = [], []
        for a in range(k):
            for b in range(k):
                if a != b:
                    rows.append(cells[:, a])
                    cols.append(cells[:, b])
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        g = coo_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(nv, nv)).tocsr()
        perm = reverse_cuthill_mckee(g, symmetric_mode=True)  # new -> old
        new_of_old = np.empty(nv, dtype=np.int64)
        new_of_old[perm] = np.arange(nv)
        xy2 = xy[perm]
        cells2 = new_of_old[cells]
        key = np.sort(cells2, axis=1)
        idx = np.lexsort(tuple(key[:, a] for a in range(key.shape[1] - 1, -1, -1)))
        return xy2, cells2[idx].astype(np.int32)
    if order == "random":
        perm = rng.permutation(nv)  # new -> old
        new_of_old = np.empty(nv, dtype=np.int64)
        new_of_old[perm] = np.arange(nv)
        cells2 = new_of_old[cells][rng.permutation(cells.shape[0])]
        return xy[perm], cells2.astype(np.int32)
    raise ValueError(f"unknown order {order!r}")


def tri_mesh(n: int, seed: int = 1604, order: str = "rcm", jitter: float = 0.2) -> BaseMesh:
    """Perturbed structured triangulation of the unit square.

    n x n squares, each split along a diagonal chosen by a fair coin, giving
    C = 2 n^2 triangles and V = (n+1)^2 vertices.  Triangles are CCW.
    """
    rng = np.random.default_rng(seed)
    xy = _grid_vertices(n, rng, jitter)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    p00 = j * (n + 1) + i
    p10 = p00 + 1
    p01 = p00 + (n + 1)
    p11 = p01 + 1
    flip = rng.random(n * n) < 0.5
    t0 = np.where(flip[:, None], np.stack([p00, p10, p01], 1), np.stack([p00, p10, p11], 1))
    t1 = np.where(flip[:, None], np.stack([p10, p11, p01], 1), np.stack([p00, p11, p01], 1))
    cells = np.empty((2 * n * n, 3), dtype=np.int64)
    cells[0::2] = t0
    cells[1::2] = t1
    xy, cells = _reorder(xy, cells, order, rng)
    m = BaseMesh(xy=np.ascontiguousarray(xy), cells=np.ascontiguousarray(cells, dtype=np.int32),
                 n=n, order=order, seed=seed)
    _check_orientation(m)
    return m


def quad_mesh(n: int, seed: int = 1604, order: str = "rcm", jitter: float = 0.2) -> BaseMesh:
    """Jittered n x n quadrilateral grid of the unit square (C = n^2, V = (n+1)^2),
    vertices of each quad CCW starting from its lower-left corner."""
    rng = np.random.default_rng(seed)
    xy = _grid_vertices(n, rng, jitter)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    p00 = (j * (n + 1) + i).ravel()
    cells = np.stack([p00, p00 + 1, p00 + n + 2, p00 + n + 1], axis=1)
    xy, cells = _reorder(xy, cells, order, rng)
    m = BaseMesh(xy=np.ascontiguousarray(xy), cells=np.ascontiguousarray(cells, dtype=np.int32),
                 n=n, order=order, seed=seed)
    _check_orientation(m)
    return m


def _check_orientation(m: BaseMesh) -> None:
    """Every corner of every cell turns left (positive orientation, convex)."""
    p = m.xy[m.cells]  # (C, k, 2)
    k = p.shape[1]
    for a in range(k):
        u = p[:, (a + 1) % k] - p[:, a]
        v = p[:, (a + k - 1) % k] - p[:, a]
        cross = u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]
        if not np.all(cross > 0):
            raise AssertionError("generated cell is not positively oriented")


def uniform_field(size: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded U(lo, hi) float64 values (a random nodal field in any numbering)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=size).astype(np.float64)


@dataclass
class BatchedParams:
    """Per-mesh sizes of the batched workload: grid size n (C = 2 n^2) and layers."""

    n: list
    layers: list
    seed: int

    @property
    def ncells(self) -> list:
        return [2 * k * k for k in self.n]


def batched_params(count: int = 64, seed: int = 1605, cmin: float = 1e4, cmax: float = 5e5,
                   lmin: int = 8, lmax: int = 256) -> BatchedParams:
    """Base cell counts log-uniform on [cmin, cmax] (realised as n = round(sqrt(C/2))),
    layer counts uniform on {lmin..lmax}."""
    rng = np.random.default_rng(seed)
    c = np.exp(rng.uniform(math.log(cmin), math.log(cmax), size=count))
    n = [max(1, int(round(math.sqrt(x / 2.0)))) for x in c]
    layers = [int(v) for v in rng.integers(lmin, lmax + 1, size=count)]
    return BatchedParams(n=n, layers=layers, seed=seed)


def column_layers(m: BaseMesh, maxlevel: int, seed: int, kind: str = "bathymetry") -> tuple[np.ndarray, np.ndarray]:
    """Per-column layer ranges (first level, layer count), int32, for meshes
    with a variable number of layers per column.

    ``bathymetry``: a smooth depth field d(x, y) in [0.15, 0.95] over the
    base (evaluated at cell centroids); column c has round(d * maxlevel)
    layers (at least 1) hanging from a flat top at ``maxlevel`` (an ocean-like
    terrain-following layout, so neighbouring columns overlap and no entity
    column has a gap).  ``random``: independent random ranges inside
    [0, maxlevel], which may leave gaps between neighbouring columns."""
    rng = np.random.default_rng(seed)
    if kind == "random":
        first = rng.integers(0, maxlevel, m.ncells)
        lay = 1 + rng.integers(0, maxlevel - first)
        return first.astype(np.int32), lay.astype(np.int32)
    if kind != "bathymetry":
        raise ValueError(kind)
    ph = rng.uniform(0.0, 2.0 * np.pi, 2)
    cxy = m.xy[m.cells].mean(axis=1)
    depth = 0.55 + 0.4 * np.sin(3.0 * cxy[:, 0] + ph[0]) * np.cos(2.0 * cxy[:, 1] + ph[1])
    lay = np.clip(np.rint(depth * maxlevel), 1, maxlevel).astype(np.int32)
    return (maxlevel - lay).astype(np.int32), lay


def level_coords(m: BaseMesh, layers: int, seed: int, kind: str = "terrain") -> np.ndarray:
    """Coordinates of every (base vertex, level) pair, float64, shape
    (nverts, layers + 1, 3), for geometries other than the flat unit-height
    extrusion.

    ``terrain``: terrain-following levels over a smooth depth field
    d(x, y) = 0.55 + 0.4 sin(3x + p1) cos(2y + p2) in [0.15, 0.95]: the vertex
    at level l sits at (x, y, (l / layers) d(x, y)), so every column is
    vertical and no two vertices of a prism's top face (away from symmetric
    points) share a height.  ``wavy``: the same with the levels bent by
    0.3 / layers sin(7x + 5y) sin(pi l / layers), so that the heights are no
    longer a fixed profile scaled per column.  ``tilted``: the terrain levels
    with x and y sheared with height, x + 0.05 z sin(2 pi y) and
    y + 0.05 z cos(2 pi x), so the columns lean as well.  The phases come
    from ``seed``."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * np.pi, 2)
    x, y = m.xy[:, 0], m.xy[:, 1]
    depth = 0.55 + 0.4 * np.sin(3.0 * x + ph[0]) * np.cos(2.0 * y + ph[1])
    lev = np.arange(layers + 1, dtype=np.float64) / float(layers)
    out = np.empty((m.nverts, layers + 1, 3))
    out[:, :, 0] = x[:, None]
    out[:, :, 1] = y[:, None]
    out[:, :, 2] = lev[None, :] * depth[:, None]
    if kind == "wavy":
        out[:, :, 2] += (0.3 / layers) * np.sin(7.0 * x + 5.0 * y)[:, None] * np.sin(np.pi * lev)[None, :]
    elif kind == "tilted":
        z = out[:, :, 2]
        out[:, :, 0] = x[:, None] + 0.05 * z * np.sin(2.0 * np.pi * y)[:, None]
        out[:, :, 1] = y[:, None] + 0.05 * z * np.cos(2.0 * np.pi * x)[:, None]
    elif kind != "terrain":
        raise ValueError(kind)
    return out


def padaptive_dent(m: BaseMesh, nedges: int, seed: int, kind: str = "disk") -> np.ndarray:
    """Per-entity DoF counts ((V + E + C) x 2, dimension-major) of a p-adaptive
    DG space: DoFs only inside the cells, each cell one of DG0xDG0 (1),
    DG0xDG1 (2), DG1xDG0 (3), DG1xDG1 (6).  ``disk``: DG1xDG1 in the cells
    whose centroid lies within 0.3 of (0.5, 0.5) (about 28 % of the cells),
    DG0xDG0 elsewhere; ``mixed``: the four kinds drawn uniformly."""
    rng = np.random.default_rng(seed)
    dent = np.zeros((m.nverts + nedges + m.ncells, 2), dtype=np.int32)
    if kind == "mixed":
        k = rng.choice(np.array([1, 2, 3, 6], dtype=np.int32), m.ncells)
    elif kind == "disk":
        c = m.xy[m.cells].mean(axis=1)
        k = np.where(((c[:, 0] - 0.5) ** 2 + (c[:, 1] - 0.5) ** 2) < 0.09, 6, 1).astype(np.int32)
    else:
        raise ValueError(kind)
    dent[m.nverts + nedges:, 1] = k
    return dent
