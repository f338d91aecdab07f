"""Pins of the oracle's horizontal-facet loops (Algorithm 3 with d2 = 0: the
facets at levels 0..lambda of each column) and of the interior-facet jump
term: facet lists against the pinned cell lists, surface areas and linear
moments in closed form, the P1 surface mass matrix of a triangle, a tilted
facet, and the jump term against int_F [u]^2 written out for constant and
linear traces."""
import numpy as np
import pytest

import meshgen
import oracle as O

FACET_SPACES = [("CG1xCG1", O.CG1), ("DG0xCG1", O.DG0), ("DG1xCG1", O.DG1)]
JUMP_SPACES = [(nm, h, v) for nm, h, v in O.TP_PAIRS]


def _areas_centroids(m):
    p = m.xy[m.cells]
    A = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    return A, p.mean(axis=1)


@pytest.mark.parametrize("name", ["CG1xCG1", "DG0xCG1", "DG1xCG1", "Q2xP2", "CG1xDG1"])
def test_facet_lists_are_cell_faces(name):
    """Facet l of a column holds the bottom horizontal DoFs of layer l (and the
    top ones of the last layer): the lists and offsets agree with the cell
    lists at every level."""
    m = meshgen.quad_mesh(4, seed=2) if name == "Q2xP2" else meshgen.tri_mesh(4, seed=2)
    L = 5
    sp = O.number(m.cells, m.nverts, L, O.DELTA[name])
    if name == "CG1xDG1":
        assert sp.hmap is None       # no DoFs on horizontal facets
        return
    fs = sp.facet()
    # bottom / top slots of the cell list, entity by entity
    bot, top, j = [], [], 0
    for d in range(3):
        a, b = sp.delta[2 * d], sp.delta[2 * d + 1]
        for _ in range(1 if d == 2 else m.kind):
            bot += list(range(j, j + a))
            top += list(range(j + a, j + 2 * a))
            j += 2 * a + b
    for l in range(L + 1):
        got = fs.map.astype(np.int64) + l * fs.offset
        if l < L:
            want = sp.map[:, bot].astype(np.int64) + l * sp.offset[bot]
        else:
            want = sp.map[:, top].astype(np.int64) + (L - 1) * sp.offset[top]
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("name,h", FACET_SPACES)
@pytest.mark.parametrize("var", [False, True])
def test_facet_area_sum(name, h, var):
    m = meshgen.tri_mesh(5, seed=3)
    A, _ = _areas_centroids(m)
    O.set_tp_element(h, O.CG1)
    if var:
        rng = np.random.default_rng(4)
        first = rng.integers(0, 4, m.ncells).astype(np.int32)
        lay = (1 + rng.integers(0, 5 - first)).astype(np.int32)
        cs, X = O.coords_var(m.cells, m.xy, first, lay)
        sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
        want = float((A * (lay + 1)).sum())
        kw = dict(cell_first=first, cell_layers=lay)
    else:
        cs, X = O.coords(m.cells, m.xy, 4)
        sp = O.number(m.cells, m.nverts, 4, O.DELTA[name])
        want = 5.0                      # five levels of the unit square
        kw = {}
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_HFACET_MASS, m.cells, sp.layers, [(cs.facet(), X, 3, O.READ),
               (sp.facet(), np.ones(sp.ndofs), 1, O.READ), (sp.facet(), b, 1, O.INC)], **kw)
    assert abs(b.sum() - want) <= 1e-13 * want


def test_facet_linear_moment():
    m = meshgen.tri_mesh(5, seed=5)
    L = 3
    cs, X = O.coords(m.cells, m.xy, L)
    sp = O.number(m.cells, m.nverts, L, O.DELTA["CG1xCG1"])
    O.set_tp_element(O.CG1, O.CG1)
    f = X.reshape(-1, 3).sum(axis=1)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_HFACET_MASS, m.cells, L, [(cs.facet(), X, 3, O.READ), (sp.facet(), f, 1, O.READ),
                                             (sp.facet(), b, 1, O.INC)])
    A, cen = _areas_centroids(m)
    want = sum(float((A * (cen[:, 0] + cen[:, 1] + l / L)).sum()) for l in range(L + 1))
    assert abs(b.sum() - want) <= 1e-13 * want


def _one_prism(xy, layers):
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    cs, X = O.coords(cells, np.asarray(xy, dtype=float), layers)
    return cells, cs, X


def test_facet_element_matrix_closed_form():
    """P1 surface mass on a flat triangle: A/12 (1 + [a = b]); DG0: A."""
    xy = [[0.1, 0.2], [1.3, 0.4], [0.5, 1.7]]
    cells, cs, X = _one_prism(xy, 1)
    A = 0.5 * abs((1.3 - 0.1) * (1.7 - 0.2) - (0.5 - 0.1) * (0.4 - 0.2))
    Mh = A / 12.0 * (np.ones((3, 3)) + np.eye(3))
    rng = np.random.default_rng(6)
    for name, h in FACET_SPACES:
        O.set_tp_element(h, O.CG1)
        sp = O.number(cells, 3, 1, O.DELTA[name])
        f = rng.standard_normal(sp.ndofs)
        b = np.zeros(sp.ndofs)
        O.par_loop(O.K_HFACET_MASS, cells, 1, [(cs.facet(), X, 3, O.READ), (sp.facet(), f, 1, O.READ),
                                               (sp.facet(), b, 1, O.INC)])
        for lev in range(2):
            idx = sp.hmap[0].astype(np.int64) + lev * sp.hoffset
            want = A * f[idx] if h == O.DG0 else Mh @ f[idx]
            np.testing.assert_allclose(b[idx], want, rtol=1e-14, atol=1e-15)


def test_tilted_facet_area():
    cells, cs, X = _one_prism([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0]], 1)
    Xr = X.reshape(-1, 3)
    # lift vertex 1 by 1 and vertex 2 by 2 at both levels: each facet has edge
    # vectors (1, 0, 1) and (0.5, 1, 2), normal (-1, -1.5, 1), area sqrt(17)/4
    for a, dz in ((1, 1.0), (2, 2.0)):
        Xr[cs.map[0, 2 * a]] += [0.0, 0.0, dz]
        Xr[cs.map[0, 2 * a + 1]] += [0.0, 0.0, dz]
    sp = O.number(cells, 3, 1, O.DELTA["CG1xCG1"])
    O.set_tp_element(O.CG1, O.CG1)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_HFACET_MASS, cells, 1, [(cs.facet(), X, 3, O.READ), (sp.facet(), np.ones(sp.ndofs), 1, O.READ),
                                           (sp.facet(), b, 1, O.INC)])
    assert abs(b.sum() - np.sqrt(17.0) / 2.0) <= 1e-15     # two facets


def _jump(m, L, name, h, v, u, X=None, cs=None, **kw):
    if cs is None:
        cs, X = O.coords(m.cells, m.xy, L)
    sp = O.number(m.cells, m.nverts, L, O.DELTA[name]) if not kw else \
        O.number_var(m.cells, m.nverts, kw["cell_first"], kw["cell_layers"], O.DELTA[name])
    O.set_tp_element(h, v)
    r = np.zeros(sp.ndofs)
    ab = np.zeros(sp.ndofs)
    O.par_loop(O.K_HFACET_JUMP, m.cells, sp.layers, [(cs, X, 3, O.READ), (sp, u(sp), 1, O.READ),
                                                     (sp, r, 1, O.INC, ab)], **kw)
    return sp, r, ab


@pytest.mark.parametrize("name,h,v", JUMP_SPACES)
def test_jump_of_constants_vanishes(name, h, v):
    m = meshgen.tri_mesh(4, seed=7)
    sp, r, ab = _jump(m, 4, name, h, v, lambda sp: np.full(sp.ndofs, 1.7))
    assert np.all(np.abs(r) <= 1e-14 * ab + 1e-300)


def test_jump_dg0_single_column_closed_form():
    m = type("M", (), {})()
    m.cells = np.array([[0, 1, 2]], dtype=np.int32)
    m.xy = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.5]])
    m.nverts = 3
    u0 = np.array([0.3, -1.1, 2.5])
    sp, r, _ = _jump(m, 3, "DG0xDG0", O.DG0, O.DG0, lambda sp: u0.copy())
    A = 1.5
    want = A * np.array([u0[0] - u0[1], (u0[1] - u0[0]) + (u0[1] - u0[2]), u0[2] - u0[1]])
    np.testing.assert_allclose(r, want, rtol=1e-14)


@pytest.mark.parametrize("name,h,v", JUMP_SPACES)
def test_jump_energy_and_symmetry(name, h, v):
    """<u, J u> = sum over interior facets of int_F [u]^2 with [u] linear on F:
    int_F g^2 = A/6 (sum g_a^2 + sum_{a<b} g_a g_b); and <w, J u> = <u, J w>."""
    m = meshgen.tri_mesh(4, seed=8, order="random")
    L = 4
    rng = np.random.default_rng(9)
    sp0 = O.number(m.cells, m.nverts, L, O.DELTA[name])
    u = rng.uniform(-1, 1, sp0.ndofs)
    w = rng.uniform(-1, 1, sp0.ndofs)
    _, Ju, _ = _jump(m, L, name, h, v, lambda sp: u)
    _, Jw, _ = _jump(m, L, name, h, v, lambda sp: w)
    assert abs(w @ Ju - u @ Jw) <= 1e-13 * (np.abs(w) @ np.abs(Ju) + 1e-300)
    # traces at the facet vertices, from the stencil layout of each space
    A, _ = _areas_centroids(m)
    dh = {O.CG1: 0, O.DG0: 1, O.DG1: 3}
    energy = 0.0
    for c in range(m.ncells):
        for l in range(1, L):
            below = sp0.map[c].astype(np.int64) + (l - 1) * sp0.offset
            above = sp0.map[c].astype(np.int64) + l * sp0.offset
            g = np.zeros(3)
            for a in range(3):
                g[a] = _trace(u[below], name, a, top=True) - _trace(u[above], name, a, top=False)
            energy += A[c] / 6.0 * (g @ g + g[0] * g[1] + g[1] * g[2] + g[0] * g[2])
    assert abs(u @ Ju - energy) <= 1e-13 * max(1.0, abs(energy))
    del dh


def _trace(vals, name, a, top):
    """Value at facet vertex a of a cell's field, from the local layout of the
    space (stencil order: vertices, edges, cell; per entity bottom, top,
    vertical DoFs)."""
    hname, vname = name.split("x")
    if hname == "CG1":
        per = {"CG1": 2, "DG0": 1, "DG1": 2}[vname]
        loc = vals[a * per:(a + 1) * per]
    elif hname == "DG0":
        loc = vals
    else:   # DG1: three nodes at the vertices, vertical index minor
        per = {"CG1": 2, "DG0": 1, "DG1": 2}[vname]
        loc = vals[a * per:(a + 1) * per] if vname != "CG1" else vals[[a, 3 + a]]
    if vname == "DG0":
        return loc[0]
    return loc[1] if top else loc[0]


def test_jump_geometry_is_the_facet():
    """Two layers whose middle level is scaled horizontally: the jump uses the
    area of the facet between them, not of the column's base."""
    cells, cs, X = _one_prism([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], 2)
    Xr = X.reshape(-1, 3)
    for a in range(3):
        Xr[cs.map[0, 2 * a] + 1, :2] *= 2.0     # level 1 of vertex a
    m = type("M", (), {})()
    m.cells, m.xy, m.nverts = cells, np.zeros((3, 2)), 3
    u0 = np.array([1.0, 0.0])
    sp, r, _ = _jump(m, 2, "DG0xDG0", O.DG0, O.DG0, lambda sp: u0.copy(), X=X, cs=cs)
    np.testing.assert_allclose(r, [2.0, -2.0], rtol=1e-14)   # facet area 4 x 1/2


def test_jump_variable_layers_sum_counts_interior_facets():
    m = meshgen.tri_mesh(4, seed=10)
    rng = np.random.default_rng(11)
    first = rng.integers(0, 3, m.ncells).astype(np.int32)
    lay = (1 + rng.integers(0, 6 - first)).astype(np.int32)
    cs, X = O.coords_var(m.cells, m.xy, first, lay)
    # DG0 u = level index of the cell layer: every interior facet has [u] = -1
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["DG0xDG0"])
    u = np.zeros(sp.ndofs)
    for c in range(m.ncells):
        u[sp.map[c, 0] + np.arange(lay[c])] = np.arange(lay[c])
    _, r, _ = _jump(m, sp.layers, "DG0xDG0", O.DG0, O.DG0, lambda s: u, X=X, cs=cs,
                    cell_first=first, cell_layers=lay)
    A, _ = _areas_centroids(m)
    assert abs(u @ r - float((A * (lay - 1)).sum())) <= 1e-13
