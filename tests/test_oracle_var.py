"""Pins of the oracle's variable-layer path (Algorithm 1 and Algorithm 3 with
a number of layers per column, which the paper's Sec. 3.1 footnote and Sec. 5
say the method allows): a hand-derived example, reduction to the pinned
constant-layer numbering, closed-form totals from independently computed
column hulls, a brute-force numbering of the explicit 3-D mesh, and integrals
with closed forms."""
import os

import numpy as np
import pytest

import meshgen
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "numbering_variable_layers.txt")
SPACES = ["CG1xCG1", "CG1xDG0", "CG1xDG1", "DG0xCG1", "DG0xDG0", "DG0xDG1", "DG1xCG1", "DG1xDG0", "DG1xDG1"]


def _parse_golden():
    cells, cases, cur = None, [], None
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(" ")
        if key == "cells":
            cells = np.array([[int(x) for x in r.split()] for r in rest.split(";")], dtype=np.int32)
        elif key == "case":
            w = rest.split()
            i, j = w.index("first"), w.index("layers")
            case = {"first": [int(x) for x in w[i + 1:j]], "layers": [int(x) for x in w[j + 1:]], "spaces": []}
            cases.append(case)
        elif key == "space":
            cur = {"delta": tuple(int(x) for x in rest.split())}
            case["spaces"].append(cur)
        elif key == "ndofs":
            cur["ndofs"] = int(rest)
        elif key == "offset":
            cur["offset"] = [int(x) for x in rest.split()]
        elif key == "map":
            cur["map"] = [[int(x) for x in r.split()] for r in rest.split(";")]
        elif key == "unreached":
            cur["unreached"] = sorted(int(x) for x in rest.split())
    return cells, cases


def _reached(sp):
    r = np.zeros(sp.ndofs, dtype=bool)
    for c in range(sp.map.shape[0]):
        for l in range(int(sp.cell_layers[c])):
            r[sp.map[c].astype(np.int64) + l * sp.offset] = True
    return r


def test_golden_variable_layers():
    cells, cases = _parse_golden()
    assert len(cases) == 2
    for case in cases:
        for want in case["spaces"]:
            sp = O.number_var(cells, 4, case["first"], case["layers"], want["delta"])
            assert sp.ndofs == want["ndofs"], want["delta"]
            assert sp.offset.tolist() == want["offset"], want["delta"]
            assert sp.map.tolist() == want["map"], want["delta"]
            assert np.nonzero(~_reached(sp))[0].tolist() == want.get("unreached", []), want["delta"]


def bathymetry(m, maxlevel, seed, gaps=False):
    return meshgen.column_layers(m, maxlevel, seed, "random" if gaps else "bathymetry")


def _mesh(name, n, seed, order="rcm"):
    return meshgen.quad_mesh(n, seed=seed, order=order) if name in ("Q2xP2", "DG2hex") else \
        meshgen.tri_mesh(n, seed=seed, order=order)


@pytest.mark.parametrize("name", sorted(O.DELTA))
def test_uniform_ranges_reduce_to_algorithm_1(name):
    m = _mesh(name, 5, 3)
    L = 4
    a = O.number(m.cells, m.nverts, L, O.DELTA[name])
    b = O.number_var(m.cells, m.nverts, np.zeros(m.ncells), np.full(m.ncells, L), O.DELTA[name])
    assert a.ndofs == b.ndofs and b.layers == L
    np.testing.assert_array_equal(a.map, b.map)
    np.testing.assert_array_equal(a.offset, b.offset)
    if a.hmap is not None:
        np.testing.assert_array_equal(a.hmap, b.hmap)


def _hulls(m, first, lay):
    """Level range of every vertex and edge, computed with numpy from the
    cells' ranges (independent of the oracle's loops)."""
    ce, ne = O.derive_edges(m.cells, m.nverts)
    top = first + lay
    vlo = np.full(m.nverts, 1 << 30)
    vhi = np.full(m.nverts, -1)
    elo = np.full(ne, 1 << 30)
    ehi = np.full(ne, -1)
    for a in range(m.kind):
        np.minimum.at(vlo, m.cells[:, a], first)
        np.maximum.at(vhi, m.cells[:, a], top)
        np.minimum.at(elo, ce[:, a], first)
        np.maximum.at(ehi, ce[:, a], top)
    return (vlo, vhi), (elo, ehi), (first, top)


@pytest.mark.parametrize("name", sorted(O.DELTA))
@pytest.mark.parametrize("gaps", [False, True])
def test_closed_form_totals(name, gaps):
    m = _mesh(name, 6, 4)
    first, lay = bathymetry(m, 9, 5, gaps)
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
    total = 0
    for d, (lo, hi) in enumerate(_hulls(m, first, lay)):
        a, b = O.DELTA[name][2 * d], O.DELTA[name][2 * d + 1]
        total += int(((hi - lo) * (a + b) + a).sum())
    assert sp.ndofs == total


@pytest.mark.parametrize("name", sorted(O.DELTA))
def test_numbered_once_contiguous_columns_and_reach(name):
    m = _mesh(name, 5, 6, "random")
    first, lay = bathymetry(m, 7, 7, gaps=True)
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name], keep_tables=True)
    count = np.zeros(sp.ndofs, dtype=np.int64)
    hulls = _hulls(m, first, lay)
    for t, tab in sp.first.items():
        d1, d2 = divmod(t, 2)
        lo, hi = hulls[d1]
        lev = np.arange(tab.shape[1])[None, :]
        inside = (lev >= lo[:, None]) & (lev < hi[:, None] + (1 - d2))
        assert np.all((tab >= 0) == inside)          # exactly the hull's entities are numbered
        for q in range(sp.delta[t]):
            np.add.at(count, tab[inside] + q, 1)
    assert np.all(count == 1)
    # every entity column is one contiguous range
    for d1, (lo, hi) in enumerate(hulls):
        a, b = sp.delta[2 * d1], sp.delta[2 * d1 + 1]
        if a + b == 0:
            continue
        for i in range(lo.size):
            nums = []
            if a:
                t0 = sp.first[2 * d1][i, lo[i]:hi[i] + 1]
                nums += [x + q for x in t0 for q in range(a)]
            if b:
                t1 = sp.first[2 * d1 + 1][i, lo[i]:hi[i]]
                nums += [x + q for x in t1 for q in range(b)]
            nums.sort()
            assert nums == list(range(nums[0], nums[0] + len(nums)))
    # reached DoFs: everything except entity levels no cell around spans
    reached = _reached(sp)
    expect_unreached = 0
    for d1, (lo, hi) in enumerate(hulls[:2]):
        a, b = sp.delta[2 * d1], sp.delta[2 * d1 + 1]
        if a + b == 0:
            continue
        ce, _ = O.derive_edges(m.cells, m.nverts)
        owner = m.cells if d1 == 0 else ce
        cover = {}
        for c in range(m.ncells):
            for e in owner[c]:
                cover.setdefault(int(e), set()).update(range(int(first[c]), int(first[c] + lay[c]) + 1))
                # layers spanned by cell c at entity e: first..first+lay-1; levels first..first+lay
        for e, levs in cover.items():
            layers_cov = {l for l in levs if l + 1 in levs and any(
                first[c] <= l < first[c] + lay[c] for c in np.nonzero((owner == e).any(axis=1))[0])}
            for l in range(lo[e], hi[e]):
                if l not in layers_cov:
                    expect_unreached += b
            for l in range(lo[e], hi[e] + 1):
                if l not in levs:
                    expect_unreached += a
    assert int((~reached).sum()) == expect_unreached


def _brute_force_var(cells, first, lay, delta):
    """Number the explicit 3-D mesh of the variable columns on first visit."""
    nvc = cells.shape[1]
    ents = [(0, (a,)) for a in range(nvc)] + [(1, (a, (a + 1) % nvc)) for a in range(nvc)] + \
        [(2, tuple(range(nvc)))]
    table, nxt, res = {}, 0, []
    for c in range(cells.shape[0]):
        for l in range(int(first[c]), int(first[c] + lay[c])):
            st = []
            for d, loc in ents:
                verts = [int(cells[c, x]) for x in loc]
                for key, t in ((frozenset((v, l) for v in verts), 2 * d),
                               (frozenset((v, l + 1) for v in verts), 2 * d),
                               (frozenset([(v, l) for v in verts] + [(v, l + 1) for v in verts]), 2 * d + 1)):
                    if delta[t] == 0:
                        continue
                    if (t, key) not in table:
                        table[(t, key)] = nxt
                        nxt += delta[t]
                    st.extend(range(table[(t, key)], table[(t, key)] + delta[t]))
            res.append(st)
    return res, nxt


@pytest.mark.parametrize("name", sorted(O.DELTA))
@pytest.mark.parametrize("gaps", [False, True])
def test_brute_force_bijection(name, gaps):
    m = _mesh(name, 3, 9, "random")
    first, lay = bathymetry(m, 5, 10, gaps)
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
    b3, n3 = _brute_force_var(m.cells, first, lay, O.DELTA[name])
    ext = [sp.map[c].astype(np.int64) + l * sp.offset for c in range(m.ncells) for l in range(int(lay[c]))]
    assert len(ext) == len(b3)
    pi = {}
    for e, b in zip(ext, b3):
        assert len(e) == len(b)
        for x, y in zip(e.tolist(), b):
            assert pi.setdefault(x, y) == y
    assert len(pi) == n3 and len(set(pi.values())) == n3
    assert n3 == int(_reached(sp).sum())


def test_extrusion_levels():
    m = meshgen.tri_mesh(5, seed=12)
    first, lay = bathymetry(m, 8, 13, gaps=True)
    sp, X = O.coords_var(m.cells, m.xy, first, lay)
    full = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"], keep_tables=True)
    X = X.reshape(-1, 3)
    (vlo, vhi), _, _ = _hulls(m, first, lay)
    tab = full.first[0]
    for v in range(m.nverts):
        for l in range(vlo[v], vhi[v] + 1):
            dof = tab[v, l]
            covered = any(first[c] <= l <= first[c] + lay[c] for c in np.nonzero((m.cells == v).any(axis=1))[0])
            if covered:
                assert X[dof].tolist() == [m.xy[v, 0], m.xy[v, 1], l / 8.0]
            else:
                assert X[dof].tolist() == [0.0, 0.0, 0.0]


def _areas_centroids(m):
    p = m.xy[m.cells]
    A = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    return A, p.mean(axis=1)


@pytest.mark.parametrize("gaps", [False, True])
def test_mass_volume_and_linear_moment(gaps):
    m = meshgen.tri_mesh(6, seed=14)
    Lmax = 10
    first, lay = bathymetry(m, Lmax, 15, gaps)
    cs, X = O.coords_var(m.cells, m.xy, first, lay)
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"])
    A, cen = _areas_centroids(m)
    zb, zt = first / Lmax, (first + lay) / Lmax
    Xr = X.reshape(-1, 3)
    # f = 1 and f = x + y + z (exact in P1xP1) at the coordinate DoFs (same numbering)
    for f, want in ((np.ones(sp.ndofs), float((A * (zt - zb)).sum())),
                    (Xr.sum(axis=1), float((A * ((zt - zb) * (cen[:, 0] + cen[:, 1]) + 0.5 * (zt ** 2 - zb ** 2))).sum()))):
        b = np.zeros(sp.ndofs)
        O.par_loop(O.K_MASS, m.cells, Lmax, [(cs, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC)],
                   cell_first=first, cell_layers=lay)
        assert abs(b.sum() - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("name", SPACES)
def test_tp_mass_volume(name):
    m = meshgen.tri_mesh(5, seed=16)
    Lmax = 8
    first, lay = bathymetry(m, Lmax, 17, gaps=True)
    cs, X = O.coords_var(m.cells, m.xy, first, lay)
    sp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
    h, v = [(hh, vv) for nm, hh, vv in O.TP_PAIRS if nm == name][0]
    O.set_tp_element(h, v)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_MASS_TP, m.cells, Lmax, [(cs, X, 3, O.READ), (sp, np.ones(sp.ndofs), 1, O.READ),
                                            (sp, b, 1, O.INC)], cell_first=first, cell_layers=lay)
    A, _ = _areas_centroids(m)
    want = float((A * lay / Lmax).sum())
    assert abs(b.sum() - want) <= 1e-13 * want


def test_interp_reads_the_right_levels():
    m = meshgen.tri_mesh(4, seed=18)
    first, lay = bathymetry(m, 6, 19, gaps=True)
    p1 = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"], keep_tables=True)
    dg = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["DG1xDG1"])
    x = meshgen.uniform_field(p1.ndofs, 20)
    out = np.full(dg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, m.cells, 6, [(p1, x, 1, O.READ), (dg, out, 1, O.WRITE)],
               cell_first=first, cell_layers=lay)
    assert not np.isnan(out).any()     # a DG1 space has no gaps: every DoF is written
    tab = p1.first[0]
    for c in range(m.ncells):
        for l in range(int(lay[c])):
            for a in range(3):
                for b in range(2):
                    lev = int(first[c]) + l + b
                    assert out[dg.map[c, 2 * a + b] + l * 6] == x[tab[m.cells[c, a], lev]]


def test_rejects_bad_ranges():
    m = meshgen.tri_mesh(2, seed=1)
    with pytest.raises(ValueError):
        O.number_var(m.cells, m.nverts, np.zeros(m.ncells), np.zeros(m.ncells), O.DELTA["CG1xCG1"])
    with pytest.raises(ValueError):   # a vertex that no cell contains
        O.number_var(m.cells, m.nverts + 1, np.zeros(m.ncells), np.ones(m.ncells), O.DELTA["CG1xCG1"])
