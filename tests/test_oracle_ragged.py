"""Pins of the oracle's per-entity DoF counts (Algorithm 1 with the constant
delta of each entity type replaced by one count per entity, which Sec. 5 says
the numbering allows) and of the p-adaptive DG kernel built on it: a
hand-derived example, reduction to the pinned constant-delta numbering (on
constant and variable layers), closed-form totals, a brute-force numbering of
the explicit 3-D mesh, and the kernels against the pinned per-space ones."""
import os

import numpy as np
import pytest

import meshgen
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "numbering_ragged.txt")
DG_KIND = {1: (O.DG0, O.DG0, "DG0xDG0"), 2: (O.DG0, O.DG1, "DG0xDG1"), 3: (O.DG1, O.DG0, "DG1xDG0"),
           6: (O.DG1, O.DG1, "DG1xDG1")}


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
            cur = {"layers": int(rest.split()[1])}
            cases.append(cur)
        elif key in ("dent_h", "dent_v"):
            cur[key] = [int(x) for g in rest.split("|") for x in g.split()]
        elif key == "ndofs":
            cur["ndofs"] = int(rest)
        elif key in ("rows", "offsets"):
            cur[key] = [[int(x) for x in r.split()] for r in rest.split(";")]
    return cells, cases


def _rows(sp, arr):
    return [arr[sp.rowptr[c]:sp.rowptr[c + 1]].tolist() for c in range(sp.rowptr.size - 1)]


def test_golden_ragged():
    cells, cases = _parse_golden()
    for case in cases:
        dent = np.stack([case["dent_h"], case["dent_v"]], axis=1)
        sp = O.number_ragged(cells, 4, dent, layers=case["layers"])
        assert sp.ndofs == case["ndofs"]
        assert _rows(sp, sp.map) == case["rows"]
        assert _rows(sp, sp.offset) == case["offsets"]


def _mesh(name, n, seed, order="rcm"):
    return meshgen.quad_mesh(n, seed=seed, order=order) if name in ("Q2xP2", "DG2hex") else \
        meshgen.tri_mesh(n, seed=seed, order=order)


@pytest.mark.parametrize("name", sorted(O.DELTA))
@pytest.mark.parametrize("var", [False, True])
def test_constant_counts_reduce_to_algorithm_1(name, var):
    m = _mesh(name, 5, 3)
    dent = O.dent_of(m.cells, m.nverts, O.DELTA[name])
    if var:
        first, lay = meshgen.column_layers(m, 6, 4, "random")
        a = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
        r = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
    else:
        a = O.number(m.cells, m.nverts, 4, O.DELTA[name])
        r = O.number_ragged(m.cells, m.nverts, dent, layers=4)
    assert a.ndofs == r.ndofs
    np.testing.assert_array_equal(r.rowptr, np.arange(m.ncells + 1) * a.k)
    np.testing.assert_array_equal(r.map, a.map.ravel())
    np.testing.assert_array_equal(r.offset, np.tile(a.offset, m.ncells))


def random_dent(m, seed, kind):
    """Per-entity counts: 'mixed' draws every entity's (h, v) counts in 0..2;
    'dg' gives every cell one of the four DG element sizes and nothing else."""
    rng = np.random.default_rng(seed)
    _, ne = O.derive_edges(m.cells, m.nverts)
    nent = m.nverts + ne + m.ncells
    if kind == "dg":
        dent = np.zeros((nent, 2), np.int32)
        dent[m.nverts + ne:, 1] = rng.choice([1, 2, 3, 6], m.ncells)
        return dent
    return rng.integers(0, 3, (nent, 2)).astype(np.int32)


def _hull(m, first, lay):
    ce, ne = O.derive_edges(m.cells, m.nverts)
    lo = np.full(m.nverts + ne + m.ncells, 1 << 30)
    hi = np.full(lo.size, -1)
    for a in range(m.kind):
        np.minimum.at(lo, m.cells[:, a], first)
        np.maximum.at(hi, m.cells[:, a], first + lay)
        np.minimum.at(lo, m.nverts + ce[:, a], first)
        np.maximum.at(hi, m.nverts + ce[:, a], first + lay)
    lo[m.nverts + ne:] = first
    hi[m.nverts + ne:] = first + lay
    return lo, hi


@pytest.mark.parametrize("kind", ["mixed", "dg"])
@pytest.mark.parametrize("var", [False, True])
def test_closed_form_total(kind, var):
    m = meshgen.tri_mesh(6, seed=5)
    dent = random_dent(m, 6, kind)
    if var:
        first, lay = meshgen.column_layers(m, 7, 8, "random")
    else:
        first, lay = np.zeros(m.ncells, np.int64), np.full(m.ncells, 5)
    sp = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
    lo, hi = _hull(m, np.asarray(first), np.asarray(lay))
    assert sp.ndofs == int(((hi - lo) * (dent[:, 0] + dent[:, 1]) + dent[:, 0]).sum())


def _brute_force(cells, first, lay, dent_of_key):
    """First-visit numbering of the explicit 3-D mesh; an entity's count comes
    from its base entity and its kind (horizontal / vertical)."""
    nvc = cells.shape[1]
    ents = [(0, (a,)) for a in range(nvc)] + [(1, (a, (a + 1) % nvc)) for a in range(nvc)] + \
        [(2, tuple(range(nvc)))]
    table, nxt, res = {}, 0, []
    for c in range(cells.shape[0]):
        for l in range(int(first[c]), int(first[c] + lay[c])):
            st = []
            for d, loc in ents:
                verts = tuple(int(cells[c, x]) for x in loc)
                base = c if d == 2 else frozenset(verts)
                for key, vert in ((frozenset((v, l) for v in verts), 0), (frozenset((v, l + 1) for v in verts), 0),
                                  (frozenset([(v, l) for v in verts] + [(v, l + 1) for v in verts]), 1)):
                    n = dent_of_key(d, base, vert)
                    if n == 0:
                        continue
                    if (d, vert, key) not in table:
                        table[(d, vert, key)] = nxt
                        nxt += n
                    st.extend(range(table[(d, vert, key)], table[(d, vert, key)] + n))
            res.append(st)
    return res, nxt


@pytest.mark.parametrize("kind", ["mixed", "dg"])
@pytest.mark.parametrize("var", [False, True])
def test_brute_force_bijection(kind, var):
    m = meshgen.tri_mesh(3, seed=9, order="random")
    dent = random_dent(m, 10, kind)
    ce, ne = O.derive_edges(m.cells, m.nverts)
    edge_id = {}
    for c in range(m.ncells):
        for a in range(3):
            edge_id[frozenset((int(m.cells[c, a]), int(m.cells[c, (a + 1) % 3])))] = int(ce[c, a])

    def count(d, base, vert):
        if d == 0:
            g = next(iter(base))
        elif d == 1:
            g = m.nverts + edge_id[base]
        else:
            g = m.nverts + ne + base
        return int(dent[g, vert])

    if var:
        first, lay = meshgen.column_layers(m, 5, 11, "random")
    else:
        first, lay = np.zeros(m.ncells, np.int64), np.full(m.ncells, 3)
    sp = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
    b3, n3 = _brute_force(m.cells, first, lay, count)
    ext = []
    for c in range(m.ncells):
        row = sp.map[sp.rowptr[c]:sp.rowptr[c + 1]].astype(np.int64)
        off = sp.offset[sp.rowptr[c]:sp.rowptr[c + 1]]
        ext += [row + l * off for l in range(int(lay[c]))]
    assert len(ext) == len(b3)
    pi = {}
    for e, b in zip(ext, b3):
        assert len(e) == len(b)
        for x, y in zip(e.tolist(), b):
            assert pi.setdefault(x, y) == y
    assert len(pi) == n3 and len(set(pi.values())) == n3


def test_ragged_copy_is_exact():
    m = meshgen.tri_mesh(5, seed=12)
    dent = random_dent(m, 13, "dg")
    sp = O.number_ragged(m.cells, m.nverts, dent, layers=4)
    x = meshgen.uniform_field(sp.ndofs, 14)
    out = np.full(sp.ndofs, np.nan)
    O.par_loop(O.K_COPY, m.cells, 4, [(sp, x, 1, O.READ), (sp, out, 1, O.WRITE)])
    np.testing.assert_array_equal(out, x)


@pytest.mark.parametrize("var", [False, True])
def test_padaptive_rhs_equals_each_element(var):
    """Every cell's block equals what the (pinned) nine-space kernel gives for
    that cell's element; and sum b = volume for f = 1."""
    m = meshgen.tri_mesh(5, seed=15)
    dent = random_dent(m, 16, "dg")
    if var:
        first, lay = meshgen.column_layers(m, 6, 17, "random")
        cs, X = O.coords_var(m.cells, m.xy, first, lay)
        kw = dict(cell_first=first, cell_layers=lay)
    else:
        first, lay = np.zeros(m.ncells, np.int32), np.full(m.ncells, 4, np.int32)
        cs, X = O.coords(m.cells, m.xy, 4)
        kw = {}
    sp = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
    f = meshgen.uniform_field(sp.ndofs, 18)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_MASS_DGP, m.cells, cs.layers, [(cs, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC)], **kw)
    for kc, (h, v, name) in DG_KIND.items():
        cells_k = np.nonzero(dent[-m.ncells:, 1] == kc)[0]
        if cells_k.size == 0:
            continue
        reg = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name]) if var else \
            O.number(m.cells, m.nverts, 4, O.DELTA[name])
        fr = np.zeros(reg.ndofs)
        for c in cells_k:   # the same input values, moved to the regular numbering
            for l in range(int(lay[c])):
                fr[reg.map[c].astype(np.int64) + l * reg.offset] = f[sp.map[sp.rowptr[c]:sp.rowptr[c + 1]] + l * kc]
        br = np.zeros(reg.ndofs)
        O.set_tp_element(h, v)
        sub = O.Space(delta=reg.delta, layers=reg.layers, ndofs=reg.ndofs, k=reg.k,
                      map=np.ascontiguousarray(reg.map[cells_k]), offset=reg.offset)
        O.par_loop(O.K_MASS_TP, np.ascontiguousarray(m.cells[cells_k]), cs.layers,
                   [(O.Space(delta=cs.delta, layers=cs.layers, ndofs=cs.ndofs, k=cs.k,
                             map=np.ascontiguousarray(cs.map[cells_k]), offset=cs.offset), X, 3, O.READ),
                    (sub, fr, 1, O.READ), (sub, br, 1, O.INC)],
                   **({} if not var else dict(cell_first=first[cells_k], cell_layers=lay[cells_k])))
        for c in cells_k:
            for l in range(int(lay[c])):
                got = b[sp.map[sp.rowptr[c]:sp.rowptr[c + 1]] + l * kc]
                want = br[reg.map[c].astype(np.int64) + l * reg.offset]
                np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-17)
    b1 = np.zeros(sp.ndofs)
    O.par_loop(O.K_MASS_DGP, m.cells, cs.layers, [(cs, X, 3, O.READ), (sp, np.ones(sp.ndofs), 1, O.READ),
                                                  (sp, b1, 1, O.INC)], **kw)
    p = m.xy[m.cells]
    A = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    want = float((A * lay / cs.layers).sum())
    assert abs(b1.sum() - want) <= 1e-13 * want


def test_rejects_unknown_element_size():
    m = meshgen.tri_mesh(2, seed=19)
    dent = random_dent(m, 20, "dg")
    dent[-1, 1] = 4   # no DG element has four DoFs per cell
    sp = O.number_ragged(m.cells, m.nverts, dent, layers=2)
    cs, X = O.coords(m.cells, m.xy, 2)
    with pytest.raises(RuntimeError):
        O.par_loop(O.K_MASS_DGP, m.cells, 2, [(cs, X, 3, O.READ), (sp, np.ones(sp.ndofs), 1, O.READ),
                                              (sp, np.zeros(sp.ndofs), 1, O.INC)])
