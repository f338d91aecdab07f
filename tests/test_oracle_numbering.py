"""Pins of the oracle's numbering (Algorithm 1, Sec. 3.2) and offsets
(Algorithm 2, Sec. 3.3) against facts fixed by the paper and by counting:
a hand-worked example, closed-form DoF totals from the entity sets
V_{d1,d2} (Sec. 3.1.3), one number per DoF, vertical sharing, contiguous
entity columns, and a brute-force numbering of the explicit 3-D mesh."""
import os

import numpy as np
import pytest

import meshgen
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "numbering_two_triangles.txt")


def _parse_golden():
    cases = []
    head = {}
    cur = None
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(" ")
        if key == "layers":
            head["layers"] = int(rest)
        elif key in ("cells", "cell_edges"):
            head[key] = np.array([[int(x) for x in r.split()] for r in rest.split(";")], dtype=np.int32)
        elif key == "space":
            cur = {"delta": tuple(int(x) for x in rest.split())}
            cases.append(cur)
        elif key == "ndofs":
            cur["ndofs"] = int(rest)
        elif key == "offset":
            cur["offset"] = [int(x) for x in rest.split()]
        elif key == "map":
            cur["map"] = [[int(x) for x in r.split()] for r in rest.split(";")]
    return head, cases


def test_golden_two_triangles():
    head, cases = _parse_golden()
    ce, ne = O.derive_edges(head["cells"], 4)
    assert ne == 5
    np.testing.assert_array_equal(ce, head["cell_edges"])
    for cs in cases:
        sp = O.number(head["cells"], 4, head["layers"], cs["delta"])
        assert sp.ndofs == cs["ndofs"], cs["delta"]
        assert sp.offset.tolist() == cs["offset"], cs["delta"]
        assert sp.map.tolist() == cs["map"], cs["delta"]


# closed-form totals: sum over (d1,d2) of delta * N_d1 * (layers + 1 - d2)
CLOSED = {
    "CG1xCG1": lambda V, E, C, L: V * (L + 1),
    "CG1xDG0": lambda V, E, C, L: V * L,
    "CG1xDG1": lambda V, E, C, L: 2 * V * L,
    "DG0xCG1": lambda V, E, C, L: C * (L + 1),
    "DG0xDG0": lambda V, E, C, L: C * L,
    "DG0xDG1": lambda V, E, C, L: 2 * C * L,
    "DG1xCG1": lambda V, E, C, L: 3 * C * (L + 1),
    "DG1xDG0": lambda V, E, C, L: 3 * C * L,
    "DG1xDG1": lambda V, E, C, L: 6 * C * L,
    "Q2xP2": lambda V, E, C, L: (V + E + C) * (2 * L + 1),
    "DG2hex": lambda V, E, C, L: 27 * C * L,
}
K = {"CG1xCG1": 6, "CG1xDG0": 3, "CG1xDG1": 6, "DG0xCG1": 2, "DG0xDG0": 1, "DG0xDG1": 2,
     "DG1xCG1": 6, "DG1xDG0": 3, "DG1xDG1": 6}
OFFSET = {"CG1xCG1": 1, "CG1xDG0": 1, "CG1xDG1": 2, "DG0xCG1": 1, "DG0xDG0": 1, "DG0xDG1": 2,
          "DG1xCG1": 3, "DG1xDG0": 3, "DG1xDG1": 6}


def test_edge_count_euler():
    # a triangulated or quadrangulated disk has V - E + F = 1
    for m in (meshgen.tri_mesh(9, seed=3), meshgen.quad_mesh(7, seed=4)):
        _, ne = O.derive_edges(m.cells, m.nverts)
        assert m.nverts - ne + m.ncells == 1
        assert ne == 2 * m.n * (m.n + 1) + (m.n * m.n if m.kind == 3 else 0)


def test_edge_first_appearance():
    m = meshgen.tri_mesh(5, seed=11, order="random")
    ce, ne = O.derive_edges(m.cells, m.nverts)
    seen = {}
    for c in range(m.ncells):
        for k in range(3):
            key = frozenset((int(m.cells[c, k]), int(m.cells[c, (k + 1) % 3])))
            if key not in seen:
                seen[key] = len(seen)
            assert ce[c, k] == seen[key]
    assert ne == len(seen)


@pytest.mark.parametrize("name", sorted(CLOSED))
@pytest.mark.parametrize("layers", [1, 3, 10])
def test_closed_form_totals_and_offsets(name, layers):
    m = meshgen.quad_mesh(6, seed=2) if name in ("Q2xP2", "DG2hex") else meshgen.tri_mesh(6, seed=2)
    _, ne = O.derive_edges(m.cells, m.nverts)
    sp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    assert sp.ndofs == CLOSED[name](m.nverts, ne, m.ncells, layers)
    if name in K:
        assert sp.k == K[name]
        assert set(sp.offset.tolist()) == {OFFSET[name]}
    elif name == "Q2xP2":
        assert sp.k == 27 and set(sp.offset.tolist()) == {2}
    else:
        assert sp.k == 27 and set(sp.offset.tolist()) == {27}


def _all_cell_dofs(sp, layers):
    """(C, layers, k) global DoFs reached by Algorithm 3's direct addressing."""
    l = np.arange(layers)[None, :, None]
    return sp.map[:, None, :].astype(np.int64) + l * sp.offset[None, None, :].astype(np.int64)


@pytest.mark.parametrize("name", sorted(CLOSED))
def test_each_dof_numbered_once_and_reached(name):
    layers = 4
    m = meshgen.quad_mesh(5, seed=8, order="random") if name in ("Q2xP2", "DG2hex") else \
        meshgen.tri_mesh(5, seed=8, order="random")
    sp = O.number(m.cells, m.nverts, layers, O.DELTA[name], keep_tables=True)
    # entity tables: every number in [0, N) is given to exactly one (entity, slot)
    count = np.zeros(sp.ndofs, dtype=np.int64)
    for t, tab in sp.first.items():
        d = sp.delta[t]
        for q in range(d):
            np.add.at(count, tab.ravel() + q, 1)
    assert np.all(count == 1)
    # the cells' stencils reach every DoF
    reached = np.zeros(sp.ndofs, dtype=bool)
    reached[_all_cell_dofs(sp, layers).ravel()] = True
    assert reached.all()


@pytest.mark.parametrize("name", ["CG1xCG1", "DG1xCG1", "DG0xCG1", "Q2xP2"])
def test_vertical_sharing(name):
    """Top horizontal DoFs of layer l are the bottom ones of layer l+1."""
    layers = 5
    hexes = name == "Q2xP2"
    m = meshgen.quad_mesh(4, seed=1) if hexes else meshgen.tri_mesh(4, seed=1)
    sp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    dofs = _all_cell_dofs(sp, layers)
    nvc = m.kind
    j = 0
    for d in range(3):
        a, b = sp.delta[2 * d], sp.delta[2 * d + 1]
        for _ in range(1 if d == 2 else nvc):
            for q in range(a):
                bot = dofs[:, :, j + q]
                top = dofs[:, :, j + a + q]
                np.testing.assert_array_equal(top[:, :-1], bot[:, 1:])
            j += 2 * a + b
    assert j == sp.k


@pytest.mark.parametrize("name", ["CG1xCG1", "CG1xDG1", "DG1xDG1", "Q2xP2", "DG1xCG1"])
def test_entity_columns_contiguous(name):
    """Sec. 3.2: vertically adjacent entities get adjacent numbers; every base
    entity's column is one contiguous range of layers*(a+b)+a numbers."""
    layers = 6
    m = meshgen.quad_mesh(4, seed=5) if name == "Q2xP2" else meshgen.tri_mesh(4, seed=5)
    sp = O.number(m.cells, m.nverts, layers, O.DELTA[name], keep_tables=True)
    for d1 in range(3):
        a, b = sp.delta[2 * d1], sp.delta[2 * d1 + 1]
        if a + b == 0:
            continue
        colsize = layers * (a + b) + a
        nums = []
        if a:
            t0 = sp.first[2 * d1]
            nums.append(t0[:, :, None] + np.arange(a)[None, None, :])
        if b:
            t1 = sp.first[2 * d1 + 1]
            nums.append(t1[:, :, None] + np.arange(b)[None, None, :])
        allnums = np.concatenate([x.reshape(x.shape[0], -1) for x in nums], axis=1)
        allnums.sort(axis=1)
        assert allnums.shape[1] == colsize
        np.testing.assert_array_equal(allnums - allnums[:, :1], np.tile(np.arange(colsize), (allnums.shape[0], 1)))


def _brute_force_numbering(cells, layers, delta):
    """Number the explicit 3-D mesh: each extruded entity is identified by its
    set of (vertex, level) points; entities are numbered on first visit while
    scanning 3-D cells, each getting delta numbers.  Returns (C, layers, k)."""
    nvc = cells.shape[1]
    ents = []
    for a in range(nvc):
        ents.append((0, (a,)))
    for a in range(nvc):
        ents.append((1, (a, (a + 1) % nvc)))
    ents.append((2, tuple(range(nvc))))
    table = {}
    nxt = 0
    out = np.zeros((cells.shape[0], layers, 0), dtype=np.int64).tolist()
    res = []
    for c in range(cells.shape[0]):
        row = []
        for l in range(layers):
            st = []
            for d, loc in ents:
                verts = [int(cells[c, x]) for x in loc]
                parts = [(frozenset((v, l) for v in verts), 2 * d),
                         (frozenset((v, l + 1) for v in verts), 2 * d),
                         (frozenset([(v, l) for v in verts] + [(v, l + 1) for v in verts]), 2 * d + 1)]
                for key, t in parts:
                    n = delta[t]
                    if n == 0:
                        continue
                    key = (t, key)
                    if key not in table:
                        table[key] = nxt
                        nxt += n
                    st.extend(range(table[key], table[key] + n))
            row.append(st)
        res.append(row)
    del out
    return np.array(res, dtype=np.int64), nxt


@pytest.mark.parametrize("name", ["CG1xCG1", "CG1xDG0", "CG1xDG1", "DG0xCG1", "DG0xDG0", "DG1xCG1",
                                  "DG1xDG1", "Q2xP2", "DG2hex", "ALL1"])
@pytest.mark.parametrize("order", ["rcm", "random"])
def test_brute_force_bijection(name, order):
    layers = 3
    if name in ("Q2xP2", "DG2hex"):
        m = meshgen.quad_mesh(3, seed=9, order=order)
    else:
        m = meshgen.tri_mesh(3, seed=9, order=order)
    delta = (1, 1, 1, 1, 1, 1) if name == "ALL1" else O.DELTA[name]
    sp = O.number(m.cells, m.nverts, layers, delta)
    ext = _all_cell_dofs(sp, layers)
    b3, n3 = _brute_force_numbering(m.cells, layers, delta)
    assert n3 == sp.ndofs
    assert ext.shape == b3.shape
    pi = -np.ones(sp.ndofs, dtype=np.int64)
    e = ext.ravel()
    b = b3.ravel()
    for x, y in zip(e, b):
        if pi[x] == -1:
            pi[x] = y
        assert pi[x] == y
    assert np.all(pi >= 0)
    assert np.unique(pi).size == sp.ndofs


def test_overflow_guard():
    # DG2 on a large column count: the int32 guard rejects more than 2^31 - 1 DoFs
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    with pytest.raises(OverflowError):
        O.number(cells, 4, 80_000_000, O.DELTA["DG2hex"])
