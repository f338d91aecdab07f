"""Parity of the CUDA path with the oracle for meshes with a variable number
of layers per column and for the horizontal-facet loops: numbering, maps,
coordinates and moves bit-exact; FP64 assembly within 1e-12 of the oracle's
absolute contribution sums."""
import numpy as np
import pytest

import meshgen
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1604_05937_gb300 as E  # noqa: E402

dev = torch.device("cuda:0")
TRI = ["CG1xCG1", "CG1xDG0", "CG1xDG1", "DG0xCG1", "DG0xDG0", "DG0xDG1", "DG1xCG1", "DG1xDG0", "DG1xDG1"]
FACET = [("CG1xCG1", O.CG1), ("DG0xCG1", O.DG0), ("DG1xCG1", O.DG1)]


def close(got, want, absref, rtol=1e-12):
    err = np.abs(np.asarray(got) - want)
    bad = np.nonzero(~(err <= rtol * absref + 1e-300))[0]
    assert bad.size == 0, f"{bad.size} entries off; worst rel {(err / (absref + 1e-300)).max():.3e}"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def var_mesh(m, maxlevel, seed, kind):
    first, lay = meshgen.column_layers(m, maxlevel, seed, kind)
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    return gm, first, lay


CASES = [(4, 3, "bathymetry"), (9, 12, "random"), (23, 40, "bathymetry"), (50, 7, "random")]


# ------------------------------------------------------------------ numbering, coordinates, moves
@pytest.mark.parametrize("name", TRI + ["ALL1"])
@pytest.mark.parametrize("n,maxlevel,kind", CASES)
def test_var_numbering_bit_exact(name, n, maxlevel, kind):
    m = meshgen.tri_mesh(n, seed=700 + n, order="random" if kind == "random" else "rcm")
    delta = (1, 1, 1, 1, 1, 1) if name == "ALL1" else O.DELTA[name]
    gm, first, lay = var_mesh(m, maxlevel, 701, kind)
    assert gm.layers == int((first + lay).max())
    gs = E.Space(gm, delta)
    osp = O.number_var(m.cells, m.nverts, first, lay, delta)
    gmap, goff = gs.stencil_map()
    assert gs.ndofs == osp.ndofs
    np.testing.assert_array_equal(gmap, osp.map)
    np.testing.assert_array_equal(goff, osp.offset)


@pytest.mark.parametrize("name", ["Q2xP2", "DG2hex", "CG1xCG1"])
def test_var_numbering_bit_exact_hexes(name):
    m = meshgen.quad_mesh(9, seed=710, order="random")
    gm, first, lay = var_mesh(m, 9, 711, "random")
    gs = E.Space(gm, O.DELTA[name])
    osp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
    gmap, _ = gs.stencil_map()
    assert gs.ndofs == osp.ndofs
    np.testing.assert_array_equal(gmap, osp.map)


def test_var_numbering_many_scan_tiles():
    """1.62M cells: 4.9M base entities, beyond one CTA of tile sums in the scan."""
    m = meshgen.tri_mesh(900, seed=712, order="rcm")
    first, lay = meshgen.column_layers(m, 20, 713, "bathymetry")
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    for name in ("CG1xCG1", "DG1xDG1"):
        gs = E.Space(gm, O.DELTA[name])
        osp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
        assert gs.ndofs == osp.ndofs
        np.testing.assert_array_equal(gs.stencil_map()[0], osp.map)


@pytest.mark.parametrize("n,maxlevel,kind", CASES)
def test_var_extrusion_bit_exact(n, maxlevel, kind):
    m = meshgen.tri_mesh(n, seed=720 + n)
    gm, first, lay = var_mesh(m, maxlevel, 721, kind)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    _, X = O.coords_var(m.cells, m.xy, first, lay)
    np.testing.assert_array_equal(host(E.extrude_coords(gm, cs)), X)


@pytest.mark.parametrize("name", ["DG0xDG0", "DG1xDG1", "DG1xDG0", "DG0xDG1"])
@pytest.mark.parametrize("n,maxlevel,kind", CASES)
def test_var_dg_copy_bit_exact(name, n, maxlevel, kind):
    m = meshgen.tri_mesh(n, seed=730 + n)
    gm, first, lay = var_mesh(m, maxlevel, 731, kind)
    sp = E.Space(gm, O.DELTA[name])
    x = meshgen.uniform_field(sp.ndofs, 732)
    out = torch.full((sp.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_COPY_DG, (sp, to_dev(x), E.EXT_READ), (sp, out, E.EXT_WRITE))
    E.ext_sync_check()
    np.testing.assert_array_equal(host(out), x)


@pytest.mark.parametrize("n,maxlevel,kind", CASES)
def test_var_interpolation_bit_exact(n, maxlevel, kind):
    m = meshgen.tri_mesh(n, seed=740 + n)
    gm, first, lay = var_mesh(m, maxlevel, 741, kind)
    p1 = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG1xDG1")
    op1 = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"])
    odg = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["DG1xDG1"])
    x = meshgen.uniform_field(op1.ndofs, 742)
    ref = np.full(odg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, m.cells, op1.layers, [(op1, x, 1, O.READ), (odg, ref, 1, O.WRITE)],
               cell_first=first, cell_layers=lay)
    out = torch.full((dg.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_INTERP_DG1, (p1, to_dev(x), E.EXT_READ), (dg, out, E.EXT_WRITE))
    E.ext_sync_check()
    np.testing.assert_array_equal(host(out), ref)


# ------------------------------------------------------------------ assembly
def _coords(m, first, lay, perturb, seed):
    _, X = O.coords_var(m.cells, m.xy, first, lay)
    if perturb:
        X = X + perturb * np.random.default_rng(seed).uniform(-1, 1, X.size) / (m.n * lay.max())
    return X


@pytest.mark.parametrize("kernel", ["mass", "rhs"])
@pytest.mark.parametrize("n,maxlevel,kind,perturb", [(4, 3, "bathymetry", 0.0), (9, 12, "random", 0.0),
                                                      (23, 40, "bathymetry", 0.0), (50, 7, "random", 0.0),
                                                      (8, 9, "random", 0.05)])
def test_var_mass_parity(kernel, n, maxlevel, kind, perturb):
    m = meshgen.tri_mesh(n, seed=750 + n, order="rcm")
    gm, first, lay = var_mesh(m, maxlevel, 751, kind)
    X = _coords(m, first, lay, perturb, 752)
    ocs = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"])
    f = np.sin(X[0::3]) * np.cos(X[1::3]) * X[2::3] if kernel == "rhs" else meshgen.uniform_field(ocs.ndofs, 753)
    ref, absr = np.zeros(ocs.ndofs), np.zeros(ocs.ndofs)
    O.par_loop(O.K_MASS, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (ocs, f, 1, O.READ), (ocs, ref, 1, O.INC, absr)],
               cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    b = ps.zeros()
    k = E.EXT_K_RHS_P1P1 if kernel == "rhs" else E.EXT_K_MASS_P1P1
    E.par_loop(gm, k, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_INC))
    E.ext_sync_check()
    close(host(b), ref, absr)


@pytest.mark.parametrize("n,maxlevel,kind", [(30, 20, "random"), (100, 100, "bathymetry")])
def test_var_mass_partial(n, maxlevel, kind):
    """Variable layers with some vertex columns moved in x, y from a level up
    and some single levels lifted: the prisms touching them take the general
    6-point rule, the rest the straight forms (on the larger case, over a
    million items, the gather form with its regular levels and the per-cell
    pass at the column ends; the random ranges of the smaller case leave gaps)."""
    m = meshgen.tri_mesh(n, seed=760 + n, order="rcm")
    gm, first, lay = var_mesh(m, maxlevel, 761, kind)
    ocs = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"])
    _, X = O.coords_var(m.cells, m.xy, first, lay)
    Xr = X.reshape(-1, 3).copy()
    # vertex v's column: DoFs start[v] .. start[v] + (hi - lo); the numbering
    # puts the vertex columns first, in vertex order
    lo = np.full(m.nverts, 1 << 30)
    hi = np.full(m.nverts, -1)
    for a in range(3):
        np.minimum.at(lo, m.cells[:, a], first)
        np.maximum.at(hi, m.cells[:, a], first + lay)
    start = np.concatenate([[0], np.cumsum(hi - lo + 1)])
    rng = np.random.default_rng(762)
    for v in rng.choice(m.nverts, m.nverts // 30, replace=False):
        k = int(rng.integers(0, hi[v] - lo[v] + 1))
        Xr[start[v] + k:start[v + 1], 0] += 0.1 / n
    for v in rng.choice(m.nverts, m.nverts // 30, replace=False):
        Xr[start[v] + int(rng.integers(0, hi[v] - lo[v] + 1)), 2] += 0.2 / maxlevel
    X = Xr.reshape(-1)
    f = meshgen.uniform_field(ocs.ndofs, 763)
    ref, absr = np.zeros(ocs.ndofs), np.zeros(ocs.ndofs)
    O.par_loop(O.K_MASS, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (ocs, f, 1, O.READ), (ocs, ref, 1, O.INC, absr)],
               cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    b = torch.full((ps.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_WRITE))
    E.ext_sync_check()
    close(host(b), ref, absr)


@pytest.mark.parametrize("name,h,v", O.TP_PAIRS)
@pytest.mark.parametrize("n,maxlevel,kind,perturb", [(5, 4, "bathymetry", 0.0), (13, 30, "random", 0.0),
                                                      (7, 6, "random", 0.05)])
def test_var_mass_tp_parity(name, h, v, n, maxlevel, kind, perturb):
    m = meshgen.tri_mesh(n, seed=760 + n, order="random")
    gm, first, lay = var_mesh(m, maxlevel, 761, kind)
    X = _coords(m, first, lay, perturb, 762)
    ocs = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["CG1xCG1"])
    osp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
    f = meshgen.uniform_field(osp.ndofs, 763)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.set_tp_element(h, v)
    O.par_loop(O.K_MASS_TP, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (osp, f, 1, O.READ),
                                                  (osp, ref, 1, O.INC, absr)], cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    b = sp.zeros()
    E.par_loop(gm, E.EXT_K_MASS_TP, (cs, to_dev(X), E.EXT_READ), (sp, to_dev(f), E.EXT_READ), (sp, b, E.EXT_INC))
    E.ext_sync_check()
    close(host(b), ref, absr)


# ------------------------------------------------------------------ horizontal facets
def _facet_case(m, name, h, v, jump, layers=None, var=None, perturb=0.0, seed=0):
    """GPU and oracle results of a facet loop on a uniform (layers) or a
    variable (var = (first, lay)) mesh."""
    if var is None:
        gm = E.Mesh(m.cells, m.xy, layers)
        ocs, X = O.coords(m.cells, m.xy, layers)
        osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
        kw = {}
    else:
        first, lay = var
        gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
        ocs, X = O.coords_var(m.cells, m.xy, first, lay)
        osp = O.number_var(m.cells, m.nverts, first, lay, O.DELTA[name])
        kw = dict(cell_first=first, cell_layers=lay)
    if perturb:
        X = X + perturb * np.random.default_rng(seed).uniform(-1, 1, X.size) / (m.n * ocs.layers)
    u = meshgen.uniform_field(osp.ndofs, seed + 1)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.set_tp_element(h, v)
    if jump:
        O.par_loop(O.K_HFACET_JUMP, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (osp, u, 1, O.READ),
                                                          (osp, ref, 1, O.INC, absr)], **kw)
        kid = E.EXT_K_HFACET_JUMP
    else:
        O.par_loop(O.K_HFACET_MASS, m.cells, ocs.layers, [(ocs.facet(), X, 3, O.READ), (osp.facet(), u, 1, O.READ),
                                                          (osp.facet(), ref, 1, O.INC, absr)], **kw)
        kid = E.EXT_K_HFACET_MASS
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    b = sp.zeros()
    E.par_loop(gm, kid, (cs, to_dev(X), E.EXT_READ), (sp, to_dev(u), E.EXT_READ), (sp, b, E.EXT_INC))
    E.ext_sync_check()
    return host(b), ref, absr


@pytest.mark.parametrize("name,h", FACET)
@pytest.mark.parametrize("n,layers,perturb", [(4, 1, 0.0), (9, 7, 0.0), (17, 40, 0.0), (6, 5, 0.05)])
def test_facet_mass_parity(name, h, n, layers, perturb):
    m = meshgen.tri_mesh(n, seed=770 + n, order="random")
    got, ref, absr = _facet_case(m, name, h, O.CG1, False, layers=layers, perturb=perturb, seed=771)
    close(got, ref, absr)


@pytest.mark.parametrize("name,h,v", O.TP_PAIRS)
@pytest.mark.parametrize("n,layers,perturb", [(4, 1, 0.0), (9, 7, 0.0), (17, 40, 0.0), (6, 5, 0.05)])
def test_facet_jump_parity(name, h, v, n, layers, perturb):
    m = meshgen.tri_mesh(n, seed=780 + n, order="rcm")
    got, ref, absr = _facet_case(m, name, h, v, True, layers=layers, perturb=perturb, seed=781)
    close(got, ref, absr)


@pytest.mark.parametrize("jump", [False, True])
@pytest.mark.parametrize("n,maxlevel,kind", [(5, 4, "bathymetry"), (13, 30, "random"), (8, 9, "random")])
def test_facet_var_parity(jump, n, maxlevel, kind):
    m = meshgen.tri_mesh(n, seed=790 + n, order="random")
    var = meshgen.column_layers(m, maxlevel, 791, kind)
    for name, h, v in O.TP_PAIRS:
        if not jump and v != O.CG1:
            continue
        got, ref, absr = _facet_case(m, name, h, v, jump, var=var, seed=792)
        close(got, ref, absr)


def test_facet_area_pin_on_gpu():
    """sum of int_F 1 ds over the lambda + 1 levels of the unit square = lambda + 1."""
    m = meshgen.tri_mesh(20, seed=793)
    gm = E.Mesh(m.cells, m.xy, 9)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, "CG1xCG1")
    X = E.extrude_coords(gm, cs)
    b = sp.zeros()
    one = torch.ones(sp.ndofs, dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_HFACET_MASS, (cs, X, E.EXT_READ), (sp, one, E.EXT_READ), (sp, b, E.EXT_INC))
    E.ext_sync_check()
    assert abs(float(b.sum()) - 10.0) < 1e-12


def test_var_and_facet_validation():
    m = meshgen.tri_mesh(4, seed=794)
    first, lay = meshgen.column_layers(m, 5, 795, "random")
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG0xDG0")
    X = E.extrude_coords(gm, cs)
    u = sp.zeros()
    with pytest.raises(E.ExtError, match="EXT_EUNSUPPORTED"):
        E.par_loop(gm, E.EXT_K_U2V_FWD, (cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, sp.zeros(), E.EXT_INC))
    with pytest.raises(E.ExtError, match="EXT_EUNSUPPORTED"):
        E.Batch([gm], E.EXT_K_U2V_FWD, [[(cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, sp.zeros(), E.EXT_INC)]])
    with pytest.raises(E.ExtError, match="horizontal facets"):
        E.par_loop(gm, E.EXT_K_HFACET_MASS, (cs, X, E.EXT_READ), (dg, dg.zeros(), E.EXT_READ),
                   (dg, dg.zeros(), E.EXT_INC))


def test_single_layer_columns_have_no_interior_facets():
    m = meshgen.tri_mesh(6, seed=796)
    first = np.random.default_rng(797).integers(0, 4, m.ncells).astype(np.int32)
    lay = np.ones(m.ncells, np.int32)
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, "DG1xDG1")
    X = E.extrude_coords(gm, cs)
    r = sp.zeros()
    u = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 798)).to(dev)
    E.par_loop(gm, E.EXT_K_HFACET_JUMP, (cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, r, E.EXT_INC))
    E.ext_sync_check()
    assert float(r.abs().max()) == 0.0
