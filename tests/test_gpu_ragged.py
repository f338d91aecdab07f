"""Parity of the CUDA path with the oracle for per-entity DoF counts (ragged
lists): numbering, lists and offsets and the DG copy bit-exact, the
p-adaptive DG right-hand side within 1e-12 of the oracle's absolute
contribution sums."""
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


def close(got, want, absref, rtol=1e-12):
    err = np.abs(np.asarray(got) - want)
    bad = np.nonzero(~(err <= rtol * absref + 1e-300))[0]
    assert bad.size == 0, f"{bad.size} entries off; worst rel {(err / (absref + 1e-300)).max():.3e}"


def dent_for(m, seed, kind):
    rng = np.random.default_rng(seed)
    _, ne = O.derive_edges(m.cells, m.nverts)
    nent = m.nverts + ne + m.ncells
    if kind == "mixed":
        return rng.integers(0, 3, (nent, 2)).astype(np.int32)
    dent = np.zeros((nent, 2), np.int32)
    sizes = [1, 2, 3, 6] if kind == "dg" else [0, 1, 2, 3, 6]
    dent[m.nverts + ne:, 1] = rng.choice(sizes, m.ncells)
    return dent


def mesh_of(m, var, maxlevel, seed):
    if var:
        first, lay = meshgen.column_layers(m, maxlevel, seed, "random")
        return E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay), first, lay
    lay = np.full(m.ncells, maxlevel, np.int32)
    return E.Mesh(m.cells, m.xy, maxlevel), np.zeros(m.ncells, np.int32), lay


@pytest.mark.parametrize("kind", ["mixed", "dg", "dg0"])
@pytest.mark.parametrize("var", [False, True])
@pytest.mark.parametrize("quad", [False, True])
def test_ragged_numbering_bit_exact(kind, var, quad):
    m = meshgen.quad_mesh(9, seed=900, order="random") if quad else meshgen.tri_mesh(11, seed=901, order="random")
    gm, first, lay = mesh_of(m, var, 7, 902)
    dent = dent_for(m, 903, kind)
    gs = E.Space(gm, dent=dent)
    o = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay) if var else \
        O.number_ragged(m.cells, m.nverts, dent, layers=7)
    rowptr, mp, off = gs.stencil_map()
    assert gs.ndofs == o.ndofs and gs.k == 0
    np.testing.assert_array_equal(rowptr, o.rowptr)
    np.testing.assert_array_equal(mp, o.map)
    np.testing.assert_array_equal(off, o.offset)


def test_ragged_numbering_many_scan_tiles():
    m = meshgen.tri_mesh(700, seed=904, order="rcm")   # 980,000 cells: 2.9M entities
    gm, first, lay = mesh_of(m, True, 12, 905)
    dent = dent_for(m, 906, "dg")
    gs = E.Space(gm, dent=dent)
    o = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
    rowptr, mp, off = gs.stencil_map()
    assert gs.ndofs == o.ndofs
    np.testing.assert_array_equal(rowptr, o.rowptr)
    np.testing.assert_array_equal(mp, o.map)


@pytest.mark.parametrize("kind", ["dg", "dg0"])
@pytest.mark.parametrize("var", [False, True])
def test_ragged_copy_bit_exact(kind, var):
    m = meshgen.tri_mesh(40, seed=907)
    gm, first, lay = mesh_of(m, var, 9, 908)
    gs = E.Space(gm, dent=dent_for(m, 909, kind))
    x = torch.from_numpy(meshgen.uniform_field(gs.ndofs, 910)).to(dev)
    out = torch.full((gs.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_COPY_DG, (gs, x, E.EXT_READ), (gs, out, E.EXT_WRITE))
    E.ext_sync_check()
    assert torch.equal(out, x)


@pytest.mark.parametrize("var", [False, True])
@pytest.mark.parametrize("perturb", [0.0, 0.05])
def test_padaptive_rhs_parity(var, perturb):
    m = meshgen.tri_mesh(13, seed=911, order="random")
    gm, first, lay = mesh_of(m, var, 8, 912)
    dent = dent_for(m, 913, "dg")
    if var:
        ocs, X = O.coords_var(m.cells, m.xy, first, lay)
        osp = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
        kw = dict(cell_first=first, cell_layers=lay)
    else:
        ocs, X = O.coords(m.cells, m.xy, 8)
        osp = O.number_ragged(m.cells, m.nverts, dent, layers=8)
        kw = {}
    if perturb:
        X = X + perturb * np.random.default_rng(914).uniform(-1, 1, X.size) / (m.n * 8)
    f = meshgen.uniform_field(osp.ndofs, 915)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS_DGP, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (osp, f, 1, O.READ),
                                                   (osp, ref, 1, O.INC, absr)], **kw)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    gs = E.Space(gm, dent=dent)
    b = gs.zeros()
    E.par_loop(gm, E.EXT_K_MASS_DGP, (cs, torch.from_numpy(X).to(dev), E.EXT_READ),
               (gs, torch.from_numpy(f).to(dev), E.EXT_READ), (gs, b, E.EXT_INC))
    E.ext_sync_check()
    close(b.cpu().numpy(), ref, absr)



@pytest.mark.parametrize("layers", [1, 30])
@pytest.mark.parametrize("var", [False, True])
def test_padaptive_rhs_disk_many_warps(layers, var):
    """Two element kinds only (DG1xDG1 in a disk, DG0xDG0 elsewhere), so two of
    the four per-kind launches are empty; 7,200 cells span many warps."""
    m = meshgen.tri_mesh(60, seed=916, order="rcm")
    _, ne = O.derive_edges(m.cells, m.nverts)
    dent = meshgen.padaptive_dent(m, ne, 917, "disk")
    assert set(np.unique(dent[m.nverts + ne:, 1])) == {1, 6}
    if var:
        first, lay = meshgen.column_layers(m, layers, 918, "bathymetry")
        gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
        ocs, X = O.coords_var(m.cells, m.xy, first, lay)
        osp = O.number_ragged(m.cells, m.nverts, dent, cell_first=first, cell_layers=lay)
        kw = dict(cell_first=first, cell_layers=lay)
    else:
        gm = E.Mesh(m.cells, m.xy, layers)
        ocs, X = O.coords(m.cells, m.xy, layers)
        osp = O.number_ragged(m.cells, m.nverts, dent, layers=layers)
        kw = {}
    f = meshgen.uniform_field(osp.ndofs, 919)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS_DGP, m.cells, ocs.layers, [(ocs, X, 3, O.READ), (osp, f, 1, O.READ),
                                                   (osp, ref, 1, O.INC, absr)], **kw)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    gs = E.Space(gm, dent=dent)
    b = gs.zeros()
    E.par_loop(gm, E.EXT_K_MASS_DGP, (cs, torch.from_numpy(X).to(dev), E.EXT_READ),
               (gs, torch.from_numpy(f).to(dev), E.EXT_READ), (gs, b, E.EXT_INC))
    E.ext_sync_check()
    close(b.cpu().numpy(), ref, absr)

def test_ragged_validation():
    m = meshgen.tri_mesh(4, seed=916)
    gm = E.Mesh(m.cells, m.xy, 3)
    _, ne = O.derive_edges(m.cells, m.nverts)
    bad = dent_for(m, 917, "dg")
    bad[0, 0] = -1
    with pytest.raises(E.ExtError, match="EXT_EINVAL"):
        E.Space(gm, dent=bad)
    with pytest.raises(E.ExtError, match="EXT_EINVAL"):
        E.Space(gm, dent=np.zeros((m.nverts + ne + m.ncells, 2), np.int32))   # no DoFs
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    X = E.extrude_coords(gm, cs)
    mixed = E.Space(gm, dent=dent_for(m, 918, "mixed"))
    dg0 = E.Space(gm, dent=dent_for(m, 919, "dg0"))   # some cells without DoFs
    with pytest.raises(E.ExtError, match="outside the cells"):
        E.par_loop(gm, E.EXT_K_COPY_DG, (mixed, mixed.zeros(), E.EXT_READ), (mixed, mixed.zeros(), E.EXT_WRITE))
    for sp in (mixed, dg0):
        with pytest.raises(E.ExtError, match="EXT_EINVAL"):
            E.par_loop(gm, E.EXT_K_MASS_DGP, (cs, X, E.EXT_READ), (sp, sp.zeros(), E.EXT_READ),
                       (sp, sp.zeros(), E.EXT_INC))
    with pytest.raises(E.ExtError, match="EXT_EINVAL"):
        E.par_loop(gm, E.EXT_K_RHS_P1P1, (cs, X, E.EXT_READ), (mixed, mixed.zeros(), E.EXT_READ),
                   (mixed, mixed.zeros(), E.EXT_INC))
    other = E.Space(gm, dent=dent_for(m, 920, "dg"))
    same = E.Space(gm, dent=dent_for(m, 920, "dg"))
    with pytest.raises(E.ExtError, match="same space"):
        E.par_loop(gm, E.EXT_K_MASS_DGP, (cs, X, E.EXT_READ), (other, other.zeros(), E.EXT_READ),
                   (same, same.zeros(), E.EXT_INC))
