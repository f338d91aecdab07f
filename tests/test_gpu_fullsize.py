"""Parity at full workload sizes, in the launch configurations the benchmark
times: numbering and coordinates compared in full (bit-exact), assembled
values on sampled cells.  For a sample of base cells S, the oracle runs
Algorithm 3 over the closure of S (every cell sharing a vertex with a cell of
S), so each DoF in S's stencils receives all of its contributions there and
is compared with the GPU result within 1e-12 of its absolute contribution
sum."""
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
P1 = O.DELTA["CG1xCG1"]


def closure(cells, sample):
    verts = np.unique(cells[sample])
    return np.nonzero(np.isin(cells, verts).any(axis=1))[0]


def sub(space, idx):
    """The oracle space restricted to base cells idx (same numbering)."""
    return O.Space(delta=space.delta, layers=space.layers, ndofs=space.ndofs, k=space.k,
                   map=np.ascontiguousarray(space.map[idx]), offset=space.offset)


def sampled_dofs(space, sample, layers):
    l = np.arange(layers)[None, :, None]
    d = space.map[sample][:, None, :].astype(np.int64) + l * space.offset[None, None, :]
    return np.unique(d.ravel())


def close_at(got, want, absref, dofs):
    err = np.abs(got[dofs] - want[dofs])
    bound = 1e-12 * absref[dofs] + 1e-300
    assert np.all(err <= bound), float((err / (absref[dofs] + 1e-300)).max())


def test_fullsize_prisms_1M_by_100():
    m = meshgen.tri_mesh(707, seed=1604, order="rcm")
    L = 100
    gm = E.Mesh(m.cells, m.xy, L)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    p1 = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG1xDG1")
    ocs, X = O.coords(m.cells, m.xy, L)
    op1 = O.number(m.cells, m.nverts, L, P1)
    odg = O.number(m.cells, m.nverts, L, O.DELTA["DG1xDG1"])
    for g, o in ((p1, op1), (dg, odg), (cs, ocs)):
        gmap, goff = g.stencil_map()
        assert g.ndofs == o.ndofs
        np.testing.assert_array_equal(gmap, o.map)
        np.testing.assert_array_equal(goff, o.offset)
    Xg = E.extrude_coords(gm, cs)
    np.testing.assert_array_equal(Xg.cpu().numpy(), X)
    Xr = X.reshape(-1, 3)
    f = np.sin(Xr[:, 0]) * np.cos(Xr[:, 1]) * Xr[:, 2]
    x = meshgen.uniform_field(op1.ndofs, 1614)
    b, y, out = p1.zeros(), p1.zeros(), dg.zeros()
    fd, xd = torch.from_numpy(f).to(dev), torch.from_numpy(x).to(dev)
    E.par_loop(gm, E.EXT_K_RHS_P1P1, (cs, Xg, E.EXT_READ), (p1, fd, E.EXT_READ), (p1, b, E.EXT_INC))
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xg, E.EXT_READ), (p1, xd, E.EXT_READ), (p1, y, E.EXT_INC))
    E.par_loop(gm, E.EXT_K_INTERP_DG1, (p1, xd, E.EXT_READ), (dg, out, E.EXT_WRITE))
    E.ext_sync_check()
    rng = np.random.default_rng(7)
    sample = np.concatenate([rng.choice(m.ncells, 300, replace=False), [0, m.ncells - 1]])
    cl = closure(m.cells, sample)
    cells_c = np.ascontiguousarray(m.cells[cl])
    for inp, got in ((f, b), (x, y)):
        ref, absr = np.zeros(op1.ndofs), np.zeros(op1.ndofs)
        O.par_loop(O.K_MASS, cells_c, L, [(sub(ocs, cl), X, 3, O.READ), (sub(op1, cl), inp, 1, O.READ),
                                          (sub(op1, cl), ref, 1, O.INC, absr)])
        close_at(got.cpu().numpy(), ref, absr, sampled_dofs(op1, sample, L))
    # interpolation: every DG1 DoF of the sample cells, bit-exact
    oref = np.full(odg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, np.ascontiguousarray(m.cells[sample]), L,
               [(sub(op1, sample), x, 1, O.READ), (sub(odg, sample), oref, 1, O.WRITE)])
    d = sampled_dofs(odg, sample, L)
    np.testing.assert_array_equal(out.cpu().numpy()[d], oref[d])
    # the interpolation writes every DoF exactly once: no NaN survives a NaN-filled output
    out.fill_(float("nan"))
    E.par_loop(gm, E.EXT_K_INTERP_DG1, (p1, xd, E.EXT_READ), (dg, out, E.EXT_WRITE))
    assert not torch.isnan(out).any()


@pytest.mark.parametrize("kind", ["terrain", "wavy", "tilted"])
def test_fullsize_non_flat_prisms_1M_by_100(kind):
    """The benchmark mesh (999,698 triangles x 100 layers) with
    terrain-following levels (every prism's top face tilted: the
    terrain-following gather), bent levels or leaning columns (the cell
    loop): the default launch of the mass action with WRITE access, on
    sampled cells."""
    m = meshgen.tri_mesh(707, seed=1604, order="rcm")
    L = 100
    gm = E.Mesh(m.cells, m.xy, L)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    p1 = E.Space(gm, "CG1xCG1")
    ocs, _ = O.coords(m.cells, m.xy, L)
    op1 = O.number(m.cells, m.nverts, L, P1)
    X = meshgen.level_coords(m, L, seed=1615, kind=kind).reshape(-1)
    x = meshgen.uniform_field(op1.ndofs, 1616)
    y = torch.full((p1.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, torch.from_numpy(X).to(dev), E.EXT_READ),
               (p1, torch.from_numpy(x).to(dev), E.EXT_READ), (p1, y, E.EXT_WRITE))
    E.ext_sync_check()
    got = y.cpu().numpy()
    assert not np.isnan(got).any()
    rng = np.random.default_rng(8)
    sample = np.concatenate([rng.choice(m.ncells, 300, replace=False), [0, m.ncells - 1]])
    cl = closure(m.cells, sample)
    ref, absr = np.zeros(op1.ndofs), np.zeros(op1.ndofs)
    O.par_loop(O.K_MASS, np.ascontiguousarray(m.cells[cl]), L,
               [(sub(ocs, cl), X, 3, O.READ), (sub(op1, cl), x, 1, O.READ), (sub(op1, cl), ref, 1, O.INC, absr)])
    close_at(got, ref, absr, sampled_dofs(op1, sample, L))


@pytest.mark.parametrize("name", ["Q2xP2", "DG2hex"])
def test_fullsize_hexes_500k_by_64(name):
    q = meshgen.quad_mesh(707, seed=1608, order="rcm")
    L = 64
    gm = E.Mesh(q.cells, q.xy, L)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    osp = O.number(q.cells, q.nverts, L, O.DELTA[name])
    gmap, goff = sp.stencil_map()
    np.testing.assert_array_equal(gmap, osp.map)
    np.testing.assert_array_equal(goff, osp.offset)
    ocs, X = O.coords(q.cells, q.xy, L)
    Xg = E.extrude_coords(gm, cs)
    np.testing.assert_array_equal(Xg.cpu().numpy(), X)
    dg = name == "DG2hex"
    acc = E.EXT_WRITE if dg else E.EXT_INC
    u = meshgen.uniform_field(osp.ndofs, 1618)
    w = meshgen.uniform_field(osp.ndofs, 1619)
    ud, wd = torch.from_numpy(u).to(dev), torch.from_numpy(w).to(dev)
    F, G = sp.zeros(), sp.zeros()
    E.par_loop(gm, E.EXT_K_U2V_FWDADJ, (cs, Xg, E.EXT_READ), (sp, ud, E.EXT_READ), (sp, wd, E.EXT_READ),
               (sp, F, acc), (sp, G, acc))
    E.ext_sync_check()
    rng = np.random.default_rng(8)
    sample = np.concatenate([rng.choice(q.ncells, 40, replace=False), [0, q.ncells - 1]])
    cl = closure(q.cells, sample)
    cc = np.ascontiguousarray(q.cells[cl])
    oacc = O.WRITE if dg else O.INC
    Fr, aF, Gr, aG = (np.zeros(osp.ndofs) for _ in range(4))
    O.par_loop(O.K_U2V, cc, L, [(sub(ocs, cl), X, 3, O.READ), (sub(osp, cl), u, 1, O.READ),
                                (sub(osp, cl), Fr, 1, oacc, aF)])
    O.par_loop(O.K_U2V_ADJ, cc, L, [(sub(ocs, cl), X, 3, O.READ), (sub(osp, cl), u, 1, O.READ),
                                    (sub(osp, cl), w, 1, O.READ), (sub(osp, cl), Gr, 1, oacc, aG)])
    d = sampled_dofs(osp, sample, L)
    close_at(F.cpu().numpy(), Fr, aF, d)
    close_at(G.cpu().numpy(), Gr, aG, d)
    # adjoint against central differences of the GPU residual, h = 1e-6 (exact for a quadratic)
    dd = torch.from_numpy(meshgen.uniform_field(osp.ndofs, 1620)).to(dev)
    h = 1e-6
    Fp = E.residual_u2v(gm, cs, Xg, sp, ud + h * dd)
    Fm = E.residual_u2v(gm, cs, Xg, sp, ud - h * dd)
    jd = (Fp - Fm) / (2 * h)
    lhs, rhs = float(wd @ jd), float(G @ dd)
    assert abs(lhs - rhs) <= 1e-8 * float(wd.abs() @ jd.abs())


def test_fullsize_batched_64_meshes():
    bp = meshgen.batched_params(count=64, seed=1609)
    meshes, per, keep, base = [], [], [], []
    for i, (n, L) in enumerate(zip(bp.n, bp.layers)):
        m = meshgen.tri_mesh(n, seed=2104 + i, order="rcm")
        gm = E.Mesh(m.cells, m.xy, L)
        cs = E.Space(gm, "CG1xCG1", ncomp=3)
        sp = E.Space(gm, "CG1xCG1")
        X = E.extrude_coords(gm, cs)
        u = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 3000 + i)).to(dev)
        w = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 4000 + i)).to(dev)
        F, G = sp.zeros(), sp.zeros()
        meshes.append(gm)
        per.append([(cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, w, E.EXT_READ), (sp, F, E.EXT_INC),
                    (sp, G, E.EXT_INC)])
        keep.append((cs, sp))
        base.append(m)
    b = E.Batch(meshes, E.EXT_K_U2V_FWDADJ, per)
    for args in per:
        args[3][1].zero_()
        args[4][1].zero_()
    b.launch()
    E.ext_sync_check()
    # check the smallest, the largest and two more meshes on sampled cells
    sizes = [m.ncells * L for m, L in zip(base, bp.layers)]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 40}
    rng = np.random.default_rng(9)
    for i in sorted(pick):
        m, L = base[i], bp.layers[i]
        ocs, X = O.coords(m.cells, m.xy, L)
        osp = O.number(m.cells, m.nverts, L, P1)
        sample = rng.choice(m.ncells, 25, replace=False)
        cl = closure(m.cells, sample)
        cc = np.ascontiguousarray(m.cells[cl])
        u = per[i][1][1].cpu().numpy()
        w = per[i][2][1].cpu().numpy()
        Fr, aF, Gr, aG = (np.zeros(osp.ndofs) for _ in range(4))
        O.par_loop(O.K_U2V, cc, L, [(sub(ocs, cl), X, 3, O.READ), (sub(osp, cl), u, 1, O.READ),
                                    (sub(osp, cl), Fr, 1, O.INC, aF)])
        O.par_loop(O.K_U2V_ADJ, cc, L, [(sub(ocs, cl), X, 3, O.READ), (sub(osp, cl), u, 1, O.READ),
                                        (sub(osp, cl), w, 1, O.READ), (sub(osp, cl), Gr, 1, O.INC, aG)])
        d = sampled_dofs(osp, sample, L)
        close_at(per[i][3][1].cpu().numpy(), Fr, aF, d)
        close_at(per[i][4][1].cpu().numpy(), Gr, aG, d)


def test_fullsize_variable_layers_1M():
    """The bathymetry workload of the variable-layer benchmark (999,698 columns,
    top level 100): numbering, coordinates and DG1 interpolation compared in
    full, the mass action and the DG1xDG1 interior-facet jump on sampled
    columns."""
    m = meshgen.tri_mesh(707, seed=1604, order="rcm")
    first, lay = meshgen.column_layers(m, 100, 1674, "bathymetry")
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    p1 = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG1xDG1")
    ocs, X = O.coords_var(m.cells, m.xy, first, lay)
    op1 = O.number_var(m.cells, m.nverts, first, lay, P1)
    odg = O.number_var(m.cells, m.nverts, first, lay, O.DELTA["DG1xDG1"])
    for g, o in ((p1, op1), (dg, odg), (cs, ocs)):
        gmap, goff = g.stencil_map()
        assert g.ndofs == o.ndofs
        np.testing.assert_array_equal(gmap, o.map)
        np.testing.assert_array_equal(goff, o.offset)
    Xg = E.extrude_coords(gm, cs)
    np.testing.assert_array_equal(Xg.cpu().numpy(), X)
    x = meshgen.uniform_field(op1.ndofs, 1675)
    xd = torch.from_numpy(x).to(dev)
    y, out = p1.zeros(), dg.zeros()
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xg, E.EXT_READ), (p1, xd, E.EXT_READ), (p1, y, E.EXT_INC))
    E.par_loop(gm, E.EXT_K_INTERP_DG1, (p1, xd, E.EXT_READ), (dg, out, E.EXT_WRITE))
    u = meshgen.uniform_field(odg.ndofs, 1676)
    r = dg.zeros()
    E.par_loop(gm, E.EXT_K_HFACET_JUMP, (cs, Xg, E.EXT_READ), (dg, torch.from_numpy(u).to(dev), E.EXT_READ),
               (dg, r, E.EXT_INC))
    E.ext_sync_check()
    rng = np.random.default_rng(10)
    sample = np.concatenate([rng.choice(m.ncells, 300, replace=False), [0, m.ncells - 1]])
    cl = closure(m.cells, sample)
    cc = np.ascontiguousarray(m.cells[cl])

    def subv(space, idx):
        return O.Space(delta=space.delta, layers=space.layers, ndofs=space.ndofs, k=space.k,
                       map=np.ascontiguousarray(space.map[idx]), offset=space.offset)

    def dofs_of(space, idx):
        out_ = [space.map[c].astype(np.int64)[None, :] + np.arange(lay[c])[:, None] * space.offset[None, :]
                for c in idx]
        return np.unique(np.concatenate([o.ravel() for o in out_]))

    ref, absr = np.zeros(op1.ndofs), np.zeros(op1.ndofs)
    O.par_loop(O.K_MASS, cc, op1.layers, [(subv(ocs, cl), X, 3, O.READ), (subv(op1, cl), x, 1, O.READ),
                                          (subv(op1, cl), ref, 1, O.INC, absr)],
               cell_first=first[cl], cell_layers=lay[cl])
    close_at(y.cpu().numpy(), ref, absr, dofs_of(op1, sample))
    oref = np.full(odg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, np.ascontiguousarray(m.cells[sample]), op1.layers,
               [(subv(op1, sample), x, 1, O.READ), (subv(odg, sample), oref, 1, O.WRITE)],
               cell_first=first[sample], cell_layers=lay[sample])
    d = dofs_of(odg, sample)
    np.testing.assert_array_equal(out.cpu().numpy()[d], oref[d])
    # the jump couples only the layers of one column: the sample alone is its closure
    jref, jabs = np.zeros(odg.ndofs), np.zeros(odg.ndofs)
    O.set_tp_element(O.DG1, O.DG1)
    O.par_loop(O.K_HFACET_JUMP, np.ascontiguousarray(m.cells[sample]), op1.layers,
               [(subv(ocs, sample), X, 3, O.READ), (subv(odg, sample), u, 1, O.READ),
                (subv(odg, sample), jref, 1, O.INC, jabs)], cell_first=first[sample], cell_layers=lay[sample])
    close_at(r.cpu().numpy(), jref, jabs, d)
