"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs: numbering and maps bit-exact, data moves bit-exact, FP64
assembly within 1e-12 of the oracle's absolute contribution sums A_i
(|y_i - y_i^oracle| <= 1e-12 * A_i + 1e-300, which allows any summation
order, FMA contraction and atomic ordering)."""
import numpy as np
import pytest

import meshgen
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1604_05937_gb300 as E  # noqa: E402

RTOL = 1e-12
dev = torch.device("cuda:0")


def close(got, want, absref, rtol=RTOL):
    got = np.asarray(got)
    err = np.abs(got - want)
    bound = rtol * absref + 1e-300
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, (f"{bad.size} entries off; worst rel "
                           f"{(err / (absref + 1e-300)).max():.3e} at {bad[:5]}")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def mesh_pair(m, layers):
    """(GPU Mesh, oracle coords space, oracle coords) for a base mesh."""
    gm = E.Mesh(m.cells, m.xy, layers)
    csp, X = O.coords(m.cells, m.xy, layers)
    return gm, csp, X


TRI_SPACES = ["CG1xCG1", "CG1xDG0", "CG1xDG1", "DG0xCG1", "DG0xDG0", "DG0xDG1", "DG1xCG1", "DG1xDG0",
              "DG1xDG1"]


# ------------------------------------------------------------------ numbering
@pytest.mark.parametrize("name", TRI_SPACES + ["ALL1"])
@pytest.mark.parametrize("n,layers,order", [(3, 1, "rcm"), (7, 5, "random"), (13, 33, "rcm")])
def test_numbering_bit_exact_prisms(name, n, layers, order):
    m = meshgen.tri_mesh(n, seed=100 + n, order=order)
    delta = (1, 1, 1, 1, 1, 1) if name == "ALL1" else O.DELTA[name]
    gm = E.Mesh(m.cells, m.xy, layers)
    gs = E.Space(gm, delta)
    osp = O.number(m.cells, m.nverts, layers, delta)
    gmap, goff = gs.stencil_map()
    assert gs.ndofs == osp.ndofs and gs.k == osp.k
    np.testing.assert_array_equal(gmap, osp.map)
    np.testing.assert_array_equal(goff, osp.offset)


@pytest.mark.parametrize("name", ["Q2xP2", "DG2hex", "CG1xCG1"])
@pytest.mark.parametrize("n,layers", [(2, 1), (5, 7), (9, 40)])
def test_numbering_bit_exact_hexes(name, n, layers):
    m = meshgen.quad_mesh(n, seed=200 + n, order="random")
    gm = E.Mesh(m.cells, m.xy, layers)
    gs = E.Space(gm, O.DELTA[name])
    osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    gmap, goff = gs.stencil_map()
    assert gs.ndofs == osp.ndofs
    np.testing.assert_array_equal(gmap, osp.map)
    np.testing.assert_array_equal(goff, osp.offset)
    assert gm.N[1] == O.derive_edges(m.cells, m.nverts)[1]


@pytest.mark.parametrize("kind", [3, 4])
def test_extrusion_bit_exact(kind):
    layers = 11
    m = meshgen.tri_mesh(9, seed=5, order="random") if kind == 3 else meshgen.quad_mesh(8, seed=5)
    gm, csp, X = mesh_pair(m, layers)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    Xg = E.extrude_coords(gm, cs)
    np.testing.assert_array_equal(host(Xg), X)


# ------------------------------------------------------------------ moves
@pytest.mark.parametrize("name", ["DG0xDG0", "DG1xDG1", "DG1xDG0"])
@pytest.mark.parametrize("layers", [1, 7, 64])
def test_dg_copy_bit_exact(name, layers):
    m = meshgen.tri_mesh(10, seed=7, order="random")
    gm = E.Mesh(m.cells, m.xy, layers)
    gs = E.Space(gm, O.DELTA[name])
    a = meshgen.uniform_field(gs.ndofs, 8)
    out = torch.full((gs.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_COPY_DG, (gs, to_dev(a), E.EXT_READ), (gs, out, E.EXT_WRITE))
    osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    ref = np.full(osp.ndofs, np.nan)
    O.par_loop(O.K_COPY, m.cells, layers, [(osp, a, 1, O.READ), (osp, ref, 1, O.WRITE)])
    np.testing.assert_array_equal(host(out), ref)


@pytest.mark.parametrize("layers", [1, 5, 32, 100])
def test_dg1_interpolation_bit_exact(layers):
    m = meshgen.tri_mesh(12, seed=9, order="random")
    gm = E.Mesh(m.cells, m.xy, layers)
    p1 = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG1xDG1")
    x = meshgen.uniform_field(p1.ndofs, 10)
    out = torch.full((dg.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_INTERP_DG1, (p1, to_dev(x), E.EXT_READ), (dg, out, E.EXT_WRITE))
    op1 = O.number(m.cells, m.nverts, layers, P1)
    odg = O.number(m.cells, m.nverts, layers, O.DELTA["DG1xDG1"])
    ref = np.full(odg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, m.cells, layers, [(op1, x, 1, O.READ), (odg, ref, 1, O.WRITE)])
    np.testing.assert_array_equal(host(out), ref)


P1 = O.DELTA["CG1xCG1"]


# ------------------------------------------------------------------ P1xP1 mass / RHS
def _mass_case(m, layers, f_of_X=None, seed=1, perturb=0.0, kernel=None):
    gm, csp, X = mesh_pair(m, layers)
    if perturb:
        rng = np.random.default_rng(seed + 99)
        X = X + perturb * rng.uniform(-1, 1, X.size) / (m.n * max(layers, 1))
    osp = O.number(m.cells, m.nverts, layers, P1)
    Xr = X.reshape(-1, 3)
    f = f_of_X(Xr) if f_of_X is not None else meshgen.uniform_field(osp.ndofs, seed)
    ref = np.zeros(osp.ndofs)
    absr = np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    b = ps.zeros()
    k = kernel if kernel is not None else E.EXT_K_MASS_P1P1
    E.par_loop(gm, k, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_INC))
    E.ext_sync_check()
    return host(b), ref, absr


@pytest.mark.parametrize("n,layers,order", [(4, 1, "rcm"), (9, 3, "random"), (17, 31, "rcm"), (23, 32, "random"),
                                            (11, 100, "rcm"), (6, 257, "rcm")])
def test_mass_action_parity(n, layers, order):
    m = meshgen.tri_mesh(n, seed=300 + n, order=order)
    got, ref, absr = _mass_case(m, layers)
    close(got, ref, absr)


@pytest.mark.parametrize("n,layers,var", [(9, 3, False), (12, 1, False), (23, 32, False), (72, 100, False),
                                          (11, 9, True), (72, 100, True)])
def test_mass_action_parity_write(n, layers, var):
    """WRITE access overwrites the output with the assembled result: the
    output starts as NaN, every DoF must come out equal to the oracle's sum
    (constant and variable layers; the last cases are over a million items,
    so the split forms run)."""
    m = meshgen.tri_mesh(n, seed=310 + n, order="rcm")
    if var:
        first, lay = meshgen.column_layers(m, layers, 311, "bathymetry")
        gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
        csp, X = O.coords_var(m.cells, m.xy, first, lay)
        osp = O.number_var(m.cells, m.nverts, first, lay, P1)
        kw = dict(cell_first=first, cell_layers=lay)
    else:
        gm = E.Mesh(m.cells, m.xy, layers)
        csp, X = O.coords(m.cells, m.xy, layers)
        osp = O.number(m.cells, m.nverts, layers, P1)
        kw = {}
    f = meshgen.uniform_field(osp.ndofs, 312)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS, m.cells, csp.layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ),
                                               (osp, ref, 1, O.INC, absr)], **kw)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    b = torch.full((ps.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_WRITE))
    E.ext_sync_check()
    got = host(b)
    assert np.isfinite(got).all()
    close(got, ref, absr)
    # a second WRITE gives the same values, a following INC doubles them
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_INC))
    E.ext_sync_check()
    close(host(b), 2 * ref, 2 * absr)


def test_rhs_sin_cos_z_parity():
    m = meshgen.tri_mesh(30, seed=1604, order="rcm")  # the 1,800-triangle, 10-layer case
    f = lambda X: np.sin(X[:, 0]) * np.cos(X[:, 1]) * X[:, 2]
    got, ref, absr = _mass_case(m, 10, f_of_X=f, kernel=E.EXT_K_RHS_P1P1)
    close(got, ref, absr)
    assert abs(got.sum() - ref.sum()) < 1e-14


def test_mass_general_geometry_fallback():
    """Perturbed (non-straight) coordinates take the full-quadrature path."""
    m = meshgen.tri_mesh(8, seed=41, order="random")
    got, ref, absr = _mass_case(m, 9, perturb=0.05)
    close(got, ref, absr)


@pytest.mark.parametrize("layers", [100, 7])
@pytest.mark.parametrize("with_xy", [True, False])
def test_mass_general_geometry_partial(layers, with_xy):
    """Straight prisms except near a few vertex columns: some columns are
    moved in x, y from a level upwards (from level 0: a vertical column off
    the mesh's base coordinates), some have one level lifted in z, so warp
    steps of the cell pass mix straight and general prisms, and deferred steps
    must take back the vertex part the vertex pass added for them.  The mesh
    has its base coordinates or not (the factored form then takes its
    reference x, y from the field's level 0).  Over a million (column, level)
    items at 100 layers: the factored split form."""
    n = 72 if layers == 100 else 40
    m = meshgen.tri_mesh(n, seed=45, order="rcm")
    gm = E.Mesh(m.cells, m.xy if with_xy else None, layers, nverts=m.nverts)
    csp, X = O.coords(m.cells, m.xy, layers)
    osp = O.number(m.cells, m.nverts, layers, P1)
    Xr = X.reshape(-1, 3).copy()
    rng = np.random.default_rng(46)
    L1 = layers + 1
    lean = rng.choice(m.nverts, m.nverts // 40, replace=False)
    # the CG1xCG1 column of vertex v is DoFs v * L1 .. v * L1 + layers (Algorithm 1)
    for v in lean:
        lv = int(rng.integers(0, layers + 1))
        Xr[v * L1 + lv:v * L1 + L1, 0] += 0.1 / n
        Xr[v * L1 + lv:v * L1 + L1, 1] -= 0.05 / n
    lift = rng.choice(np.setdiff1d(np.arange(m.nverts), lean), m.nverts // 40, replace=False)
    for v in lift:
        lv = int(rng.integers(0, L1))
        Xr[v * L1 + lv, 2] += 0.3 / layers
    X = Xr.reshape(-1)
    f = meshgen.uniform_field(osp.ndofs, 47)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    b = ps.zeros()
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, to_dev(X), E.EXT_READ), (ps, to_dev(f), E.EXT_READ), (ps, b, E.EXT_INC))
    E.ext_sync_check()
    close(host(b), ref, absr)


@pytest.mark.parametrize("form", [{"EXTMESH_P1_FORM": "split"}, {"EXTMESH_P1_FORM": "split", "EXTMESH_P1_FLAT": "fused"},
                                  {"EXTMESH_P1_FORM": "single"},
                                  {"EXTMESH_P1_FORM": "gather"}, {"EXTMESH_P1_FORM": "unfactored"},
                                  {"EXTMESH_P1_FORM": "factored"}, {"EXTMESH_P1_FORM": "cells"},
                                  {"EXTMESH_TP_FLAGS": "1"}, {"EXTMESH_TP_FLAGS": "1", "EXTMESH_TP_LEVELS": "1"},
                                  {"EXTMESH_TP_FLAGS": "0", "EXTMESH_TP_LEVELS": "1"},
                                  {"EXTMESH_TP_FLAGS": "1", "EXTMESH_TP_OPTIMISTIC": "0"}],
                         ids=["split", "split-flat-fused", "single", "gather", "split-unfactored", "split-factored",
                              "cells", "tp-flags",
                              "tp-levels-flags", "tp-levels", "tp-flags-not-optimistic"])
def test_mass_forced_form(form):
    """Every form of the P1xP1 launch passes the same parity tests, each
    forced at every size by EXTMESH_P1_FORM (read once per process, so in a
    child process): the split form (a probe of the coordinates picks the
    gather form on a flat, straight extrusion -- Mv per vertex column, then
    the base mass matrix's vertex rows per level -- and the cell loop
    otherwise), the gather form without the probe, the factored and
    unfactored cell passes over vertical sums, the cell loop (one element
    vector per prism), and the single-pass kernel (the default below a
    million items, and the fallback when the split forms' scratch cannot be
    allocated); and the nine-space kernels' flagged form (straightness bits
    per coordinate DoF, the default from a million items) forced at every
    size by EXTMESH_TP_FLAGS, with and without the level kernel for DG x CG1
    (EXTMESH_TP_LEVELS=1: the DoFs shared by consecutive layers merged in
    registers), and with the optimistic WRITE form of the DG x DG spaces
    turned off (EXTMESH_TP_OPTIMISTIC=0: flags first, then the element
    vectors)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **form)
    sel = "mass_action_parity or rhs_sin_cos or mass_general_geometry or volume_pin or tp_parity or var_mass"
    if "EXTMESH_TP_OPTIMISTIC" in form:
        sel += " or tp_flags_partial"
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(root, "tests", "test_gpu_parity.py"),
                        os.path.join(root, "tests", "test_gpu_var_facets.py"), "-k", sel],
                       cwd=root, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:]
    assert " passed" in r.stdout


@pytest.mark.parametrize("layers", [1, 2, 100])
def test_mass_gather_form_deterministic(layers):
    """The gather form writes every DoF from one thread in a fixed order, so
    two launches give bitwise equal results; WRITE and INC agree with the
    oracle; and a NaN in f reaches exactly the DoFs whose stencil holds it
    (they are recomputed by the general path, which yields NaN as well),
    leaving every other DoF equal to the oracle's."""
    n = {1: 710, 2: 420, 100: 72}[layers]  # over a million (column, level) items
    m = meshgen.tri_mesh(n, seed=320 + layers, order="rcm")
    old_form = E.ext_get_option(E.EXT_OPT_P1_FORM)
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_SPLIT if layers >= 32 else E.EXT_P1_GATHER)
    try:
        gm, csp, X = mesh_pair(m, layers)
        osp = O.number(m.cells, m.nverts, layers, P1)
        f = meshgen.uniform_field(osp.ndofs, 321)
        ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
        O.par_loop(O.K_MASS, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
        cs = E.Space(gm, "CG1xCG1", ncomp=3)
        ps = E.Space(gm, "CG1xCG1")
        Xd, fd = to_dev(X), to_dev(f)
        outs = []
        for _ in range(2):
            b = torch.full((ps.ndofs,), float("nan"), dtype=torch.float64, device=dev)
            E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xd, E.EXT_READ), (ps, fd, E.EXT_READ), (ps, b, E.EXT_WRITE))
            E.ext_sync_check()
            outs.append(host(b))
        assert np.array_equal(outs[0].view(np.int64), outs[1].view(np.int64))
        close(outs[0], ref, absr)
        b = to_dev(np.full(osp.ndofs, 0.25))
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xd, E.EXT_READ), (ps, fd, E.EXT_READ), (ps, b, E.EXT_INC))
        E.ext_sync_check()
        close(host(b), ref + 0.25, absr + 0.25)
        # one NaN in f at vertex v0, level 0: the DoFs of v0 and its neighbours at
        # levels 0 and 1 become NaN, all others keep the oracle's value
        L1 = layers + 1
        v0 = m.nverts // 2
        fn = f.copy()
        fn[v0 * L1] = np.nan
        b = ps.zeros()
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xd, E.EXT_READ), (ps, to_dev(fn), E.EXT_READ), (ps, b, E.EXT_WRITE))
        E.ext_sync_check()
        got = host(b)
        nb = np.unique(m.cells[np.any(m.cells == v0, axis=1)].reshape(-1))
        hit = np.zeros(osp.ndofs, dtype=bool)
        for v in nb:
            hit[v * L1:v * L1 + 2] = True
        assert np.isnan(got[hit]).all()
        close(got[~hit], ref[~hit], absr[~hit])
    finally:
        E.ext_set_option(E.EXT_OPT_P1_FORM, old_form)


def test_mass_volume_pin_on_gpu():
    m = meshgen.tri_mesh(20, seed=42)
    got, ref, absr = _mass_case(m, 13, f_of_X=lambda X: np.ones(X.shape[0]))
    assert abs(got.sum() - 1.0) < 1e-13


# ------------------------------------------------------------------ u^2 v and adjoint
def _u2v_case(m, layers, delta, mode, perturb=0.0, seed=3):
    gm, csp, X = mesh_pair(m, layers)
    if perturb:
        rng = np.random.default_rng(seed + 7)
        X = X + perturb * rng.uniform(-1, 1, X.size) / (m.n * layers)
    osp = O.number(m.cells, m.nverts, layers, delta)
    dg = delta == O.DELTA["DG2hex"]
    acc = O.WRITE if dg else O.INC
    u = meshgen.uniform_field(osp.ndofs, seed)
    w = meshgen.uniform_field(osp.ndofs, seed + 1)
    F = np.zeros(osp.ndofs); aF = np.zeros(osp.ndofs)
    G = np.zeros(osp.ndofs); aG = np.zeros(osp.ndofs)
    O.par_loop(O.K_U2V, m.cells, layers, [(csp, X, 3, O.READ), (osp, u, 1, O.READ), (osp, F, 1, acc, aF)])
    O.par_loop(O.K_U2V_ADJ, m.cells, layers,
               [(csp, X, 3, O.READ), (osp, u, 1, O.READ), (osp, w, 1, O.READ), (osp, G, 1, acc, aG)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, delta)
    Xd, ud, wd = to_dev(X), to_dev(u), to_dev(w)
    gacc = E.EXT_WRITE if dg else E.EXT_INC
    Fg = sp.zeros(); Gg = sp.zeros()
    if mode == "separate":
        E.par_loop(gm, E.EXT_K_U2V_FWD, (cs, Xd, E.EXT_READ), (sp, ud, E.EXT_READ), (sp, Fg, gacc))
        E.par_loop(gm, E.EXT_K_U2V_ADJ, (cs, Xd, E.EXT_READ), (sp, ud, E.EXT_READ), (sp, wd, E.EXT_READ),
                   (sp, Gg, gacc))
    else:
        E.par_loop(gm, E.EXT_K_U2V_FWDADJ, (cs, Xd, E.EXT_READ), (sp, ud, E.EXT_READ), (sp, wd, E.EXT_READ),
                   (sp, Fg, gacc), (sp, Gg, gacc))
    E.ext_sync_check()
    close(host(Fg), F, aF)
    close(host(Gg), G, aG)


@pytest.mark.parametrize("mode", ["separate", "fused"])
@pytest.mark.parametrize("n,layers", [(5, 1), (9, 7), (13, 40)])
def test_u2v_prism_parity(mode, n, layers):
    _u2v_case(meshgen.tri_mesh(n, seed=400 + n, order="random"), layers, P1, mode)


@pytest.mark.parametrize("name", ["Q2xP2", "DG2hex"])
@pytest.mark.parametrize("mode", ["separate", "fused"])
@pytest.mark.parametrize("n,layers", [(3, 1), (6, 5), (9, 33)])
def test_u2v_hex_parity(name, mode, n, layers):
    _u2v_case(meshgen.quad_mesh(n, seed=500 + n, order="random"), layers, O.DELTA[name], mode)


@pytest.mark.parametrize("kind,delta", [(3, P1), (4, O.DELTA["Q2xP2"]), (4, O.DELTA["DG2hex"])])
def test_u2v_general_geometry_fallback(kind, delta):
    m = meshgen.tri_mesh(6, seed=61) if kind == 3 else meshgen.quad_mesh(4, seed=61)
    _u2v_case(m, 4, delta, "fused", perturb=0.05)


def test_residual_autograd_gradcheck():
    m = meshgen.quad_mesh(2, seed=71)
    layers = 2
    gm = E.Mesh(m.cells, m.xy, layers)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    X = E.extrude_coords(gm, cs)
    sp = E.Space(gm, "Q2xP2")
    Fn = E.ResidualFn()
    u = torch.tensor(meshgen.uniform_field(sp.ndofs, 72), device=dev, requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: Fn.apply(v, gm, cs, X, sp), (u,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_residual_adjoint_matches_finite_differences():
    m = meshgen.tri_mesh(10, seed=73, order="random")
    layers = 8
    gm = E.Mesh(m.cells, m.xy, layers)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    X = E.extrude_coords(gm, cs)
    sp = E.Space(gm, "CG1xCG1")
    u = to_dev(meshgen.uniform_field(sp.ndofs, 74))
    w = to_dev(meshgen.uniform_field(sp.ndofs, 75))
    d = to_dev(meshgen.uniform_field(sp.ndofs, 76))
    g = E.residual_u2v_adjoint(gm, cs, X, sp, u, w)
    h = 1e-6
    jd = (E.residual_u2v(gm, cs, X, sp, u + h * d) - E.residual_u2v(gm, cs, X, sp, u - h * d)) / (2 * h)
    lhs, rhs = float(w @ jd), float(g @ d)
    assert abs(lhs - rhs) <= 1e-8 * float(w.abs() @ jd.abs())
    # Euler identity: F homogeneous of degree 2
    F = E.residual_u2v(gm, cs, X, sp, u)
    assert abs(float(g @ u) - 2 * float(w @ F)) <= 1e-12 * float(g.abs() @ u.abs())


# ------------------------------------------------------------------ batched
def _batch_case(params, count=5, mode=E.EXT_K_U2V_FWDADJ):
    bp = meshgen.batched_params(count=count, seed=1700, cmin=50, cmax=3000, lmin=1, lmax=40)
    meshes, per, refs, keep = [], [], [], []
    for i, (n, L) in enumerate(zip(bp.n, bp.layers)):
        m = meshgen.tri_mesh(n, seed=1800 + i, order="rcm" if i % 2 else "random")
        gm, csp, X = mesh_pair(m, L)
        osp = O.number(m.cells, m.nverts, L, P1)
        u = meshgen.uniform_field(osp.ndofs, 1900 + i)
        w = meshgen.uniform_field(osp.ndofs, 2000 + i)
        F = np.zeros(osp.ndofs); aF = np.zeros(osp.ndofs)
        G = np.zeros(osp.ndofs); aG = np.zeros(osp.ndofs)
        O.par_loop(O.K_U2V, m.cells, L, [(csp, X, 3, O.READ), (osp, u, 1, O.READ), (osp, F, 1, O.INC, aF)])
        O.par_loop(O.K_U2V_ADJ, m.cells, L, [(csp, X, 3, O.READ), (osp, u, 1, O.READ), (osp, w, 1, O.READ),
                                             (osp, G, 1, O.INC, aG)])
        cs = E.Space(gm, "CG1xCG1", ncomp=3)
        sp = E.Space(gm, "CG1xCG1")
        Fg, Gg = sp.zeros(), sp.zeros()
        args = [(cs, to_dev(X), E.EXT_READ), (sp, to_dev(u), E.EXT_READ), (sp, to_dev(w), E.EXT_READ),
                (sp, Fg, E.EXT_INC), (sp, Gg, E.EXT_INC)]
        meshes.append(gm)
        per.append(args)
        refs.append((F, aF, G, aG, Fg, Gg))
        keep.append((cs, sp))
    b = E.Batch(meshes, mode, per, params=params)
    for (_, _, _, _, Fg, Gg) in refs:  # autotuning/capture leaves partial sums behind
        Fg.zero_()
        Gg.zero_()
    b.launch()
    E.ext_sync_check()
    for (F, aF, G, aG, Fg, Gg) in refs:
        close(host(Fg), F, aF)
        close(host(Gg), G, aG)
    return b


@pytest.mark.parametrize("params", [
    dict(cols_per_item=1, layer_tile=0, use_atomics=1, threads=256, ctas_per_sm=2),
    dict(cols_per_item=4, layer_tile=8, use_atomics=1, threads=128, ctas_per_sm=4),
    dict(cols_per_item=32, layer_tile=0, use_atomics=0, threads=256, ctas_per_sm=2),
    dict(cols_per_item=16, layer_tile=5, use_atomics=0, threads=64, ctas_per_sm=8),
])
def test_batched_parity_explicit_params(params):
    b = _batch_case(params)
    assert b.params == params


def test_batched_parity_autotuned_and_replayed():
    b = _batch_case(None)
    p = b.params
    assert p["cols_per_item"] >= 1 and p["threads"] in (64, 128, 256)


def test_batched_tuning_cache(tmp_path, monkeypatch):
    """The second plan of the same workload reads its parameters from the
    tuning cache (file of JSON lines) instead of timing the candidates again,
    and EXTMESH_TUNE=force re-tunes."""
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("EXTMESH_TUNE_CACHE", str(path))
    monkeypatch.setenv("EXTMESH_TUNE", "force")
    a = _batch_case(None)
    assert a.plan_info["source"] == "autotuned"
    assert path.exists() and '"params": [' in path.read_text()
    monkeypatch.delenv("EXTMESH_TUNE")
    b = _batch_case(None)
    assert b.plan_info["source"] == "cache"
    assert b.params == a.params
    assert b.plan_info["setup_seconds"] < a.plan_info["setup_seconds"]
    monkeypatch.setenv("EXTMESH_TUNE", "off")
    c = _batch_case(dict(cols_per_item=2, layer_tile=0, use_atomics=1, threads=256, ctas_per_sm=4))
    assert c.plan_info["source"] == "given"


# ------------------------------------------------------------------ edge cases
def test_empty_mesh_and_single_cell():
    cells = np.zeros((0, 3), dtype=np.int32)
    gm = E.Mesh(cells, np.zeros((0, 2)), 3, )
    sp = E.Space(gm, "DG0xDG0")
    assert sp.ndofs == 0
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    gm = E.Mesh(cells, xy, 1)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    X = E.extrude_coords(gm, cs)
    ps = E.Space(gm, "CG1xCG1")
    b = ps.zeros()
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, torch.ones(ps.ndofs, dtype=torch.float64, device=dev),
                                                             E.EXT_READ), (ps, b, E.EXT_INC))
    assert abs(float(b.sum()) - 0.5) < 1e-15


def test_argument_validation():
    m = meshgen.tri_mesh(3, seed=1)
    gm = E.Mesh(m.cells, m.xy, 2)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    dg = E.Space(gm, "DG0xDG0")
    X = E.extrude_coords(gm, cs)
    b = ps.zeros()
    with pytest.raises(E.ExtError, match="EXT_EINVAL"):
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, b, E.EXT_READ), (ps, b, E.EXT_WRITE))
    with pytest.raises(E.ExtError, match="wrong space"):
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (dg, dg.zeros(), E.EXT_READ), (ps, b, E.EXT_INC))
    with pytest.raises(E.ExtError, match="unknown kernel"):
        E.ext_par_loop(gm.handle, 99, [])
    # an INC output may not overlap an input, wholly or in part
    with pytest.raises(E.ExtError, match="overlaps"):
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, b, E.EXT_READ), (ps, b, E.EXT_INC))
    buf = torch.zeros(2 * ps.ndofs, dtype=torch.float64, device=dev)
    with pytest.raises(E.ExtError, match="overlaps"):
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, buf[:ps.ndofs], E.EXT_READ),
                   (ps, buf[ps.ndofs // 2:ps.ndofs // 2 + ps.ndofs], E.EXT_INC))
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, buf[:ps.ndofs], E.EXT_READ),
               (ps, buf[ps.ndofs:], E.EXT_INC))  # adjacent, not overlapping
    other = E.Mesh(m.cells, m.xy, 3)
    os_ = E.Space(other, "CG1xCG1")
    with pytest.raises(E.ExtError, match="another mesh"):
        E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (os_, os_.zeros(), E.EXT_READ), (ps, b, E.EXT_INC))
    deep = E.Mesh(np.array([[0, 1, 2]], dtype=np.int32), np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]),
                  100_000_000)
    with pytest.raises(E.ExtError, match="EXT_EOVERFLOW"):
        E.Space(deep, (0, 0, 0, 0, 0, 27))  # 2.7e9 DoFs do not fit int32


# ------------------------------------------------------------------ the nine prism spaces (Sec. 4.1.2)
@pytest.mark.parametrize("name,h,v", O.TP_PAIRS)
@pytest.mark.parametrize("n,layers,order,perturb", [(5, 1, "rcm", 0.0), (9, 7, "random", 0.0),
                                                    (13, 33, "rcm", 0.0), (6, 5, "random", 0.05)])
def test_mass_tp_parity(name, h, v, n, layers, order, perturb):
    m = meshgen.tri_mesh(n, seed=600 + n, order=order)
    gm, csp, X = mesh_pair(m, layers)
    if perturb:
        rng = np.random.default_rng(601)
        X = X + perturb * rng.uniform(-1, 1, X.size) / (m.n * layers)
    osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    f = meshgen.uniform_field(osp.ndofs, 602)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.set_tp_element(h, v)
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    check_tp_access(gm, cs, sp, X, f, ref, absr)


def check_tp_access(gm, cs, sp, X, f, ref, absr):
    """INC onto 0.25 everywhere, and WRITE onto NaN (every DoF overwritten)."""
    Xd, fd = to_dev(X), to_dev(f)
    b = torch.full((sp.ndofs,), 0.25, dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_MASS_TP, (cs, Xd, E.EXT_READ), (sp, fd, E.EXT_READ), (sp, b, E.EXT_INC))
    E.ext_sync_check()
    close(host(b), ref + 0.25, absr + 0.25)
    b = torch.full((sp.ndofs,), float("nan"), dtype=torch.float64, device=dev)
    E.par_loop(gm, E.EXT_K_MASS_TP, (cs, Xd, E.EXT_READ), (sp, fd, E.EXT_READ), (sp, b, E.EXT_WRITE))
    E.ext_sync_check()
    close(host(b), ref, absr)


@pytest.mark.parametrize("name", ["CG1xDG0", "CG1xDG1"])
@pytest.mark.parametrize("kind", ["flat", "terrain", "wavy", "tilted"])
def test_mass_tp_cgdg_geometry(name, kind):
    """CG1 x DG0 and CG1 x DG1 with WRITE from 32 layers take the gather path
    of the P1xP1 launch (row weights from this launch's coordinates, the
    gather beside the straightness flags): on a flat extrusion the flat
    gather, on terrain-following levels the depth-weighted gather with the
    model check, on bent levels and leaning columns the probe's cell-loop
    mode, where the nine-space cell kernel runs (b cleared first).  INC keeps
    the cell kernel on every geometry.  All match the oracle."""
    n, layers = 24, 40
    m = meshgen.tri_mesh(n, seed=660, order="rcm")
    gm = E.Mesh(m.cells, m.xy, layers)
    csp, X = O.coords(m.cells, m.xy, layers)
    if kind != "flat":
        X = meshgen.level_coords(m, layers, seed=661, kind=kind).reshape(-1)
    h = {"CG1": O.CG1, "DG0": O.DG0, "DG1": O.DG1}
    osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    f = meshgen.uniform_field(osp.ndofs, 662)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.set_tp_element(h[name[:3]], h[name[4:]])
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    check_tp_access(gm, cs, sp, X, f, ref, absr)


@pytest.mark.parametrize("name", ["DG0xDG0", "CG1xDG1", "DG1xCG1", "DG0xDG1", "DG0xCG1", "DG1xDG1", "DG1xDG0",
                                  "CG1xDG0"])
def test_mass_tp_flags_partial(name):
    """Over a million (column, layer) items the nine-space kernels take their
    flagged form (one straightness bit per coordinate DoF against the base
    coordinates and the level heights); columns moved in x, y from some level
    up, single lifted levels and a level-0 vertex moved off its base position
    must send exactly the prisms that touch them to the general 6-point rule.
    With WRITE the DG x DG spaces take the optimistic form (closed form for
    every prism beside the flag pass, then a fix-up launch over the prisms
    whose flags are not all set) and CG1 x DG the gather path (its fix-up
    recomputes the DoFs next to a moved DoF with the general rule), so the
    NaN that WRITE starts from must be overwritten everywhere and the moved
    prisms must come out of the fix-ups."""
    n, layers = 72, 100
    m = meshgen.tri_mesh(n, seed=650, order="rcm")
    gm = E.Mesh(m.cells, m.xy, layers)
    csp, X = O.coords(m.cells, m.xy, layers)
    Xr = X.reshape(-1, 3).copy()
    rng = np.random.default_rng(651)
    L1 = layers + 1
    lean = rng.choice(m.nverts, m.nverts // 40, replace=False)
    for v in lean:
        lv = int(rng.integers(0, L1))
        Xr[v * L1 + lv:v * L1 + L1, 0] += 0.1 / n
        Xr[v * L1 + lv:v * L1 + L1, 1] -= 0.05 / n
    lift = rng.choice(np.setdiff1d(np.arange(m.nverts), lean), m.nverts // 40, replace=False)
    for v in lift:
        Xr[v * L1 + int(rng.integers(0, L1)), 2] += 0.3 / layers
    X = Xr.reshape(-1)
    h = {"CG1": O.CG1, "DG0": O.DG0, "DG1": O.DG1}
    osp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    f = meshgen.uniform_field(osp.ndofs, 652)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.set_tp_element(h[name[:3]], h[name[4:]])
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, O.DELTA[name])
    check_tp_access(gm, cs, sp, X, f, ref, absr)
