"""P1xP1 right-hand side / mass action on coordinate fields that are not a
flat, straight extrusion: terrain-following levels (vertical columns, every
prism's top and bottom faces tilted; the heights a fixed profile scaled per
column), bent levels (vertical columns, no such profile) and sheared columns
(tilted vertical edges), over a million (column, level) items so that the
split forms run.  Every form of the launch (ext_set_option(EXT_OPT_P1_FORM,
...)) must match the oracle within 1e-12 of its absolute contribution sums,
with WRITE and INC access.  The probe of the automatic form picks the flat
gather on a flat extrusion, the terrain-following gather on terrain levels
and the cell loop otherwise; when its sample misses a perturbed column, the
gather form recomputes the DoFs next to it one by one."""
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
FORMS = ["auto", "split", "gather", "factored", "unfactored", "cells", "single"]


def close(got, want, absref, rtol=1e-12):
    err = np.abs(np.asarray(got) - want)
    bad = np.nonzero(~(err <= rtol * absref + 1e-300))[0]
    assert bad.size == 0, f"{bad.size} entries off; worst rel {(err / (absref + 1e-300)).max():.3e} at {bad[:5]}"


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


FLAT = {"optimistic": E.EXT_P1_FLAT_OPTIMISTIC, "fused": E.EXT_P1_FLAT_FUSED, "split": E.EXT_P1_FLAT_SPLIT}


@pytest.fixture(autouse=True, params=list(FLAT))
def flat(request):
    """Every test runs with each form of the flat gather (EXT_OPT_P1_FLAT):
    optimistic (one pass with the straightness bits set beside it, then a
    fix-up of the DoFs next to a DoF that is not straight; WRITE only, INC
    takes the split form), one pass with every row entry checked, and vertex
    pass + gather."""
    old = E.ext_get_option(E.EXT_OPT_P1_FORM)
    oldf = E.ext_get_option(E.EXT_OPT_P1_FLAT)
    E.ext_set_option(E.EXT_OPT_P1_FLAT, FLAT[request.param])
    yield request.param
    E.ext_set_option(E.EXT_OPT_P1_FORM, old)
    E.ext_set_option(E.EXT_OPT_P1_FLAT, oldf)


_cache = {}


def case(kind, n=71, layers=100):
    """Mesh, spaces and the oracle's mass action on a seeded geometry."""
    key = (kind, n, layers)
    if key in _cache:
        return _cache[key]
    m = meshgen.tri_mesh(n, seed=880 + n, order="rcm")
    csp, Xflat = O.coords(m.cells, m.xy, layers)
    if kind == "flat":
        X = Xflat
    else:
        X = meshgen.level_coords(m, layers, seed=881, kind=kind).reshape(-1)
    osp = O.number(m.cells, m.nverts, layers, P1)
    f = meshgen.uniform_field(osp.ndofs, 882)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    gm = E.Mesh(m.cells, m.xy, layers)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    out = (m, gm, cs, ps, torch.from_numpy(X).to(dev), torch.from_numpy(f).to(dev), ref, absr)
    _cache[key] = out
    return out


def run(gm, cs, ps, Xd, fd, access, init=None):
    b = torch.full((ps.ndofs,), float("nan"), dtype=torch.float64, device=dev) if init is None else init.clone()
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, Xd, E.EXT_READ), (ps, fd, E.EXT_READ), (ps, b, access))
    E.ext_sync_check()
    return host(b)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("kind", ["terrain", "wavy", "tilted"])
def test_every_form_on_non_flat_geometry(kind, form):
    m, gm, cs, ps, Xd, fd, ref, absr = case(kind)
    assert m.ncells * 101 >= 1_000_000
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.P1_FORMS[form])
    close(run(gm, cs, ps, Xd, fd, E.EXT_WRITE), ref, absr)
    init = torch.full((ps.ndofs,), 0.5, dtype=torch.float64, device=dev)
    close(run(gm, cs, ps, Xd, fd, E.EXT_INC, init), ref + 0.5, absr + 0.5)


def test_every_prism_of_the_terrain_is_non_straight():
    """The terrain field leaves no prism with a flat top face, so no part of
    the launch can take the tensor-product shortcut."""
    m, gm, cs, ps, Xd, fd, ref, absr = case("terrain")
    Z = host(Xd).reshape(m.nverts, 101, 3)[:, :, 2]
    zt = Z[m.cells][:, :, 1:]  # (cells, 3 vertices, levels 1..100)
    assert np.all((zt[:, 0] != zt[:, 1]) | (zt[:, 1] != zt[:, 2]))


@pytest.mark.parametrize("base", ["flat", "terrain"])
@pytest.mark.parametrize("column,mode", [(1, "gather"), (2, "cells")])
def test_probe_sample_and_recorded_dofs(base, column, mode):
    """A flat or terrain-following extrusion with one perturbed vertex
    column.  The probe samples every second column on this mesh (5,184
    vertex columns, about 4,096 sampled): column 1 escapes it and the gather
    form (flat or terrain-following) recomputes the DoFs next to that column
    one by one; column 2 is sampled and the whole launch runs as the cell
    loop.  Both match the oracle."""
    n, layers = 71, 100
    m = meshgen.tri_mesh(n, seed=880 + n, order="rcm")
    assert m.nverts == 5184
    csp, X = O.coords(m.cells, m.xy, layers)
    if base == "terrain":
        X = meshgen.level_coords(m, layers, seed=884, kind="terrain").reshape(-1)
    Xr = X.reshape(m.nverts, layers + 1, 3).copy()
    Xr[column, 3:60, 2] += 0.2 / layers        # levels off their heights
    Xr[column, 70:, 0] += 0.3 / n              # and a leaning top part
    X = Xr.reshape(-1)
    osp = O.number(m.cells, m.nverts, layers, P1)
    f = meshgen.uniform_field(osp.ndofs, 883)
    ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
    O.par_loop(O.K_MASS, m.cells, layers, [(csp, X, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
    gm = E.Mesh(m.cells, m.xy, layers)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    ps = E.Space(gm, "CG1xCG1")
    Xd, fd = torch.from_numpy(X).to(dev), torch.from_numpy(f).to(dev)
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_SPLIT)
    a = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    b = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    close(a, ref, absr)
    close(b, ref, absr)
    # the gather form writes every DoF from one thread in a fixed order:
    # launches agree bit for bit; the cell loop adds with atomics
    if mode == "gather":
        assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_terrain_takes_the_terrain_following_gather():
    """On terrain-following levels the automatic split form is the gather
    form (bitwise reproducible from launch to launch), and it differs from the
    flat-gather-without-probe result only by rounding (that form recomputes
    every DoF with the element rule)."""
    m, gm, cs, ps, Xd, fd, ref, absr = case("terrain")
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_SPLIT)
    a = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    b = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    close(a, ref, absr)
    assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_flat_extrusion_takes_the_gather_form():
    """On the flat extrusion the automatic split form gives the gather
    form's result bit for bit (the cell loop would not, in general)."""
    m, gm, cs, ps, Xd, fd, ref, absr = case("flat")
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_SPLIT)
    a = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_GATHER)
    b = run(gm, cs, ps, Xd, fd, E.EXT_WRITE)
    close(a, ref, absr)
    assert np.array_equal(a.view(np.int64), b.view(np.int64))
