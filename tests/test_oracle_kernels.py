"""Pins of the oracle's par_loop local kernels (Algorithm 3, Sec. 3.3, with the
residual of Sec. 4.1.1 and the nonlinear residual int u^2 v dx and its adjoint)
against closed forms, invariants, finite differences, exactness of Gauss rules
and a library Gauss-Legendre routine."""
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle as O

P1 = O.DELTA["CG1xCG1"]


def _mesh_space(m, layers, delta):
    sp = O.number(m.cells, m.nverts, layers, delta, keep_tables=True)
    csp, X = O.coords(m.cells, m.xy, layers)
    return sp, csp, X


def _mass(cells, layers, csp, X, sp, f, absd=None):
    b = np.zeros(sp.ndofs)
    args = [(csp, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC) + ((absd,) if absd is not None else ())]
    O.par_loop(O.K_MASS, cells, layers, args)
    return b


# ----------------------------------------------------------------------------- extrusion
@pytest.mark.parametrize("kind", [3, 4])
def test_extrusion_places_vertex_levels(kind):
    layers = 7
    m = meshgen.tri_mesh(5, seed=21, order="random") if kind == 3 else meshgen.quad_mesh(5, seed=21)
    csp = O.number(m.cells, m.nverts, layers, P1, keep_tables=True)
    _, X = O.coords(m.cells, m.xy, layers)
    X = X.reshape(-1, 3)
    dof = csp.first[0]  # (V, layers+1): DoF of vertex v at level l
    np.testing.assert_array_equal(X[dof, 0], np.repeat(m.xy[:, 0:1], layers + 1, 1))
    np.testing.assert_array_equal(X[dof, 1], np.repeat(m.xy[:, 1:2], layers + 1, 1))
    np.testing.assert_array_equal(X[dof, 2], np.tile(np.arange(layers + 1) / layers, (m.nverts, 1)))


# ----------------------------------------------------------------------------- mass / RHS
@pytest.mark.parametrize("order", ["rcm", "random"])
def test_rhs_of_one_is_volume(order):
    """int 1 * v dx summed over all v = |Omega| = 1 (partition of unity)."""
    layers = 4
    m = meshgen.tri_mesh(8, seed=3, order=order)
    sp, csp, X = _mesh_space(m, layers, P1)
    b = _mass(m.cells, layers, csp, X, sp, np.ones(sp.ndofs))
    assert abs(b.sum() - 1.0) < 1e-14
    assert np.all(b > 0)


def test_rhs_of_linear_is_exact():
    """f = x + y + z is in P1xP1, so sum_i b_i = int (x+y+z) = 3/2."""
    layers = 5
    m = meshgen.tri_mesh(7, seed=4)
    sp, csp, X = _mesh_space(m, layers, P1)
    Xr = X.reshape(-1, 3)
    b = _mass(m.cells, layers, csp, X, sp, Xr[:, 0] + Xr[:, 1] + Xr[:, 2])
    assert abs(b.sum() - 1.5) < 1e-14


def _one_prism(tri_xy, h=1.0):
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    xy = np.array(tri_xy, dtype=np.float64)
    return cells, xy


@pytest.mark.parametrize("tri", [[(0, 0), (1, 0), (0, 1)], [(0.1, 0.2), (0.9, 0.35), (0.3, 0.8)],
                                 [(0.3, 0.8), (0.9, 0.35), (0.1, 0.2)]])  # last one clockwise
def test_straight_prism_element_matrix_closed_form(tri):
    """On a straight prism the P1xP1 mass matrix is (A h / 72)(1+[a=a'])(1+[b=b'])."""
    cells, xy = _one_prism(tri)
    layers = 1
    sp = O.number(cells, 3, layers, P1)
    csp, X = O.coords(cells, xy, layers)
    p = np.array(tri)
    A = 0.5 * abs((p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1]))
    h = 1.0
    M = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(sp.ndofs)
        e[sp.map[0, j]] = 1.0
        b = _mass(cells, layers, csp, X, sp, e)
        M[:, j] = b[sp.map[0]]
    expect = np.empty((6, 6))
    for i in range(6):
        for j in range(6):
            a, bb = divmod(i, 2)
            a2, b2 = divmod(j, 2)
            expect[i, j] = A * h / 72.0 * (1 + (a == a2)) * (1 + (bb == b2))
    np.testing.assert_allclose(M, expect, rtol=1e-14, atol=1e-17)


def test_tilted_prism_volume_and_symmetry():
    """A prism whose top is the plane z = h + al*x + be*y (coordinates given
    directly, not extruded): sum_i int phi_i = volume = A (h + al xc + be yc),
    and the element matrix is symmetric."""
    tri = np.array([[0.1, 0.2], [0.9, 0.35], [0.3, 0.8]])
    h, al, be = 0.7, 0.3, -0.2
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    sp = O.number(cells, 3, 1, P1)
    X = np.zeros(sp.ndofs * 3).reshape(-1, 3)
    for a in range(3):
        X[sp.map[0, 2 * a]] = (tri[a, 0], tri[a, 1], 0.0)
        X[sp.map[0, 2 * a + 1]] = (tri[a, 0], tri[a, 1], h + al * tri[a, 0] + be * tri[a, 1])
    X = X.ravel()
    A = 0.5 * abs((tri[1, 0] - tri[0, 0]) * (tri[2, 1] - tri[0, 1]) - (tri[2, 0] - tri[0, 0]) * (tri[1, 1] - tri[0, 1]))
    xc, yc = tri.mean(0)
    b = _mass(cells, 1, sp, X, sp, np.ones(sp.ndofs))
    assert abs(b.sum() - A * (h + al * xc + be * yc)) < 1e-15
    M = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(sp.ndofs)
        e[sp.map[0, j]] = 1.0
        M[:, j] = _mass(cells, 1, sp, X, sp, e)[sp.map[0]]
    np.testing.assert_allclose(M, M.T, rtol=1e-14)
    # not a straight-prism matrix: the column height differs between vertices
    assert abs(M[2, 2] - M[0, 0]) > 1e-2 * M[0, 0]


@pytest.mark.parametrize("n,layers,order", [(6, 4, "rcm"), (9, 7, "random")])
def test_mass_is_kronecker_product_on_straight_extrusions(n, layers, order):
    """On a straight extrusion with flat levels the P1xP1 mass matrix is
    Mh (x) Mv: Mh the base triangulation's P1 mass matrix as vertex rows (the
    weight of neighbour j is the sum of |2A_c|/144 over the cells holding edge
    (a, j), the diagonal weight the row's sum) and Mv the column's
    |h_{m-1}| f_{m-1} + 2 (|h_{m-1}| + |h_m|) f_m + |h_m| f_{m+1} -- the
    factorisation the library's gather form evaluates.  Built here with numpy
    from the base mesh alone, it equals the oracle's cell-by-cell assembly
    (6-point rule, full Jacobian) within the parity tolerance; non-uniform
    layer heights make Mv level dependent."""
    m = meshgen.tri_mesh(n, seed=170 + n, order=order)
    sp, csp, X = _mesh_space(m, layers, P1)
    # non-uniform flat levels: move every level to z_m = (m / L)^1.5
    Xr = X.reshape(-1, 3).copy()
    lev = np.tile(np.arange(layers + 1), m.nverts)  # level of CG1xCG1 DoF v (L+1) + m
    Xr[:, 2] = (lev / layers) ** 1.5
    X = Xr.reshape(-1)
    f = meshgen.uniform_field(sp.ndofs, 171)
    absr = np.zeros(sp.ndofs)
    ref = _mass(m.cells, layers, csp, X, sp, f, absr)
    # Mh as vertex rows
    V = m.nverts
    xy = m.xy
    c = m.cells
    alpha = np.abs((xy[c[:, 1], 0] - xy[c[:, 0], 0]) * (xy[c[:, 2], 1] - xy[c[:, 0], 1])
                   - (xy[c[:, 2], 0] - xy[c[:, 0], 0]) * (xy[c[:, 1], 1] - xy[c[:, 0], 1])) / 144.0
    Mh = np.zeros((V, V))
    for k in range(3):
        a, b = c[:, k], c[:, (k + 1) % 3]
        np.add.at(Mh, (a, b), alpha)
        np.add.at(Mh, (b, a), alpha)
    Mh[np.arange(V), np.arange(V)] = Mh.sum(axis=1)
    # Mv from the level heights
    z = (np.arange(layers + 1) / layers) ** 1.5
    h = np.abs(np.diff(z))
    Mv = np.zeros((layers + 1, layers + 1))
    for l in range(layers):
        Mv[l:l + 2, l:l + 2] += h[l] * np.array([[2.0, 1.0], [1.0, 2.0]])
    F = f.reshape(V, layers + 1)  # vertex columns are contiguous (Algorithm 1)
    got = (Mh @ F @ Mv.T).reshape(-1)
    assert np.all(np.abs(got - ref) <= 1e-12 * absr + 1e-300)


def test_mass_action_symmetric_and_bounded():
    layers = 6
    m = meshgen.tri_mesh(6, seed=12, order="random")
    sp, csp, X = _mesh_space(m, layers, P1)
    x = meshgen.uniform_field(sp.ndofs, 1)
    y = meshgen.uniform_field(sp.ndofs, 2)
    ax = np.zeros(sp.ndofs)
    Mx = _mass(m.cells, layers, csp, X, sp, x, ax)
    My = _mass(m.cells, layers, csp, X, sp, y)
    assert abs(y @ Mx - x @ My) < 1e-14 * (np.abs(y) @ ax)
    assert np.all(np.abs(Mx) <= ax * (1 + 1e-14))


# ----------------------------------------------------------------------------- copy / interpolation
def test_dg0_copy_exact():
    layers = 9
    m = meshgen.tri_mesh(6, seed=5, order="random")
    sp = O.number(m.cells, m.nverts, layers, O.DELTA["DG0xDG0"])
    a = meshgen.uniform_field(sp.ndofs, 3)
    out = np.full(sp.ndofs, np.nan)
    O.par_loop(O.K_COPY, m.cells, layers, [(sp, a, 1, O.READ), (sp, out, 1, O.WRITE)])
    np.testing.assert_array_equal(out, a)


def test_dg1_interpolation_is_nodal_gather():
    """DG1xDG1 DoF (c, l, 2a+b) holds the P1xP1 value at vertex a, level l+b."""
    layers = 5
    m = meshgen.tri_mesh(5, seed=6, order="random")
    p1 = O.number(m.cells, m.nverts, layers, P1, keep_tables=True)
    dg = O.number(m.cells, m.nverts, layers, O.DELTA["DG1xDG1"], keep_tables=True)
    x = meshgen.uniform_field(p1.ndofs, 4)
    out = np.full(dg.ndofs, np.nan)
    O.par_loop(O.K_INTERP, m.cells, layers, [(p1, x, 1, O.READ), (dg, out, 1, O.WRITE)])
    vdof = p1.first[0]   # (V, layers+1)
    cdof = dg.first[5]   # (C, layers): first DoF of cell c's layer-l entity
    for a in range(3):
        for b in range(2):
            got = out[cdof + 2 * a + b]
            want = x[vdof[m.cells[:, a]][:, b:b + layers]]
            np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------------------------- Gauss rules
@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_legendre_matches_library(n):
    x, w = O.gauss_legendre(n)
    t, v = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (t + 1), rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, 0.5 * v, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_gauss_legendre_high_precision(n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    P = lambda z: mp.legendre(n, z)
    roots = sorted(mp.polyroots(mp.taylor(P, 0, n)[::-1], maxsteps=200, extraprec=200))
    x, w = O.gauss_legendre(n)
    for i, r in enumerate(roots):
        assert abs(float((r + 1) / 2) - x[i]) <= 2.3e-16
        wr = 1 / ((1 - r ** 2) * mp.diff(P, r) ** 2)
        assert abs(float(wr) - w[i]) <= 1.2e-16


# ----------------------------------------------------------------------------- u^2 v
def _u2v(kind, m, layers, sp, csp, X, u, w=None, acc=O.INC):
    F = np.zeros(sp.ndofs)
    if w is None:
        O.par_loop(O.K_U2V, m.cells if hasattr(m, "cells") else m, layers,
                   [(csp, X, 3, O.READ), (sp, u, 1, O.READ), (sp, F, 1, acc)])
    else:
        O.par_loop(O.K_U2V_ADJ, m.cells if hasattr(m, "cells") else m, layers,
                   [(csp, X, 3, O.READ), (sp, u, 1, O.READ), (sp, w, 1, O.READ), (sp, F, 1, acc)])
    return F


SPACES = [("prism", 3, P1, O.INC), ("Q2", 4, O.DELTA["Q2xP2"], O.INC), ("DG2", 4, O.DELTA["DG2hex"], O.WRITE)]


@pytest.mark.parametrize("name,kind,delta,acc", SPACES)
def test_u2v_of_one_is_volume(name, kind, delta, acc):
    layers = 3
    m = meshgen.tri_mesh(4, seed=7) if kind == 3 else meshgen.quad_mesh(4, seed=7)
    sp, csp, X = _mesh_space(m, layers, delta)
    F = _u2v(kind, m, layers, sp, csp, X, np.ones(sp.ndofs), acc=acc)
    assert abs(F.sum() - 1.0) < 1e-13
    F2 = _u2v(kind, m, layers, sp, csp, X, np.full(sp.ndofs, -3.0), acc=acc)
    np.testing.assert_allclose(F2, 9.0 * F, rtol=1e-14)


@pytest.mark.parametrize("name,kind,delta,acc", SPACES)
def test_u2v_euler_identity_and_fd(name, kind, delta, acc):
    """F is homogeneous of degree 2: (dF/du)^T w . u = 2 w . F(u); and the
    adjoint is the transpose of the derivative (central differences are exact
    for a quadratic up to rounding)."""
    layers = 3
    m = meshgen.tri_mesh(4, seed=8, order="random") if kind == 3 else meshgen.quad_mesh(3, seed=8, order="random")
    sp, csp, X = _mesh_space(m, layers, delta)
    u = meshgen.uniform_field(sp.ndofs, 10)
    w = meshgen.uniform_field(sp.ndofs, 11)
    d = meshgen.uniform_field(sp.ndofs, 12)
    F = _u2v(kind, m, layers, sp, csp, X, u, acc=acc)
    g = _u2v(kind, m, layers, sp, csp, X, u, w=w, acc=acc)
    lhs, rhs = g @ u, 2.0 * (w @ F)
    assert abs(lhs - rhs) < 1e-13 * (np.abs(g) @ np.abs(u) + 1e-300)
    eps = 1e-6
    Fp = _u2v(kind, m, layers, sp, csp, X, u + eps * d, acc=acc)
    Fm = _u2v(kind, m, layers, sp, csp, X, u - eps * d, acc=acc)
    jd = (Fp - Fm) / (2 * eps)
    assert abs(w @ jd - g @ d) < 1e-8 * (np.abs(w) @ np.abs(jd))


def _lagrange_integrals(power):
    """int_0^1 t^power l_k(t) dt for the P2 Lagrange basis on nodes (0, 1, 1/2),
    by exact rational polynomial integration."""
    nodes = [Fraction(0), Fraction(1), Fraction(1, 2)]
    out = []
    for k in range(3):
        coeffs = [Fraction(1)]  # polynomial, ascending powers
        for m_ in range(3):
            if m_ == k:
                continue
            den = nodes[k] - nodes[m_]
            new = [Fraction(0)] * (len(coeffs) + 1)
            for i, c in enumerate(coeffs):
                new[i + 1] += c / den
                new[i] -= c * nodes[m_] / den
            coeffs = new
        out.append(sum(c / (i + power + 1) for i, c in enumerate(coeffs)))
    return out


IX = [0, 1, 1, 0, 2, 1, 2, 0, 2]
IY = [0, 0, 1, 1, 0, 2, 1, 2, 2]


@pytest.mark.parametrize("delta", [O.DELTA["Q2xP2"], O.DELTA["DG2hex"]])
@pytest.mark.parametrize("upow", [0, 1])
def test_unit_hex_closed_form(delta, upow):
    """One unit-cube hexahedron: with u = x^upow, F_{3e+v} = int x^{2 upow}
    l_ix(x) dx * int l_iy(y) dy * int l_v(z) dz (exact 1-D integrals)."""
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    sp = O.number(cells, 4, 1, delta)
    csp, X = O.coords(cells, xy, 1)
    node = [0.0, 1.0, 0.5]
    u = np.zeros(sp.ndofs)
    for i in range(27):
        e, v = divmod(i, 3)
        u[sp.map[0, i]] = node[IX[e]] ** upow
    F = _u2v(4, cells, 1, sp, csp, X, u, acc=O.INC)
    I0 = _lagrange_integrals(0)
    Ix = _lagrange_integrals(2 * upow)
    for i in range(27):
        e, v = divmod(i, 3)
        want = float(Ix[IX[e]] * I0[IY[e]] * I0[v])
        assert abs(F[sp.map[0, i]] - want) < 1e-15, (i, F[sp.map[0, i]], want)


def test_hex_rule_is_exact():
    """On straight-sided hexahedra the integrand u^2 v detJ has degree <= 7 per
    direction, so the 4-point and 6-point Gauss rules agree to rounding."""
    layers = 2
    m = meshgen.quad_mesh(3, seed=13, order="random")
    sp, csp, X = _mesh_space(m, layers, O.DELTA["Q2xP2"])
    u = meshgen.uniform_field(sp.ndofs, 14)
    w = meshgen.uniform_field(sp.ndofs, 15)
    try:
        F4 = _u2v(4, m, layers, sp, csp, X, u)
        g4 = _u2v(4, m, layers, sp, csp, X, u, w=w)
        O.set_hex_rule(6)
        F6 = _u2v(4, m, layers, sp, csp, X, u)
        g6 = _u2v(4, m, layers, sp, csp, X, u, w=w)
        O.set_hex_rule(3)
        F3 = _u2v(4, m, layers, sp, csp, X, u)
    finally:
        O.set_hex_rule(4)
    np.testing.assert_allclose(F4, F6, rtol=0, atol=1e-14 * np.abs(F4).max())
    np.testing.assert_allclose(g4, g6, rtol=0, atol=1e-14 * np.abs(g4).max())
    assert np.abs(F3 - F4).max() > 1e-8 * np.abs(F4).max()  # 3 points are not enough


def test_prism_u2v_vertical_closed_form():
    """One straight prism on the reference triangle, u = z: the integrand is
    linear horizontally and cubic vertically, so the 6-point rule is exact:
    F_{2a+b} = (A/3) * int_0^1 z^2 psi_b(z) dz with psi = (1-z, z)."""
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    xy = np.array([[0, 0], [1, 0], [0, 1]], dtype=np.float64)
    sp = O.number(cells, 3, 1, P1)
    csp, X = O.coords(cells, xy, 1)
    u = np.zeros(sp.ndofs)
    for a in range(3):
        u[sp.map[0, 2 * a + 1]] = 1.0
    F = _u2v(3, cells, 1, sp, csp, X, u)
    A = 0.5
    for a in range(3):
        assert abs(F[sp.map[0, 2 * a]] - A / 3 / 12) < 1e-16
        assert abs(F[sp.map[0, 2 * a + 1]] - A / 3 / 4) < 1e-16


def test_dg2_single_cell_equals_q2():
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    xy = np.array([[0.05, 0.0], [1.0, 0.1], [0.9, 1.1], [0.0, 0.8]], dtype=np.float64)
    layers = 2
    q2 = O.number(cells, 4, layers, O.DELTA["Q2xP2"])
    dg = O.number(cells, 4, layers, O.DELTA["DG2hex"])
    csp, X = O.coords(cells, xy, layers)
    rng = np.random.default_rng(0)
    uq = rng.uniform(-1, 1, q2.ndofs)
    # DG2 copy of the continuous field, layer by layer
    ud = np.zeros(dg.ndofs)
    for l in range(layers):
        ud[dg.map[0] + l * dg.offset] = uq[q2.map[0] + l * q2.offset]
    Fq = _u2v(4, cells, layers, q2, csp, X, uq)
    Fd = _u2v(4, cells, layers, dg, csp, X, ud, acc=O.WRITE)
    # summing the DG2 layer contributions onto the continuous numbering gives Fq
    acc = np.zeros(q2.ndofs)
    for l in range(layers):
        np.add.at(acc, q2.map[0] + l * q2.offset, Fd[dg.map[0] + l * dg.offset])
    np.testing.assert_allclose(acc, Fq, rtol=1e-14, atol=1e-17)


# ----------------------------------------------------------------------------- the nine prism spaces
def _tp_local_nodes(h, v):
    """(horizontal node, vertical node) of every stencil slot, read off the
    stencil rule: entities vertices, edges, cell; per entity bottom, top,
    vertical DoFs; horizontal index major.  Horizontal node: vertex a or 'c'
    (cell constant); vertical node: 0 (z=0), 1 (z=h) or 'i' (constant)."""
    dh = {O.CG1: (1, 0, 0), O.DG0: (0, 0, 1), O.DG1: (0, 0, 3)}[h]
    dv0 = 1 if v == O.CG1 else 0
    dv1 = {O.CG1: 0, O.DG0: 1, O.DG1: 2}[v]
    out = []
    for d, ents in ((0, 3), (1, 3), (2, 1)):
        for e in range(ents):
            for part, nv in ((0, dv0), (1, dv0), (2, dv1)):
                for j in range(dh[d]):
                    for beta in range(nv):
                        hn = "c" if h == O.DG0 else (e if d == 0 else j)
                        vn = part if part < 2 else ("i" if v == O.DG0 else beta)
                        out.append((hn, vn))
    return out


@pytest.mark.parametrize("name,h,v", O.TP_PAIRS)
def test_tp_element_matrix_closed_form(name, h, v):
    """Straight prism: M = Mh (x) Mv with Mh = A/12 (1 + [a=a']) (CG1, DG1) or A
    (DG0) and Mv = hz/6 (1 + [b=b']) (CG1, DG1) or hz (DG0)."""
    tri = [(0.1, 0.2), (0.9, 0.35), (0.3, 0.8)]
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    xy = np.array(tri)
    L = 2
    sp = O.number(cells, 3, L, O.DELTA[name])
    csp, X = O.coords(cells, xy, L)
    O.set_tp_element(h, v)
    p = np.array(tri)
    A = 0.5 * abs((p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1]))
    hz = 1.0 / L
    nodes = _tp_local_nodes(h, v)
    assert len(nodes) == sp.k
    # assemble column by column on layer 0 only (a one-layer slice of the stencil)
    M = np.zeros((sp.k, sp.k))
    for j in range(sp.k):
        e = np.zeros(sp.ndofs)
        e[sp.map[0, j]] = 1.0
        b = np.zeros(sp.ndofs)
        O.par_loop(O.K_MASS_TP, cells, 1, [(csp, X, 3, O.READ), (sp, e, 1, O.READ), (sp, b, 1, O.INC)])
        M[:, j] = b[sp.map[0]]
    want = np.zeros_like(M)
    for i, (ha, va) in enumerate(nodes):
        for j, (hb, vb) in enumerate(nodes):
            mh = A if ha == "c" else A / 12 * (1 + (ha == hb))
            mv = hz if va == "i" else hz / 6 * (1 + (va == vb))
            want[i, j] = mh * mv
    np.testing.assert_allclose(M, want, rtol=1e-13, atol=1e-18)


@pytest.mark.parametrize("name,h,v", O.TP_PAIRS)
def test_tp_volume_and_symmetry(name, h, v):
    layers = 3
    m = meshgen.tri_mesh(5, seed=31, order="random")
    sp = O.number(m.cells, m.nverts, layers, O.DELTA[name])
    csp, X = O.coords(m.cells, m.xy, layers)
    O.set_tp_element(h, v)

    def apply(f):
        b = np.zeros(sp.ndofs)
        O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC)])
        return b
    assert abs(apply(np.ones(sp.ndofs)).sum() - 1.0) < 1e-14
    x = meshgen.uniform_field(sp.ndofs, 32)
    y = meshgen.uniform_field(sp.ndofs, 33)
    assert abs(y @ apply(x) - x @ apply(y)) < 1e-14 * (np.abs(x).sum() + np.abs(y).sum()) / sp.ndofs


def test_tp_cg1xcg1_equals_p1_kernel():
    layers = 4
    m = meshgen.tri_mesh(6, seed=34)
    sp, csp, X = _mesh_space(m, layers, P1)
    f = meshgen.uniform_field(sp.ndofs, 35)
    O.set_tp_element(O.CG1, O.CG1)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC)])
    np.testing.assert_allclose(b, _mass(m.cells, layers, csp, X, sp, f), rtol=1e-14, atol=1e-18)


def _perturbed_coords(m, layers, seed):
    csp, X = O.coords(m.cells, m.xy, layers)
    rng = np.random.default_rng(seed)
    return csp, X + 0.3 * rng.uniform(-1, 1, X.size) / (m.n * layers)


def test_tp_matches_p1_kernel_on_general_prisms():
    """On non-straight prisms the element matrix depends on which basis function
    sits at which vertex, so the tensor-product kernel must reproduce the
    P1xP1 kernel exactly there as well."""
    layers = 3
    m = meshgen.tri_mesh(5, seed=36, order="random")
    sp = O.number(m.cells, m.nverts, layers, P1)
    csp, X = _perturbed_coords(m, layers, 37)
    f = meshgen.uniform_field(sp.ndofs, 38)
    O.set_tp_element(O.CG1, O.CG1)
    b = np.zeros(sp.ndofs)
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (sp, f, 1, O.READ), (sp, b, 1, O.INC)])
    np.testing.assert_allclose(b, _mass(m.cells, layers, csp, X, sp, f), rtol=1e-14, atol=1e-18)


@pytest.mark.parametrize("dgname,h,v", [("DG1xDG1", O.DG1, O.DG1), ("DG1xCG1", O.DG1, O.CG1),
                                        ("CG1xDG1", O.CG1, O.DG1)])
def test_tp_broken_space_assembles_to_continuous(dgname, h, v):
    """Restrict a continuous P1xP1 field to a broken space (same nodes), apply
    the broken mass operator, sum every broken DoF back onto the continuous
    DoF at the same node: the result is the continuous mass action.  Holds on
    general prisms only if the broken space's nodes sit where the stencil rule
    puts them."""
    layers = 3
    m = meshgen.tri_mesh(4, seed=39, order="random")
    cg = O.number(m.cells, m.nverts, layers, P1)
    br = O.number(m.cells, m.nverts, layers, O.DELTA[dgname])
    csp, X = _perturbed_coords(m, layers, 40)
    f = meshgen.uniform_field(cg.ndofs, 41)
    nodes = _tp_local_nodes(h, v)           # broken slot -> (vertex a, level 0/1)
    slot_cg = [2 * a + b for a, b in nodes]  # the continuous slot at that node
    fb = np.zeros(br.ndofs)
    for l in range(layers):
        fb[br.map[:, :] + l * br.offset[None, :]] = f[cg.map[:, slot_cg] + l * cg.offset[None, slot_cg]]
    O.set_tp_element(h, v)
    bb = np.zeros(br.ndofs)
    O.par_loop(O.K_MASS_TP, m.cells, layers, [(csp, X, 3, O.READ), (br, fb, 1, O.READ), (br, bb, 1, O.INC)])
    # every broken DoF once, onto the continuous DoF at its node
    cg_of = np.full(br.ndofs, -1, dtype=np.int64)
    for l in range(layers):
        cg_of[br.map + l * br.offset[None, :]] = cg.map[:, slot_cg] + l * cg.offset[None, slot_cg]
    assert np.all(cg_of >= 0)
    back = np.zeros(cg.ndofs)
    np.add.at(back, cg_of, bb)
    np.testing.assert_allclose(back, _mass(m.cells, layers, csp, X, cg, f), rtol=1e-13, atol=1e-17)
