"""The oracle's pins must be strong enough that a plausible mistake anywhere
in it fails at least one of them.  Each case plants one mistake in a copy of
oracle.c (on the CPU), builds it, and runs the numbering and kernel pins
against it in a subprocess; the run must fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # Algorithm 1
    "top_copy_not_numbered": ("for (int64_t s = s_lo; s <= s_hi; ++s) {", "for (int64_t s = s_lo; s < s_hi; ++s) {"),
    "bottom_copy_not_numbered": ("const int64_t s_lo = 2 * (int64_t)(lo ? lo[g] : 0),",
                                 "const int64_t s_lo = 2 * (int64_t)(lo ? lo[g] : 0) + 1,"),
    "vertical_counted_as_horizontal": ("next += dent ? dent[2 * g + d2] : delta[t];",
                                       "next += dent ? dent[2 * g + d2] : delta[2 * d1];"),
    "number_taken_after_counting": ("if (first[t]) first[t][i * (maxlevel + 1 - d2) + level] = next;",
                                    "if (first[t]) first[t][i * (maxlevel + 1 - d2) + level] = next + (d2 ? 0 : delta[t]);"),
    # explicit lists and Algorithm 2
    "top_slot_reads_bottom": ("first[2 * d][id * (layers + 1) + 1] + q", "first[2 * d][id * (layers + 1) + 0] + q"),
    "offset_from_same_layer": ("list_at_layer(nvc, 2, delta, first, 1, l1);", "list_at_layer(nvc, 2, delta, first, 0, l1);"),
    "edge_wrong_neighbour": ("cell_verts[c * nvc + (k + 1) % nvc]", "cell_verts[c * nvc + (k + nvc - 1) % nvc]"),
    # quadrature and elements
    "prism_weight": ("wts[q] = (1.0 / 6.0) * gw[g];", "wts[q] = (1.0 / 3.0) * gw[g];"),
    "triangle_point": ("{2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}", "{2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 6.0}"),
    "det_sign_term": ("J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -",
                      "J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) +"),
    "no_abs_detJ": ("return fabs(det3(J));", "return det3(J);"),
    "jacobian_transposed": ("J[r][s] += X[3 * i + r] * grad[i][s];", "J[s][r] += X[3 * i + r] * grad[i][s] * (r == 2 ? 2.0 : 1.0);"),
    "p2_node_order": ("const double nodes[3] = {0.0, 1.0, 0.5};", "const double nodes[3] = {0.0, 0.5, 1.0};"),
    "q2_edge_table": ("static const int q2_ix[9] = {0, 1, 1, 0, 2, 1, 2, 0, 2};",
                      "static const int q2_ix[9] = {0, 1, 1, 0, 1, 2, 2, 0, 2};"),
    "gauss_weight": ("w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);",
                     "w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp);"),
    "u2v_linear": ("out[2][i] += T->w[q] * dj * uq * uq * T->phi[q][i];",
                   "out[2][i] += T->w[q] * dj * uq * T->phi[q][i];"),
    "adjoint_factor": ("out[3][j] += T->w[q] * dj * 2.0 * uq * wq * T->phi[q][j];",
                       "out[3][j] += T->w[q] * dj * uq * wq * T->phi[q][j];"),
    "adjoint_uses_u_twice": ("out[3][j] += T->w[q] * dj * 2.0 * uq * wq * T->phi[q][j];",
                             "out[3][j] += T->w[q] * dj * 2.0 * uq * uq * T->phi[q][j];"),
    "extrude_level": ("(double)(s + l + b) / (double)layers;", "(double)(s + l) / (double)layers;"),
    "interp_node_swap": ("out[1][2 * a + b] = v;", "out[1][2 * a + (1 - b)] = v;"),
    "tp_dg0_vertical_not_constant": ("else vf = (v == ORC_DG0) ? 2 : beta;", "else vf = (v == ORC_DG0) ? 0 : beta;"),
    "tp_cg1_vertex_shift": ("else if (d == 0) hf = e;  /* CG1 vertex */", "else if (d == 0) hf = (e + 1) % 3;"),
    "tp_bottom_top_same": ("            if (part == 0) vf = 0;", "            if (part == 0) vf = 1;"),
    "mass_wrong_basis": ("out[2][i] += wts[q] * dj * fq * phi[i];", "out[2][i] += wts[q] * dj * fq * phi[(i + 2) % 6];"),
    # variable layers per column
    "var_hull_max_bottom": ("if (lo[id] < 0 || bottom < lo[id]) lo[id] = bottom;",
                            "if (lo[id] < 0 || bottom > lo[id]) lo[id] = bottom;"),
    "var_column_stops_a_layer_early": ("s_hi = 2 * (int64_t)(hi ? hi[g] : maxlevel);",
                                       "s_hi = 2 * (int64_t)(hi ? hi[g] - 1 : maxlevel);"),
    "var_list_at_level_0": ("map[c * k + j++] = (int32_t)(first[2 * d + 1][id * maxlevel + s] + q);",
                            "map[c * k + j++] = (int32_t)(first[2 * d + 1][id * maxlevel + 0] + q);"),
    "var_uniform_trip_count": ("const int32_t lam = cell_layers ? cell_layers[c] : layers;",
                               "const int32_t lam = layers;"),
    "extrude_ignores_first": ("(double)(s + l + b) / (double)layers;", "(double)(l + b) / (double)layers;"),
    # horizontal facets
    "facet_loop_skips_top": ("if (kernel == ORC_K_HFACET_MASS) l1 = lam + 1;", "if (kernel == ORC_K_HFACET_MASS) l1 = lam;"),
    "facet_offset_horizontal_only": ("offset[i] = (int32_t)(first[2 * d][e * 3 + 1] - first[2 * d][e * 3 + 0]);",
                                     "offset[i] = (int32_t)(first[2 * d][e * 3 + 1] - first[2 * d][e * 3 + 0] - delta[2 * d + 1]);"),
    "facet_normal_sign": ("const double n1 = e1[2] * e2[0] - e1[0] * e2[2];",
                          "const double n1 = e1[2] * e2[0] + e1[0] * e2[2];"),
    "facet_weight": ("static const double tri_w = 1.0 / 6.0;", "static const double tri_w = 1.0 / 3.0;"),
    "facet_dg1_wrong_node": ("phi[j] = (g_tp_h == ORC_DG0) ? 1.0 : tri_lam(j, tri_pts[q][0], tri_pts[q][1]);",
                              "phi[j] = (g_tp_h == ORC_DG0) ? 1.0 : tri_lam(j % 2, tri_pts[q][0], tri_pts[q][1]);"),
    "jump_sign": ("jump += u[j] * pb[j] - u[k + j] * pa[j];", "jump += u[j] * pb[j] + u[k + j] * pa[j];"),
    "jump_trace_of_bottom": ("pb[j] = tp_phi(hfun[j], vfun[j], tri_pts[q][0], tri_pts[q][1], 1.0, g);",
                             "pb[j] = tp_phi(hfun[j], vfun[j], tri_pts[q][0], tri_pts[q][1], 0.0, g);"),
    "jump_above_added": ("out[2][k + i] -= tri_w * ds * jump * pa[i];", "out[2][k + i] += tri_w * ds * jump * pa[i];"),
    "jump_same_cell_twice": ("+ (j >= kc[a] ? offs[a][j] : 0);", "+ 0;"),
    "jump_base_face": ("const double ds = tri_area_element(X + 3, 6);", "const double ds = tri_area_element(X, 6);"),
    # per-entity DoF counts and the p-adaptive DG kernel
    "ragged_counts_swapped": ("next += dent ? dent[2 * g + d2] : delta[t];",
                              "next += dent ? dent[2 * g + 1 - d2] : delta[t];"),
    "ragged_offset_horizontal_only": ("            offset[j] = a + b;", "            offset[j] = a;"),
    "ragged_top_list_at_bottom": ("else if (part == 1) map[j] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s + 1] + q);",
                                  "else if (part == 1) map[j] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s] + q);"),
    "dgp_two_dofs_as_dg0": ("else if (k == 2) { h = ORC_DG0; v = ORC_DG1; }", "else if (k == 2) { h = ORC_DG0; v = ORC_DG0; }"),
}


def _run_pins(source: str, tmp_path):
    c = tmp_path / "oracle_mut.c"
    c.write_text(source)
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_numbering.py"),
                        os.path.join(ROOT, "tests", "test_oracle_kernels.py"),
                        os.path.join(ROOT, "tests", "test_oracle_var.py"),
                        os.path.join(ROOT, "tests", "test_oracle_facets.py"),
                        os.path.join(ROOT, "tests", "test_oracle_ragged.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r


def test_unmutated_copy_passes(tmp_path):
    r = _run_pins(open(SRC).read(), tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    r = _run_pins(src.replace(old, new, 1), tmp_path)
    assert r.returncode != 0, f"planted mistake {name!r} passed every pin:\n{r.stdout[-2000:]}"
