"""The benchmark's bookkeeping, checked without a GPU: which form the library
runs for a launch (and so how many kernels it starts, the `gpu_launches`
claim), and the FP64 operation counts the roofline fractions divide by.

The form rules restate the launchers' dispatch (P1xP1: single pass below a
million (column, level) items, factored or unfactored cell pass below 32
layers, the probe's gather modes from 32; nine spaces: the optimistic DG x DG
and DG x CG1 forms from 8 layers with WRITE and the straightness flags, the
CG1 x DG gather from 32 layers with WRITE), and the operation counts are
checked against sums written out per entity for a small mesh."""
import pytest

import bench
import meshgen


@pytest.fixture(autouse=True)
def clean_env(monkeypatch):
    for k in ("EXTMESH_TP_FLAGS", "EXTMESH_TP_OPTIMISTIC", "EXTMESH_TP_CGDG"):
        monkeypatch.delenv(k, raising=False)


def test_p1_form_rules():
    assert bench.p1_form(999_999, 100) == "single"
    assert bench.p1_form(10_000_000, 1) == "plain"
    assert bench.p1_form(10_000_000, 2) == "plain"
    assert bench.p1_form(10_000_000, 3) == "factored"
    assert bench.p1_form(10_000_000, 31) == "factored"
    assert bench.p1_form(10_000_000, 32) == "gather"
    assert bench.p1_form(10_000_000, 100, geometry="terrain") == "gather-sigma"
    assert bench.p1_form(10_000_000, 100, geometry="wavy") == "cells"
    assert bench.p1_form(10_000_000, 100, var=True) == "var"


def test_p1_kernel_counts_by_access():
    # the gather modes launch 9 kernels with WRITE (optimistic pass + fix-up)
    # and with INC (the split form's two vertex passes and the gather)
    assert bench.p1_kernels(100_000_000, 100) == 9
    assert bench.p1_kernels(100_000_000, 100, write=False) == 9
    assert bench.p1_kernels(500_000, 100) == 1
    assert bench.p1_kernels(100_000_000, 10) == 4


def test_nine_space_kernel_counts():
    big = 15_000_000
    # DG x DG and DG x CG1 with WRITE from 8 layers: area pass, optimistic pass, fix-up
    assert bench.tp_kernels(big, 100, "DG0xDG0", write=True) == 3
    assert bench.tp_kernels(big, 100, "DG0xCG1", write=True) == 3
    assert bench.tp_kernels(big, 7, "DG0xCG1", write=True) == 3  # flags, levels, cell kernel
    # CG1 x DG with WRITE from 32 layers: the gather path
    assert bench.tp_kernels(big, 32, "CG1xDG1", write=True) == 9
    assert bench.tp_kernels(big, 31, "CG1xDG1", write=True) == 3
    # INC keeps the flagged cell kernel; small launches run the cell kernel alone
    assert bench.tp_kernels(big, 100, "CG1xDG0", write=False) == 3
    assert bench.tp_kernels(1000, 100, "DG1xCG1", write=True) == 1


def test_switches_turn_the_forms_off(monkeypatch):
    big = 15_000_000
    monkeypatch.setenv("EXTMESH_TP_OPTIMISTIC", "0")
    assert not bench.dgcg_optimistic("DG1xCG1", 100, big)
    assert bench.tp_kernels(big, 100, "DG1xCG1", write=True) == 3
    monkeypatch.setenv("EXTMESH_TP_CGDG", "0")
    assert not bench.cgdg_gather("CG1xDG0", 100)
    monkeypatch.setenv("EXTMESH_TP_FLAGS", "0")
    assert bench.tp_kernels(big, 100, "DG0xDG0", write=True) == 1


def test_dgcg_window():
    big = 15_000_000
    assert bench.dgcg_optimistic("DG0xCG1", 8, big)
    assert bench.dgcg_optimistic("DG0xCG1", 1024, big)
    assert not bench.dgcg_optimistic("DG0xCG1", 7, big)
    assert not bench.dgcg_optimistic("DG0xCG1", 1025, big)
    assert not bench.dgcg_optimistic("DG0xCG1", 100, 999_999)  # below a million items the flags do not run
    assert not bench.dgcg_optimistic("DG0xDG1", 100, big)


def test_cgdg_ops_against_entity_sums():
    m = meshgen.tri_mesh(6, seed=5)
    V, C = m.nverts, m.ncells
    E = bench.base_edges(m.cells)
    assert E == bench.euler_edges(V, C)
    # vertex rows: every vertex has itself plus its neighbours
    nbr = [set() for _ in range(V)]
    for c in m.cells:
        for a in c:
            for b in c:
                if a != b:
                    nbr[a].add(int(b))
    entries = sum(1 + len(s) for s in nbr)
    assert entries == V + 2 * E
    L = 40
    for nv in (1, 2):
        want = entries * nv * L + 2 * V * nv * L + 7 * C + 4 * E
        assert bench.cgdg_ops(V, E, C, L, nv) == want


def test_p1_gather_ops_and_bytes():
    m = meshgen.tri_mesh(6, seed=6)
    V, C = m.nverts, m.ncells
    E = bench.base_edges(m.cells)
    L = 50
    n = V * (L + 1)
    assert bench.p1_ops_form("gather", n, C * (L + 1), C, L, E) == 3 * n + (V + 2 * E) * (L + 1) + 7 * C + 4 * E
    assert bench.p1_bytes_8d(V, C, L) == 24 * n + 16 * n + 24 * C


def test_dgcg_item_ops_are_the_closed_form_counts():
    # DG0: three FMA for the column matrix and one product; DG1: three nodes of
    # three FMA, two sums, the scaled sum and three FMA
    assert bench.DGCG_ITEM_OPS == {"DG0xCG1": 3 + 1, "DG1xCG1": 3 * 3 + 2 + 1 + 3}
