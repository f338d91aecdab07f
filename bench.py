#!/usr/bin/env python3
"""Benchmark of the extruded-mesh par_loop on GB300: valuable HBM GB/s.

Default workload (one step = the three FP64 loops of the ~1M-triangle,
100-layer prism mesh, RCM-ordered): P1xP1 RHS assembly of int f v dx with
f = sin(x) cos(y) z, P1xP1 mass-matrix action y = M x with x ~ U(-1,1) (both
with WRITE access), and DG1xDG1 nodal interpolation of x (WRITE).  Valuable
bytes (each coordinate, input, output DoF and stencil-map entry moved once) /
device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 2|3|4|5|6|7|8] [--geometry flat|terrain|tilted]

--impl reference times the CPU oracle (all host cores) on a bounded sample of
the same workload (the reference arm: there is no reference GPU code).  Under torchrun
every rank runs its own independent copy of the workload (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SMS = 152
FP64_OPS_PER_CLK_PER_SM = 2.0  # 1.25 TFLOP/s nominal = 2 FMA/clk/SM x 152 SMs x 2.07 GHz x 2 flops
SM_MAX_MHZ = 2070.0
P1_DELTA = (1, 0, 0, 0, 0, 0)
DG1_DELTA = (0, 0, 0, 0, 0, 6)
# FP64 work of one P1xP1 RHS / mass-action par_loop on straight prisms in the
# split form the library runs.  Constant layers, two or more (factored form):
#   alpha_c = |2A_c| / 144, A_a = sum of alpha_c around a   4 DADD, 2 DMUL, 1 DFMA per cell,
#   w = |h_lo| (f_lo + 2 f) + |h_hi| (2 f + f_hi),
#   b += A_a w                                             6 per DoF,
#   alpha_c (w_0 + w_1 + w_2) to the three vertices        3 per item,
# four kernels (areas, vertex pass, cell pass, and the pass over deferred
# non-straight warp steps, which finds none on a straight mesh).  One
# constant layer: w alone (5 per DoF) and
#   value_a = alpha (w_a + w_0 + w_1 + w_2)                6 per item,
# three kernels.  Variable layers: w and its two one-layer halves (6 per DoF)
# and the same 6 per item, three kernels.  The vertex and cell passes issue
# their products and sums as DFMA (a b + (-0), a (+-1) + b).  All send 3 FP64
# atomic adds per item to L2.  Evaluating each cell's element matrix by itself
# instead needs 18 FP64 operations per item.
# FP64 operations of one P1xP1 RHS / mass-action launch, per form (as the
# kernels issue them; products and sums all go to the DFMA pipe):
#   gather   3 per DoF (column mass matrix Mv) + 1 per vertex-row entry and
#            level (V + 2E entries: base mass matrix Mh) + the per-launch
#            geometry (7 per cell for the level-0 areas, 4 per edge for the
#            row weights); no atomics (the optimistic one-pass form issues the
#            Mh and Mv work of 32 DoFs for every 30 it writes: the two halo
#            lanes of each window are not counted);
#   gather-sigma (terrain-following levels) the same + 2 per DoF (the check
#            against the terrain-following model) + 14 per edge, 11 per cell
#            and 5 per vertex for the depth-weighted rows;
#   factored 6 per DoF + 3 per (column, level) item + 7 per cell, 3 L2 atomic
#            adds per item;
#   cells    42 per prism with vertical edges (closed form of the 6-point
#            rule), 132 per prism otherwise (general Jacobian), + 3 per item,
#            3 L2 atomic adds per item;
#   single   13 per item (below a million items).
P1_PRISM_OPS = {"vertical": 42, "general": 132}
# kernels of one launch: the gather modes' launch runs 9 (WRITE access: the
# optimistic one pass and its fix-up in place of the vertex passes of the
# split form that INC access runs; the one-pass checked form also 9)
P1_KERNELS = {"gather": 9, "gather-split": 9, "gather-sigma": 9, "cells": 9, "cells-forced": 1, "factored": 4,
              "plain": 3, "var": 3, "single": 1}
CELL_ATOMICS_PER_ITEM = 3
P1_SPLIT_MIN_ITEMS = 1_000_000
P1_FACTORED_MIN_LAYERS = 3
P1_GATHER_MIN_LAYERS = 32


def p1_form(items: int, layers: int, var: bool = False, geometry: str = "flat") -> str:
    """The form the library's default picks for a P1xP1 launch on a triangle
    mesh: the single pass below a million items, the variable-layer split form
    on variable layers, else the probe's choice (gather on a flat straight
    extrusion, the cell loop on any other geometry)."""
    if items < P1_SPLIT_MIN_ITEMS:
        return "single"
    if var:
        return "var"
    if layers < P1_GATHER_MIN_LAYERS:
        return "factored" if layers >= P1_FACTORED_MIN_LAYERS else "plain"
    return {"flat": "gather", "terrain": "gather-sigma"}.get(geometry, "cells")


def p1_ops_form(form: str, ndofs: int, items: int, ncells: int, layers: int, nedges: int,
                geometry: str = "flat") -> int:
    nv = ndofs // (layers + 1)
    if form == "gather":
        return 3 * ndofs + (nv + 2 * nedges) * (layers + 1) + 7 * ncells + 4 * nedges
    if form == "gather-sigma":
        return 5 * ndofs + (nv + 2 * nedges) * (layers + 1) + 18 * ncells + 14 * nedges + 5 * nv
    if form == "factored":
        return 6 * ndofs + 3 * items + 7 * ncells
    if form in ("cells", "cells-forced"):
        per = P1_PRISM_OPS["general" if geometry == "tilted" else "vertical"]
        return per * ncells * layers + 3 * items
    if form == "var":
        return 6 * ndofs + 6 * items
    if form == "plain":
        return 5 * ndofs + 6 * items
    return 13 * items


def p1_bytes_8d(nverts: int, ncells: int, layers: int) -> int:
    """Algorithmic bytes of one P1xP1 RHS / mass-action launch: coordinates
    (24 per vertex level), input and output (8 + 8), one int32 map row of 6
    entries per base cell, each moved once."""
    return 40 * nverts * (layers + 1) + 24 * ncells


def euler_edges(nverts: int, ncells: int) -> int:
    """Edges of a triangulated disc (Euler: V - E + F = 1), as the unit-square
    meshes here are."""
    return nverts + ncells - 1


def p1_ops(ndofs: int, items: int, ncells: int, layers: int, var: bool = False, nedges: int | None = None,
           geometry: str = "flat") -> int:
    """FP64 operations of the default form (nedges: Euler's formula unless given)."""
    nv = ndofs // (layers + 1)
    ne = euler_edges(nv, ncells) if nedges is None else nedges
    return p1_ops_form(p1_form(items, layers, var, geometry), ndofs, items, ncells, layers, ne, geometry)


P1_OPS_NOTE = ("default form from a million (column, level) items: gather on a flat straight extrusion "
               "(3 per DoF + 1 per vertex-row entry and level + 7 per cell + 4 per edge), cell loop otherwise "
               "(42 per prism with vertical edges + 3 per item); single pass below: 13 per item")


def cgdg_gather(name: str, layers: int, write: bool = True) -> bool:
    """CG1 x DG0 / CG1 x DG1 with WRITE from 32 layers run the gather path of
    the P1xP1 launch (EXTMESH_TP_CGDG=0 keeps the cell kernel)."""
    return (write and name in ("CG1xDG0", "CG1xDG1") and layers >= P1_GATHER_MIN_LAYERS
            and os.environ.get("EXTMESH_TP_CGDG", "") != "0")


# FP64 operations per (column, level) item of the optimistic DG x CG1 form
# (the DoFs of a level formed once from three levels of f: 3 per node for the
# column matrix, 1 product (DG0) or the node sum and its product, 6 (DG1))
DGCG_ITEM_OPS = {"DG0xCG1": 4, "DG1xCG1": 15}


def dgcg_optimistic(name: str, layers: int, items: int, write: bool = True) -> bool:
    """DG0 x CG1 / DG1 x CG1 with WRITE from 8 to 1,024 layers run the
    optimistic level form when the flags run (a million cell-layers or more,
    EXTMESH_TP_FLAGS and EXTMESH_TP_OPTIMISTIC not 0)."""
    env = os.environ.get("EXTMESH_TP_FLAGS", "")
    flagged = env == "1" or (env != "0" and items >= 1_000_000)
    return (write and flagged and name in DGCG_ITEM_OPS and 8 <= layers <= 1024
            and os.environ.get("EXTMESH_TP_OPTIMISTIC", "") != "0")


def cgdg_ops(nverts: int, nedges: int, ncells: int, layers: int, nv: int) -> int:
    """FP64 operations of the CG1 x DG gather path: one per vertex-row entry
    and DoF layer (V + 2E entries, nv DoFs per layer), two per DoF for the
    layer's DG mass, and the per-launch geometry (7 per cell, 4 per edge)."""
    return (nverts + 2 * nedges) * nv * layers + 2 * nverts * nv * layers + 7 * ncells + 4 * nedges


def tp_kernels(items: int, layers: int = 1, name: str = "", write: bool = False) -> int:
    """Kernels of one EXT_K_MASS_TP launch on constant layers over a mesh with
    base coordinates: the level table, the straightness flags and the cell
    kernel from a million (column, layer) items (EXTMESH_TP_FLAGS=1 / 0: at any
    size / never), the cell kernel alone otherwise; with WRITE on a DG x DG
    space from 8 to 2048 layers the optimistic form (the area pass, flags and
    element vectors in one launch, then the fix-up launch)."""
    if cgdg_gather(name, layers, write):
        return 9  # the gather path: levels, probe, sigma, rows, gather, fix-up, general, clear, cell kernel
    if dgcg_optimistic(name, layers, items, write):
        return 3  # areas and level tables, the optimistic pass, the fix-up
    env = os.environ.get("EXTMESH_TP_FLAGS", "")
    flagged = env == "1" or (env != "0" and items >= 1_000_000)
    dgdg = name[:2] == "DG" and name[4:6] == "DG"
    if flagged and write and dgdg and 8 <= layers <= 2048 and os.environ.get("EXTMESH_TP_OPTIMISTIC", "") != "0":
        return 3  # areas, the optimistic pass, the fix-up
    return 3 if flagged else 1


def base_edges(cells) -> int:
    """Distinct edges of a base triangulation (C x 3 vertex ids)."""
    c = np.asarray(cells, dtype=np.int64)
    e = np.concatenate([c[:, [0, 1]], c[:, [1, 2]], c[:, [2, 0]]])
    e.sort(axis=1)
    return int(np.unique(e[:, 0] * (int(c.max()) + 1) + e[:, 1]).size) if c.size else 0


def p1_kernels(items: int, layers: int, var: bool = False, geometry: str = "flat", write: bool = True) -> int:
    """Kernels of one launch in the default form (INC access: the gather
    forms launch the split flat pass instead of the optimistic pair)."""
    form = p1_form(items, layers, var, geometry)
    if not write and form in ("gather", "gather-sigma", "cells"):
        return P1_KERNELS["gather-split"]
    return P1_KERNELS[form]


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", float(p.get("sm_max_mhz", SM_MAX_MHZ))
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", SM_MAX_MHZ


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, local):
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's time (the job finishes when its last rank does)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank: float, ms_per_rank: float, world: int) -> float:
    """Whole-job GB/s under weak scaling: every rank moves bytes_per_rank; the
    job takes as long as the slowest rank."""
    return world * bytes_per_rank / (max_over_ranks(ms_per_rank, world) * 1e-3) / 1e9


# ----------------------------------------------------------------------------- workload (config 2)
N_CFG2, LAYERS_CFG2, SEED = 707, 100, 1604


def valuable_bytes_cfg2(V, C, L, maps=True):
    nP1 = V * (L + 1)
    k1 = 24 * nP1 + 8 * nP1 + 8 * nP1 + (2 * 24 * C if maps else 0)        # coords, f, b (+ coords/P1 maps)
    k5 = 8 * nP1 + 48 * C * L + (2 * 24 * C if maps else 0)                 # x, out (+ P1/DG1 maps)
    return {"rhs": k1, "mass": k1, "interp": k5, "total": 2 * k1 + k5}


def geometry_coords(m, L, geometry, dev):
    """Coordinate field of the benchmark mesh: the flat unit-height extrusion
    comes from EXT_K_EXTRUDE; terrain-following levels and leaning columns
    (meshgen.level_coords) are uploaded."""
    import torch
    return torch.from_numpy(meshgen.level_coords(m, L, seed=SEED + 20, kind=geometry).reshape(-1)).to(dev)


def time_p1_forms(E, gm, cs, p1, X, x, y, stream, forms, reps):
    """Mean device time (ms) of one mass-action launch (WRITE) in each form,
    forced with ext_set_option; reps back to back after one warm-up launch
    (inputs larger than L2)."""
    import torch
    old = E.ext_get_option(E.EXT_OPT_P1_FORM)
    out = {}
    args = [(cs.handle, X, E.EXT_READ), (p1.handle, x, E.EXT_READ), (p1.handle, y, E.EXT_WRITE)]
    try:
        for name in forms:
            E.ext_set_option(E.EXT_OPT_P1_FORM, E.P1_FORMS[name])
            E.ext_par_loop(gm.handle, E.EXT_K_MASS_P1P1, args, stream.cuda_stream)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                E.ext_par_loop(gm.handle, E.EXT_K_MASS_P1P1, args, stream.cuda_stream)
            b.record(stream)
            b.synchronize()
            E.ext_sync_check(stream.cuda_stream)
            out[name] = a.elapsed_time(b) / reps
    finally:
        E.ext_set_option(E.EXT_OPT_P1_FORM, old)
    return out


def form_entry(form, ms, V, C, L, E_, geometry, ops_peak, hbm, launches=None):
    ndofs, items = V * (L + 1), C * (L + 1)
    ops = p1_ops_form(form, ndofs, items, C, L, E_, geometry)
    nbytes = p1_bytes_8d(V, C, L)
    gops = ops / (ms * 1e-3) / 1e9
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"ms": round(ms, 4), "fp64_ops": ops, "fp64_gops": round(gops, 1),
            "fp64_frac": round(gops / ops_peak, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
            "l2_atomic_adds_per_item": 0 if form.startswith("gather") else CELL_ATOMICS_PER_ITEM,
            "kernels": P1_KERNELS[form] if launches is None else launches}


def run_ours(args, rank, world, local):
    import torch
    import paper_1604_05937_gb300 as E

    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    geometry = args.geometry
    m = meshgen.tri_mesh(args.n or N_CFG2, seed=SEED + rank, order=args.order)
    L = args.layers or LAYERS_CFG2
    torch.cuda.synchronize()
    t = time.perf_counter()
    gm = E.Mesh(m.cells, m.xy, L)  # ext_mesh_create: device topology, vertex rows
    t_mesh = time.perf_counter() - t
    t = time.perf_counter()
    cs = E.Space(gm, P1_DELTA, ncomp=3)
    p1 = E.Space(gm, P1_DELTA)
    dg = E.Space(gm, DG1_DELTA)
    torch.cuda.synchronize()
    t_spaces = time.perf_counter() - t
    X = E.extrude_coords(gm, cs) if geometry == "flat" else geometry_coords(m, L, geometry, dev)
    Xr = X.view(-1, 3)
    f = (torch.sin(Xr[:, 0]) * torch.cos(Xr[:, 1]) * Xr[:, 2]).contiguous()  # synthetic input data
    x = torch.from_numpy(meshgen.uniform_field(p1.ndofs, SEED + 10 + rank)).to(dev)
    b, y, out = p1.zeros(), p1.zeros(), dg.zeros()
    V, C = m.nverts, m.ncells
    vb = valuable_bytes_cfg2(V, C, L)
    vb_paper = valuable_bytes_cfg2(V, C, L, maps=False)
    READ, WRITE = E.EXT_READ, E.EXT_WRITE
    h = {"gm": gm.handle}
    # WRITE: the P1xP1 loops overwrite b and y with the assembled results
    a_rhs = [(cs.handle, X, READ), (p1.handle, f, READ), (p1.handle, b, WRITE)]
    a_mass = [(cs.handle, X, READ), (p1.handle, x, READ), (p1.handle, y, WRITE)]
    a_int = [(p1.handle, x, READ), (dg.handle, out, WRITE)]
    s = stream.cuda_stream

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        E.ext_par_loop(h["gm"], E.EXT_K_RHS_P1P1, a_rhs, s)
        if ev is not None:
            ev[1].record(stream)
        E.ext_par_loop(h["gm"], E.EXT_K_MASS_P1P1, a_mass, s)
        if ev is not None:
            ev[2].record(stream)
        E.ext_par_loop(h["gm"], E.EXT_K_INTERP_DG1, a_int, s)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    E.ext_sync_check(s)
    rates = E.ext_fp64_rates(s)  # FP64 issue rates of this GPU, for the roofline
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clk = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(world)
    E.ext_sync_check(s)
    ms = t0.elapsed_time(t1) / args.steps
    ms = max_over_ranks(ms, world)
    k_rhs = [e[0].elapsed_time(e[1]) for e in evs]
    k_mass = [e[1].elapsed_time(e[2]) for e in evs]
    k_int = [e[2].elapsed_time(e[3]) for e in evs]
    extra = {"setup_s": {"mesh_create": round(t_mesh, 3), "spaces": round(t_spaces, 3),
                         "note": "host wall time of ext_mesh_create (topology upload, edges, vertex rows) and "
                                 "ext_number_dofs for the three spaces; outside the timed step"}}
    reps = 20
    if geometry == "flat" and not args.no_forms:
        extra["forms_ms"] = time_p1_forms(E, gm, cs, p1, X, x, y, stream, ["split", "factored", "cells"], reps)
        old_flat = E.ext_get_option(E.EXT_OPT_P1_FLAT)
        E.ext_set_option(E.EXT_OPT_P1_FLAT, E.EXT_P1_FLAT_FUSED)
        extra["forms_ms"]["gather_fused"] = time_p1_forms(E, gm, cs, p1, X, x, y, stream, ["split"], reps)["split"]
        E.ext_set_option(E.EXT_OPT_P1_FLAT, E.EXT_P1_FLAT_SPLIT)
        extra["forms_ms"]["gather_split"] = time_p1_forms(E, gm, cs, p1, X, x, y, stream, ["split"], reps)["split"]
        E.ext_set_option(E.EXT_OPT_P1_FLAT, old_flat)
        for kind in ("terrain", "wavy", "tilted"):
            Xk = geometry_coords(m, L, kind, dev)
            extra["forms_ms"][kind] = time_p1_forms(E, gm, cs, p1, Xk, x, y, stream, ["split"], reps)["split"]
            del Xk
        torch.cuda.empty_cache()
    if args.no_e2e:
        e2e_ms = None
    else:
        e2e_ms = e2e_time(args, world, stream.device, gm, cs, p1, dg, X, f, x)
    h2d = (X.numel() + f.numel() + x.numel()) * 8
    d2h = (b.numel() + y.numel() + out.numel()) * 8
    if rank != 0:
        return None
    return report(args, world, m, L, vb, vb_paper, ms, k_rhs, k_mass, k_int, clocks, e2e_ms, h2d, d2h, rates,
                  extra)


def e2e_time(args, world, dev, gm, cs, p1, dg, X, f, x):
    """The benchmark step end to end through the public API: every step copies
    its inputs (coordinates, f, x) from pinned host memory, runs the three
    par_loops and reads all three outputs back into pinned host memory.
    Steps are pipelined over two device buffer sets and three streams
    (copy-in, compute, copy-out), so one step's read-back overlaps the next
    step's uploads and kernels; the timed region spans the first upload to
    the last read-back."""
    import torch
    import paper_1604_05937_gb300 as E
    pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t.cpu())
    hX, hf, hx = pin(X), pin(f), pin(x)
    hb = torch.empty(p1.ndofs, dtype=torch.float64, pin_memory=True)
    hy = torch.empty(p1.ndofs, dtype=torch.float64, pin_memory=True)
    hout = torch.empty(dg.ndofs, dtype=torch.float64, pin_memory=True)
    sets = []
    for _ in range(2):
        d = {"X": torch.empty_like(X), "f": torch.empty_like(f), "x": torch.empty_like(x),
             "b": p1.zeros(), "y": p1.zeros(), "out": dg.zeros()}
        R, W, I = E.EXT_READ, E.EXT_WRITE, E.EXT_INC
        d["rhs"] = [(cs.handle, d["X"], R), (p1.handle, d["f"], R), (p1.handle, d["b"], W)]
        d["mass"] = [(cs.handle, d["X"], R), (p1.handle, d["x"], R), (p1.handle, d["y"], W)]
        d["int"] = [(p1.handle, d["x"], R), (dg.handle, d["out"], W)]
        sets.append(d)
    s_in, s_cmp, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    ev = lambda: torch.cuda.Event()
    in_done, int_done, cmp_done, out_done = ([ev() for _ in range(2)] for _ in range(4))

    def run(nsteps):
        for i in range(nsteps):
            k = i % 2
            d = sets[k]
            s_in.wait_event(cmp_done[k])          # step i-2 finished reading this set's inputs
            with torch.cuda.stream(s_in):
                d["X"].copy_(hX, non_blocking=True)
                d["f"].copy_(hf, non_blocking=True)
                d["x"].copy_(hx, non_blocking=True)
            in_done[k].record(s_in)
            s_cmp.wait_event(in_done[k])
            s_cmp.wait_event(out_done[k])         # step i-2's outputs have been read back
            with torch.cuda.stream(s_cmp):
                E.ext_par_loop(gm.handle, E.EXT_K_INTERP_DG1, d["int"], s_cmp.cuda_stream)
                int_done[k].record(s_cmp)
                E.ext_par_loop(gm.handle, E.EXT_K_RHS_P1P1, d["rhs"], s_cmp.cuda_stream)
                E.ext_par_loop(gm.handle, E.EXT_K_MASS_P1P1, d["mass"], s_cmp.cuda_stream)
            cmp_done[k].record(s_cmp)
            s_out.wait_event(int_done[k])
            with torch.cuda.stream(s_out):
                hout.copy_(d["out"], non_blocking=True)
            s_out.wait_event(cmp_done[k])
            with torch.cuda.stream(s_out):
                hb.copy_(d["b"], non_blocking=True)
                hy.copy_(d["y"], non_blocking=True)
            out_done[k].record(s_out)

    run(2)
    torch.cuda.synchronize()
    barrier(world)
    n = max(4, min(args.steps, 12))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    s_cmp.wait_event(t0)
    s_out.wait_event(t0)
    run(n)
    s_out.wait_stream(s_in)
    s_out.wait_stream(s_cmp)
    t1.record(s_out)
    torch.cuda.synchronize()
    E.ext_sync_check(s_cmp.cuda_stream)
    # the read-back equals the device result of the same step
    assert torch.equal(hout, sets[(n - 1) % 2]["out"].cpu())
    ms = max_over_ranks(t0.elapsed_time(t1) / n, world)
    del sets
    torch.cuda.empty_cache()
    return ms


def report(args, world, m, L, vb, vb_paper, ms, k_rhs, k_mass, k_int, clocks, e2e_ms, h2d, d2h, rates, extra):
    hbm, hbm_kind, sm_max = peaks()
    V, C = m.nverts, m.ncells
    geometry = args.geometry
    value = world * vb["total"] / (ms * 1e-3) / 1e9
    items = C * (L + 1)
    mass_ms = statistics.mean(k_rhs + k_mass)
    ops_peak = FP64_OPS_PER_CLK_PER_SM * SMS * sm_max * 1e6 / 1e9  # G FP64 ops/s
    E_ = base_edges(m.cells)
    form = p1_form(items, L, geometry=geometry)
    main = form_entry(form, mass_ms, V, C, L, E_, geometry, ops_peak, hbm)
    traffic = load_traffic({"gather": "p1_mass_launch", "gather-sigma": "p1_sigma_launch"}.get(form, "p1_cells_launch"))
    nbytes = p1_bytes_8d(V, C, L)
    if form in ("gather", "gather-sigma"):
        if form == "gather":
            label = ("gather (flat-level special case): the probe found a straight extrusion with flat levels, so "
                     "M = Mh (x) Mv, formed in one optimistic pass (g = Mh f per level through the vertex rows, then "
                     "Mv by warp shuffles along each column) beside one straightness bit per coordinate DoF, and a "
                     "fix-up launch that sends the DoFs next to a DoF that is not straight to the general rule; "
                     "the row weights and the level table are computed from the coordinate field in every launch")
            algorithmic = (f"3 FP64 ops per DoF x {V * (L + 1)} DoFs + 1 per vertex-row entry and level x "
                           f"{V + 2 * E_} entries x {L + 1} levels + 7 per cell x {C} + 4 per edge x {E_} = "
                           f"{main['fp64_ops']} per launch")
        else:
            label = ("terrain-following gather: the probe found vertical columns with z = z0 + sigma_l D(x, y), so "
                     "M = Hd (x) Mv(sigma) with Hd the depth-weighted P1 mass matrix of the base, formed in one "
                     "optimistic pass beside the check of every DoF against that model within 2^-42 D min(sigma "
                     "spacing); DoFs next to a DoF that fails go to the general rule")
            algorithmic = (f"5 FP64 ops per DoF x {V * (L + 1)} DoFs (Mv and the model check) + 1 per vertex-row "
                           f"entry and level x {V + 2 * E_} x {L + 1} + 18 per cell + 14 per edge + 5 per vertex = "
                           f"{main['fp64_ops']} per launch")
        kname = ("P1xP1 RHS / mass-action launch (k_p1_levels + k_p1_prep + k_p1_sigma_prep + k_p1_rowweights + "
                 "k_p1_opt + k_p1_fix + k_vgather + k_vgather_general + k_p1_cells; the kernels of the other modes "
                 "exit at once)")
    else:
        per = P1_PRISM_OPS["general" if geometry == "tilted" else "vertical"]
        label = (f"cell loop (Algorithm 3 over cells, one element vector per prism, {geometry} geometry): the probe "
                 "found no flat straight extrusion")
        algorithmic = (f"{per} FP64 ops per prism x {C * L} prisms + 3 per (column, level) item x {items} = "
                       f"{main['fp64_ops']} per launch")
        kname = ("P1xP1 RHS / mass-action launch (k_p1_levels + k_p1_prep probe + k_vgather clearing b + "
                 "k_p1_cells; the gather-form kernels exit at once)")
    line = {
        "metric": "par_loop valuable HBM GB/s (P1xP1 RHS + mass action + DG1 interpolation, 100 layers, RCM)",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64",
        "data": f"synthetic (seeded perturbed structured triangulation, RCM; {geometry} levels; f = sin x cos y z; "
                "x ~ U(-1,1))",
        "config": {"workload": f"extruded prisms: {C} base triangles x {L} layers, {args.order} base order, "
                               f"{geometry} geometry, P1xP1 RHS + P1xP1 mass action + DG1xDG1 interpolation",
                   "base_cells": C, "base_vertices": V, "layers": L, "geometry": geometry, "global_batch": world,
                   "l2": "inputs larger than L2 (7.5 GB working set per step, L2 129 MB)",
                   "valuable_bytes_per_step": vb["total"], "valuable_bytes_paper_definition": vb_paper["total"],
                   "parallelism": f"replicas x{world}"},
        "kernels_ms": {"rhs_p1p1": round(statistics.mean(k_rhs), 4), "mass_p1p1": round(statistics.mean(k_mass), 4),
                       "interp_dg1": round(statistics.mean(k_int), 4)},
        "kernels_gbs": {"rhs_p1p1": round(vb["rhs"] / statistics.mean(k_rhs) / 1e6, 1),
                        "mass_p1p1": round(vb["mass"] / statistics.mean(k_mass) / 1e6, 1),
                        "interp_dg1": round(vb["interp"] / statistics.mean(k_int) / 1e6, 1)},
        "hbm_frac": {"interp_dg1": round(vb["interp"] / statistics.mean(k_int) / 1e6 / hbm, 4),
                     "p1p1": main["hbm_frac"], "step": round(value / world / hbm, 4), "peak_gbs": hbm,
                     "peak_kind": hbm_kind},
        "roofline": {"kernel": kname, "form": label, "bound": "alu",
                     "achieved": main["fp64_gops"], "peak": round(ops_peak, 2), "unit": "G FP64 ops/s",
                     "frac": main["fp64_frac"], "traffic": traffic, "algorithmic": algorithmic,
                     "peak_note": "2 FP64 FMA/clk/SM x 152 SMs x max SM clock (nominal 1.25 TFLOP/s); "
                                  "all products and sums issued as DFMA",
                     "hbm": {"algorithmic_bytes": nbytes,
                             "bytes_note": "24 per vertex level (coordinates) + 16 (input, output) + 24 per base "
                                           "cell (one map row), each moved once",
                             "achieved_gbs": main["gbs"], "peak_gbs": hbm, "frac": main["hbm_frac"]},
                     "measured_fp64_rates_gops": {k: round(v, 1) for k, v in rates.items()},
                     "frac_of_measured_dfma": round(main["fp64_gops"] / rates["dfma"], 4)},
        "setup_s": extra["setup_s"],
        "e2e": None if e2e_ms is None else {
            "value": round(world * vb["total"] / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": (2 * P1_KERNELS[form] + 1) * args.steps,
        "clocks": clocks,
    }
    if "forms_ms" in extra:
        fm = extra["forms_ms"]
        line["p1_forms"] = {
            "note": "one mass-action launch (WRITE) on this mesh in each form, forced with ext_set_option, mean of "
                    "20 back-to-back launches; terrain, wavy, tilted: the same mesh with terrain-following levels "
                    "(every prism's top face tilted; the probe picks the terrain-following gather), with bent "
                    "levels (no common profile; the cell loop) and with leaning columns (the cell loop), default "
                    "form",
            "gather": form_entry("gather", fm["split"], V, C, L, E_, "flat", ops_peak, hbm),
            "gather_split": form_entry("gather", fm["gather_split"], V, C, L, E_, "flat", ops_peak, hbm,
                                       launches=P1_KERNELS["gather-split"]),
            "gather_fused": form_entry("gather", fm["gather_fused"], V, C, L, E_, "flat", ops_peak, hbm,
                                       launches=P1_KERNELS["gather-split"]),
            "factored_cell_pass": form_entry("factored", fm["factored"], V, C, L, E_, "flat", ops_peak, hbm),
            "cell_loop": form_entry("cells-forced", fm["cells"], V, C, L, E_, "flat", ops_peak, hbm),
            "terrain_gather": form_entry("gather-sigma", fm["terrain"], V, C, L, E_, "terrain", ops_peak, hbm),
            "wavy_cell_loop": form_entry("cells", fm["wavy"], V, C, L, E_, "wavy", ops_peak, hbm),
            "tilted_cell_loop": form_entry("cells", fm["tilted"], V, C, L, E_, "tilted", ops_peak, hbm),
        }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, L, args.cpu_runs, geometry)
    return line


def code_hash(path: str) -> str:
    """SHA-256 of a source file's code: // comments, trailing blanks and blank
    lines removed, so that editing a comment keeps a kernel's counters valid
    and any change to its code voids them."""
    import hashlib
    import re
    lines = []
    with open(path) as f:
        for line in f:
            line = re.sub(r"//.*$", "", line).rstrip()
            if line:
                lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def load_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel's code has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)[kernel]
        if code_hash(os.path.join(ROOT, t["source"])) != t["code_sha256"]:
            return None
        return t["bytes_per_launch"]
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle baseline
CPU_SAMPLE_COLUMNS = 2048  # base columns of the CPU sample (all layers, all three loops)


def host_cpu() -> str:
    """Host CPU model: /proc/cpuinfo's model name, else lscpu's (Arm kernels
    list only part numbers in /proc/cpuinfo)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name") and ":" in line:
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name") and ":" in line:
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


class CpuSample:
    """The benchmark step of the oracle on the first S base columns (all
    layers): RHS, mass action and DG1 interpolation, serial (one core) or
    over base-cell colours on every host core (OpenMP).  Valuable bytes of
    the sample: the touched vertex columns (coordinates, input, output), the
    DG1 output of the S cell columns and S map rows per map, each once."""

    def __init__(self, m, L, S=CPU_SAMPLE_COLUMNS, geometry="flat"):
        import oracle as O
        self.O = O
        self.L, self.S = L, min(S, m.ncells)
        self.cells = np.ascontiguousarray(m.cells[:self.S])
        self.X_sp, self.X = O.coords(m.cells, m.xy, L)
        if geometry != "flat":
            self.X = meshgen.level_coords(m, L, seed=SEED + 20, kind=geometry).reshape(-1)
        self.p1 = O.number(m.cells, m.nverts, L, P1_DELTA)
        self.dg = O.number(m.cells, m.nverts, L, DG1_DELTA)
        Xr = self.X.reshape(-1, 3)
        self.f = np.sin(Xr[:, 0]) * np.cos(Xr[:, 1]) * Xr[:, 2]
        self.x = meshgen.uniform_field(self.p1.ndofs, SEED + 10)
        self.b = np.zeros(self.p1.ndofs)
        self.y = np.zeros(self.p1.ndofs)
        self.out = np.zeros(self.dg.ndofs)
        sub = lambda sp: O.Space(delta=sp.delta, layers=sp.layers, ndofs=sp.ndofs, k=sp.k,
                                 map=np.ascontiguousarray(sp.map[:self.S]), offset=sp.offset)
        self.sX, self.sp1, self.sdg = sub(self.X_sp), sub(self.p1), sub(self.dg)
        self.ptr, self.ids = O.color_cells(self.cells, m.nverts)
        self.threads = O.max_threads()
        Vs = np.unique(self.cells).size
        self.bytes = 2 * (40 * Vs * (L + 1) + 48 * self.S) + (8 * Vs * (L + 1) + 48 * self.S * L + 48 * self.S)

    def run(self, parallel: bool) -> float:
        O, L = self.O, self.L
        loops = ((O.K_MASS, [(self.sX, self.X, 3, O.READ), (self.sp1, self.f, 1, O.READ), (self.sp1, self.b, 1, O.INC)]),
                 (O.K_MASS, [(self.sX, self.X, 3, O.READ), (self.sp1, self.x, 1, O.READ), (self.sp1, self.y, 1, O.INC)]),
                 (O.K_INTERP, [(self.sp1, self.x, 1, O.READ), (self.sdg, self.out, 1, O.WRITE)]))
        t = time.perf_counter()
        for k, a in loops:
            if parallel:
                O.par_loop_colored(k, self.cells, L, a, self.ptr, self.ids, self.threads)
            else:
                O.par_loop(k, self.cells, L, a)
        return time.perf_counter() - t

    def describe(self, m) -> str:
        return (f"first {self.S} of {m.ncells} base columns x {self.L} layers, RHS + mass action + DG1 "
                f"interpolation")


def cpu_baseline(m, L, runs: int = 10, geometry: str = "flat"):
    """The oracle on the CPU sample: the all-core variant (base-cell colours
    in sequence, cells of a colour over every host core) and the serial one,
    each the minimum of `runs` runs (the paper's timing rule)."""
    cs = CpuSample(m, L, geometry=geometry)
    cs.run(True)  # first touch of the sample's pages
    tp = min(cs.run(True) for _ in range(runs))
    ts = min(cs.run(False) for _ in range(runs))
    return {"value": round(cs.bytes / tp / 1e9, 4), "unit": "GB/s", "cores": cs.threads, "kind": "oracle",
            "sample": f"{cs.describe(m)}; min of {runs} runs each",
            "variant": f"OpenMP over {cs.ptr.size - 1} vertex-disjoint base-cell colours, {cs.threads} threads",
            "serial": {"value": round(cs.bytes / ts / 1e9, 4), "unit": "GB/s", "cores": 1, "s_per_run": round(ts, 3)},
            "s_per_run": round(tp, 3), "nproc": os.cpu_count(), "host_cpu": host_cpu()}


# ----------------------------------------------------------------------------- other workloads
class Flusher:
    """Writes a buffer twice the L2 size between timed repetitions."""

    def __init__(self, dev):
        import torch
        l2 = torch.cuda.get_device_properties(dev).L2_cache_size
        self.buf = torch.empty(max(2 * l2, 64 << 20) // 8, dtype=torch.float64, device=dev)

    def __call__(self):
        self.buf.fill_(1.0)


def time_kernel(fn, reps, stream, flush=None, pre=None):
    """min and median device time (ms) of fn() over reps, flushing L2 before each."""
    import torch
    ts = []
    for _ in range(reps):
        if pre is not None:
            pre()
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return min(ts), statistics.median(ts)


def _common(args, world, metric, value, unit, cfg, extra, clocks, launches, ms_step=None):
    line = {"metric": metric, "value": round(value, 2), "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None if ms_step is None else round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "gpu_launches": launches, "clocks": clocks}
    line.update(extra)
    return line


def run_cfg3(args, rank, world, local):
    """Layer sweep on the 250k-triangle base: P1xP1 RHS, DG0 copy, DG1xDG1 copy,
    RCM and random base orderings, L2 flushed before every timed launch."""
    import torch
    import paper_1604_05937_gb300 as E
    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = Flusher(dev)
    sweep = {}
    launches = 0
    clk = ClockSampler(local)
    clk.start()
    for order in ("rcm", "random"):
        m = meshgen.tri_mesh(354, seed=SEED + 3, order=order)
        V, C = m.nverts, m.ncells
        sweep[order] = {}
        for L in (1, 2, 5, 10, 20, 50, 100, 200):
            gm = E.Mesh(m.cells, m.xy, L)
            cs = E.Space(gm, P1_DELTA, ncomp=3)
            p1 = E.Space(gm, P1_DELTA)
            d0 = E.Space(gm, (0, 0, 0, 0, 0, 1))
            d1 = E.Space(gm, DG1_DELTA)
            X = E.extrude_coords(gm, cs)
            Xr = X.view(-1, 3)
            f = (torch.sin(Xr[:, 0]) * torch.cos(Xr[:, 1]) * Xr[:, 2]).contiguous()
            b = p1.zeros()
            a0 = torch.rand(d0.ndofs, dtype=torch.float64, device=dev)
            o0 = d0.zeros()
            a1 = torch.rand(d1.ndofs, dtype=torch.float64, device=dev)
            o1 = d1.zeros()
            rhs = lambda: E.ext_par_loop(gm.handle, E.EXT_K_RHS_P1P1, [(cs.handle, X, E.EXT_READ),
                                         (p1.handle, f, E.EXT_READ), (p1.handle, b, E.EXT_INC)], s)
            c0 = lambda: E.ext_par_loop(gm.handle, E.EXT_K_COPY_DG, [(d0.handle, a0, E.EXT_READ),
                                        (d0.handle, o0, E.EXT_WRITE)], s)
            c1 = lambda: E.ext_par_loop(gm.handle, E.EXT_K_COPY_DG, [(d1.handle, a1, E.EXT_READ),
                                        (d1.handle, o1, E.EXT_WRITE)], s)
            for fn in (rhs, c0, c1):
                for _ in range(args.warmup):
                    fn()
            reps = max(5, args.steps)
            t_rhs = time_kernel(rhs, reps, stream, flush, pre=b.zero_)
            t_c0 = time_kernel(c0, reps, stream, flush)
            t_c1 = time_kernel(c1, reps, stream, flush)
            launches += (p1_kernels(C * (L + 1), L, write=False) + 2) * (reps + args.warmup)
            nP1 = V * (L + 1)
            vb_rhs = 40 * nP1 + 48 * C
            vb_c0 = 16 * C * L + 4 * C
            vb_c1 = 96 * C * L + 24 * C
            items = C * (L + 1)
            sweep[order][L] = {
                "rhs_ms": round(t_rhs[0], 4), "rhs_gbs": round(vb_rhs / t_rhs[0] / 1e6, 1),
                "rhs_gops": round(p1_ops(nP1, items, C, L) / t_rhs[0] / 1e6, 1),
                "dg0_ms": round(t_c0[0], 4), "dg0_gbs": round(vb_c0 / t_c0[0] / 1e6, 1),
                "dg1_ms": round(t_c1[0], 4), "dg1_gbs": round(vb_c1 / t_c1[0] / 1e6, 1)}
            E.ext_sync_check(s)
            del gm, cs, p1, d0, d1, X, f, b, a0, o0, a1, o1
            torch.cuda.empty_cache()
    clocks = clk.stop()
    if rank != 0:
        return None
    hbm, hbm_kind, _ = peaks()
    top = sweep["rcm"][100]
    extra = {"sweep": sweep, "hbm_peak_gbs": hbm, "peak_kind": hbm_kind,
             "timing": "min over reps, L2 flushed (2x L2 buffer written) before every timed launch"}
    return _common(args, world, "layer sweep: P1xP1 RHS valuable GB/s at 100 layers (RCM); sweep of RHS, DG0, DG1 copy",
                   top["rhs_gbs"], "GB/s",
                   {"workload": "extruded prisms: 250632 base triangles x {1,2,5,10,20,50,100,200} layers, RCM and "
                                "random base order; P1xP1 RHS, DG0 copy, DG1xDG1 copy", "l2": "flushed"},
                   extra, clocks, launches)


# FP64 operations per hexahedral cell-layer (straight columns) of the Q2/DG2
# u^2 v kernels, counted from the sum-factorised pipeline: per vertical Gauss
# point 18 (A) + 30 (C) + 40 (D) + 16 (P) + 16 (r) + 114 (projection) for the
# residual, plus 1 (h) + 18 (differences) + 27 (scaling); the adjoint
# evaluates two fields and forms 2 P w; the fused pass shares P.
HEX_OPS = {1: 1 + 18 + 4 * 234 + 27, 2: 1 + 36 + 4 * 338 + 27, 3: 1 + 36 + 4 * 468 + 54}
# per prism cell-layer of the P1xP1 u^2 v residual / adjoint / both (straight
# prism, all issued as DFMA): 2 for the weight |2A| |h| / 12, 21 per field
# evaluated at the six points, 2 for the projection constants (weight / 6,
# weight / 2; 1 more for the adjoint's doubled ones), 6 point products and
# 24 for the projection per output
PRISM_U2V_OPS = {1: 55, 2: 77, 3: 107}


def run_cfg4(args, rank, world, local):
    """Q2xP2 and DG2 u^2 v residual and adjoint on the 500k-quad base, 64 layers."""
    import torch
    import paper_1604_05937_gb300 as E
    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    m = meshgen.quad_mesh(args.n or 707, seed=SEED + 4, order="rcm")
    L = args.layers or 64
    V, C = m.nverts, m.ncells
    gm = E.Mesh(m.cells, m.xy, L)
    E_ = gm.N[1]
    cs = E.Space(gm, P1_DELTA, ncomp=3)
    X = E.extrude_coords(gm, cs)
    res = {}
    launches = 0
    clk = ClockSampler(local)
    clk.start()
    tot_bytes, tot_ms = 0, 0.0
    for name, delta, acc in (("Q2xP2", (1, 1, 1, 1, 1, 1), E.EXT_INC), ("DG2", (0, 0, 0, 0, 0, 27), E.EXT_WRITE)):
        sp = E.Space(gm, delta)
        u = torch.from_numpy(meshgen.uniform_field(sp.ndofs, SEED + 40)).to(dev)
        w = torch.from_numpy(meshgen.uniform_field(sp.ndofs, SEED + 41)).to(dev)
        F, G = sp.zeros(), sp.zeros()
        R = E.EXT_READ
        fwd = lambda: E.ext_par_loop(gm.handle, E.EXT_K_U2V_FWD, [(cs.handle, X, R), (sp.handle, u, R),
                                     (sp.handle, F, acc)], s)
        adj = lambda: E.ext_par_loop(gm.handle, E.EXT_K_U2V_ADJ, [(cs.handle, X, R), (sp.handle, u, R),
                                     (sp.handle, w, R), (sp.handle, G, acc)], s)
        both = lambda: E.ext_par_loop(gm.handle, E.EXT_K_U2V_FWDADJ, [(cs.handle, X, R), (sp.handle, u, R),
                                      (sp.handle, w, R), (sp.handle, F, acc), (sp.handle, G, acc)], s)
        for fn in (fwd, adj, both):
            fn()
        reps = max(3, min(args.steps, 10))
        tf = time_kernel(fwd, reps, stream)
        ta = time_kernel(adj, reps, stream)
        tb = time_kernel(both, reps, stream)
        launches += 3 * (reps + 1)
        E.ext_sync_check(s)
        n = sp.ndofs
        coords_b = 24 * V * (L + 1) + 32 * C
        umap_b = 4 * 27 * C
        vb_f = coords_b + umap_b + 16 * n
        vb_a = coords_b + umap_b + 24 * n
        vb_b = coords_b + umap_b + 32 * n
        cells = C * L
        res[name] = {"ndofs": n,
                     "fwd_ms": round(tf[0], 3), "fwd_gbs": round(vb_f / tf[0] / 1e6, 1),
                     "fwd_gops": round(HEX_OPS[1] * cells / tf[0] / 1e6, 1),
                     "adj_ms": round(ta[0], 3), "adj_gbs": round(vb_a / ta[0] / 1e6, 1),
                     "adj_gops": round(HEX_OPS[2] * cells / ta[0] / 1e6, 1),
                     "fwdadj_ms": round(tb[0], 3), "fwdadj_gbs": round(vb_b / tb[0] / 1e6, 1),
                     "fwdadj_gops": round(HEX_OPS[3] * cells / tb[0] / 1e6, 1)}
        tot_bytes += vb_b
        tot_ms += tb[0]
        del sp, u, w, F, G
        torch.cuda.empty_cache()
    clocks = clk.stop()
    if rank != 0:
        return None
    extra = {"hex": res, "fp64_ops_per_cell": HEX_OPS, "fp64_peak_gops_nominal": 2 * SMS * SM_MAX_MHZ / 1e3}
    return _common(args, world, "u^2 v residual + adjoint on hexahedra: valuable GB/s (Q2xP2 and DG2, fused pass)",
                   world * tot_bytes / tot_ms / 1e6, "GB/s",
                   {"workload": f"extruded hexahedra: {C} base quads x {L} layers, RCM; Q2xP2 ({E_} edges) and DG2"},
                   extra, clocks, launches, ms_step=tot_ms)


def run_cfg5(args, rank, world, local):
    """64 prism meshes (log-uniform base sizes, uniform layer counts): u^2 v
    residual + adjoint in one captured persistent launch vs 64 plain launches."""
    import torch
    import paper_1604_05937_gb300 as E
    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    bp = meshgen.batched_params(count=args.count, seed=SEED + 5 + 1000 * rank, cmin=args.cmin, cmax=args.cmax,
                                lmax=args.lmax)
    meshes, per, keep = [], [], []
    vb, ops, cells_total = 0, 0, 0
    for i, (n, L) in enumerate(zip(bp.n, bp.layers)):
        m = meshgen.tri_mesh(n, seed=SEED + 500 + i, order="rcm")
        gm = E.Mesh(m.cells, m.xy, L)
        cs = E.Space(gm, P1_DELTA, ncomp=3)
        sp = E.Space(gm, P1_DELTA)
        X = E.extrude_coords(gm, cs)
        u = torch.rand(sp.ndofs, dtype=torch.float64, device=dev) * 2 - 1
        w = torch.rand(sp.ndofs, dtype=torch.float64, device=dev) * 2 - 1
        F, G = sp.zeros(), sp.zeros()
        meshes.append(gm)
        per.append([(cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, w, E.EXT_READ), (sp, F, E.EXT_INC),
                    (sp, G, E.EXT_INC)])
        keep.append((cs, sp))
        vb += 56 * m.nverts * (L + 1) + 48 * m.ncells
        ops += PRISM_U2V_OPS[3] * m.ncells * L
        cells_total += m.ncells * L
    # the first plan times the candidates (EXTMESH_TUNE=force, its result
    # stored in the tuning cache: EXTMESH_TUNE_CACHE, else the user's cache
    # folder); the second plan of the same workload reads its parameters from
    # the cache
    os.environ["EXTMESH_TUNE"] = "force"
    t0 = time.time()
    tuned = E.Batch(meshes, E.EXT_K_U2V_FWDADJ, per, params=None)
    tune_s = time.time() - t0
    del os.environ["EXTMESH_TUNE"]
    t0 = time.time()
    batch = E.Batch(meshes, E.EXT_K_U2V_FWDADJ, per, params=None)
    cached_s = time.time() - t0
    plans = {"tuned": dict(tuned.plan_info, wall_seconds=round(tune_s, 2), params=tuned.params),
             "cached": dict(batch.plan_info, wall_seconds=round(cached_s, 2), params=batch.params)}

    def plain():
        for gm, args_ in zip(meshes, per):
            E.ext_par_loop(gm.handle, E.EXT_K_U2V_FWDADJ, [(sp.handle, t, a) for sp, t, a in args_], s)

    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        plain()  # warm-up on the side stream before capture
    stream.wait_stream(side)
    with torch.cuda.graph(g, stream=side):
        for gm, args_ in zip(meshes, per):
            E.ext_par_loop(gm.handle, E.EXT_K_U2V_FWDADJ, [(sp.handle, t, a) for sp, t, a in args_],
                           side.cuda_stream)
    reps = max(3, min(args.steps, 10))
    for _ in range(args.warmup):
        batch.launch(s)
        plain()
    clk = ClockSampler(local)
    clk.start()
    tb = time_kernel(lambda: batch.launch(s), reps, stream)
    tt = time_kernel(lambda: tuned.launch(s), reps, stream)
    tp = time_kernel(plain, reps, stream)
    tg = time_kernel(g.replay, reps, stream)
    clocks = clk.stop()
    E.ext_sync_check(s)
    if rank != 0:
        return None
    extra = {"batched_ms": round(tb[0], 3), "plain_64_launches_ms": round(tp[0], 3),
             "plain_captured_graph_ms": round(tg[0], 3),
             "speedup_vs_plain": round(tp[0] / tb[0], 3), "speedup_vs_captured_plain": round(tg[0] / tb[0], 3),
             "autotuned_params": batch.params, "autotune_seconds": round(tune_s, 2),
             "plans": dict(plans, tuned_launch_ms=round(tt[0], 3), cached_launch_ms=round(tb[0], 3)),
             "fp64_gops": round(ops / tb[0] / 1e6, 1), "cells": cells_total,
             "meshes": {"count": args.count, "base_cells": [2 * n * n for n in bp.n], "layers": bp.layers,
                        "base_cells_range": [args.cmin, args.cmax], "layers_range": [8, args.lmax]}}
    return _common(args, world, f"batched u^2 v residual + adjoint over {args.count} prism meshes: valuable GB/s "
                   "(one captured persistent launch)", world * vb / tb[0] / 1e6, "GB/s",
                   {"workload": f"{args.count} extruded prism meshes, {cells_total} prisms, P1xP1 u^2 v forward + adjoint",
                    "valuable_bytes": vb},
                   extra, clocks, args.count * (2 * reps + args.warmup) + 2 * reps, ms_step=tb[0])


# FP64 ops per unit of the nine-space mass kernels (straight prisms); unit =
# cell-layer (see k_tp.cu); CG1xCG1 runs the P1xP1 split form (p1_ops)
TP_SPACES = [("CG1xCG1", (1, 0, 0, 0, 0, 0), None), ("CG1xDG0", (0, 1, 0, 0, 0, 0), 8),
             ("CG1xDG1", (0, 2, 0, 0, 0, 0), 20), ("DG0xCG1", (0, 0, 0, 0, 1, 0), 7),
             ("DG0xDG0", (0, 0, 0, 0, 0, 1), 3), ("DG0xDG1", (0, 0, 0, 0, 0, 2), 7),
             ("DG1xCG1", (0, 0, 0, 0, 3, 0), 20), ("DG1xDG0", (0, 0, 0, 0, 0, 3), 8),
             ("DG1xDG1", (0, 0, 0, 0, 0, 6), 20)]


def run_cfg6(args, rank, world, local):
    """The paper's Sec. 4.1 experiment on GB300: I_1 = int f v dx on all nine
    prism spaces (CG1/DG0/DG1 horizontal x vertical), ~15M cells; (a) at 100
    layers on a 150k-triangle base (the Tables 4/5 analogue), (b) with the
    total cell count held near 15M while the layers vary (Sec. 4.1.3), RCM and
    random base orders, L2 flushed before every timed launch."""
    import torch
    import paper_1604_05937_gb300 as E
    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = Flusher(dev)
    rates = E.ext_fp64_rates(s)
    hbm, hbm_kind, sm_max = peaks()
    nominal = FP64_OPS_PER_CLK_PER_SM * SMS * sm_max / 1e3
    layer_set = [int(x) for x in args.sweep.split(",")] if args.sweep else [1, 2, 5, 10, 20, 50, 100]
    results = {}
    launches = 0
    clk = ClockSampler(local)
    clk.start()
    orders = args.orders.split(",") if args.orders else ["rcm", "random"]
    only = set(args.spaces.split(",")) if args.spaces else None
    for order in orders:
        results[order] = {}
        for L in layer_set:
            n = max(2, int(round(math.sqrt(15e6 / (2 * L)))))
            m = meshgen.tri_mesh(n, seed=SEED + 6, order=order)
            V, C = m.nverts, m.ncells
            gm = E.Mesh(m.cells, m.xy, L)
            cs = E.Space(gm, P1_DELTA, ncomp=3)
            X = E.extrude_coords(gm, cs)
            row = {"base_cells": C, "cells": C * L}
            for name, delta, ops in TP_SPACES:
                if only is not None and name not in only:
                    continue
                sp = E.Space(gm, delta)
                f = torch.rand(sp.ndofs, dtype=torch.float64, device=dev)
                b = sp.zeros()
                # WRITE: b = M f (spaces with horizontal CG1 clear b inside the launch)
                fn = lambda: E.ext_par_loop(gm.handle, E.EXT_K_MASS_TP, [(cs.handle, X, E.EXT_READ),
                                            (sp.handle, f, E.EXT_READ), (sp.handle, b, E.EXT_WRITE)], s)
                fn()
                reps = max(3, min(args.steps, 10))
                t = time_kernel(fn, reps, stream, flush)[0]
                launches += (reps + 1) * (p1_kernels(C * (L + 1), L) if ops is None
                                          else tp_kernels(C * L, L, name, write=True))
                if ops is None:
                    work = p1_ops(V * (L + 1), C * (L + 1), C, L)
                elif cgdg_gather(name, L):
                    work = cgdg_ops(V, euler_edges(V, C), C, L, 2 if name == "CG1xDG1" else 1)
                elif dgcg_optimistic(name, L, C * L):
                    work = DGCG_ITEM_OPS[name] * C * (L + 1) + 5 * C
                else:
                    work = ops * C * L
                vb_paper = 24 * V * (L + 1) + 16 * sp.ndofs
                vb = vb_paper + 24 * C + 4 * sp.k * C
                gops = work / t / 1e6
                row[name] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1),
                             "hbm_pct": round(100 * vb / t / 1e6 / hbm, 2),
                             "hbm_pct_paper_bytes": round(100 * vb_paper / t / 1e6 / hbm, 2),
                             "fp64_gops": round(gops, 1), "fp64_pct_nominal": round(100 * gops / nominal, 2)}
                del sp, f, b
            results[order][L] = row
            E.ext_sync_check(s)
            del gm, cs, X
            torch.cuda.empty_cache()
    clocks = clk.stop()
    if rank != 0:
        return None
    first = results[orders[0]]
    top = first[100] if 100 in first else first[layer_set[-1]]
    tot_b = sum(top[nm]["gbs"] * top[nm]["ms"] for nm, _, _ in TP_SPACES if nm in top)
    tot_t = sum(top[nm]["ms"] for nm, _, _ in TP_SPACES if nm in top)
    extra = {"spaces": results, "hbm_peak_gbs": hbm, "peak_kind": hbm_kind, "fp64_nominal_gops": round(nominal, 1),
             "fp64_rates_gops": {k: round(v, 1) for k, v in rates.items()},
             "fp64_ops_per_unit": {nm: (ops if ops is not None else P1_OPS_NOTE) for nm, _, ops in TP_SPACES},
             "timing": "min over reps, L2 flushed before every timed launch"}
    return _common(args, world, "I_1 = int f v dx on the nine prism spaces at 100 layers (~15M cells, RCM): valuable "
                   "GB/s over the nine launches", world * tot_b / tot_t, "GB/s",
                   {"workload": "~15M prisms: base n = sqrt(15e6 / (2 layers)), layers " +
                                ",".join(map(str, layer_set)) + "; nine CG1/DG0/DG1 x CG1/DG0/DG1 spaces; "
                                "RCM and random base order", "l2": "flushed"},
                   extra, clocks, launches)

# FP64 ops per facet of the straight-column facet kernels (the weight factor
# |2A|/24 or |2A|/2 is hoisted per column): surface mass with three nodes, c g2,
# two DFMA for c sum g and three DFMA = 6; one node: 1.  Jump: three (or one)
# differences more: 9 and 2.
FACET_MASS_OPS = {3: 6, 1: 1}
FACET_JUMP_OPS = {3: 9, 1: 2}
# FP64 ops per cell-layer of the p-adaptive DG right-hand side on a straight
# prism, by the cell's DoF count (layer height, node scaling, the element's
# closed form, and the K additions into the output block).
DGP_OPS = {1: 4, 2: 10, 3: 12, 6: 27}
FACET_SPACES = [("CG1xCG1", (1, 0, 0, 0, 0, 0), 3), ("DG0xCG1", (0, 0, 0, 0, 1, 0), 1),
                ("DG1xCG1", (0, 0, 0, 0, 3, 0), 3)]
JUMP_SPACES = [("DG0xDG0", (0, 0, 0, 0, 0, 1), 1), ("DG1xDG0", (0, 0, 0, 0, 0, 3), 3),
               ("DG0xDG1", (0, 0, 0, 0, 0, 2), 1), ("DG1xDG1", (0, 0, 0, 0, 0, 6), 3),
               ("CG1xDG1", (0, 2, 0, 0, 0, 0), 3)]


def vertex_hulls(m, first, lay):
    """Level range of every base vertex column: the hull of its cells' ranges."""
    lo = np.full(m.nverts, 1 << 30, dtype=np.int64)
    hi = np.full(m.nverts, -1, dtype=np.int64)
    for a in range(m.cells.shape[1]):
        np.minimum.at(lo, m.cells[:, a], first)
        np.maximum.at(hi, m.cells[:, a], first + lay)
    return lo, hi


def run_cfg7(args, rank, world, local):
    """Variable layers per column and horizontal-facet loops on the 999,698-
    triangle base.  (a) The default step (RHS, mass action, DG1 interpolation)
    plus DG0/DG1 copies on a mesh whose columns hang from a flat top at level
    100 with a smooth bathymetry-like depth (mean about 55 layers), against
    the same loops on the constant-layer mesh with the rounded mean; (b) the
    facet loops at 100 layers: surface mass over the 101 horizontal facets of
    each column (CG1xCG1, DG0xCG1, DG1xCG1) and the interior-facet jump on five
    vertically discontinuous spaces, and both kinds on the variable mesh.
    L2 flushed before every timed launch; min over the repetitions."""
    import torch
    import paper_1604_05937_gb300 as E
    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = Flusher(dev)
    rates = E.ext_fp64_rates(s)
    hbm, hbm_kind, sm_max = peaks()
    nominal = FP64_OPS_PER_CLK_PER_SM * SMS * sm_max / 1e3
    reps = max(3, min(args.steps, 20))
    m = meshgen.tri_mesh(args.n or N_CFG2, seed=SEED + rank, order=args.order)
    V, C = m.nverts, m.ncells
    top = args.layers or LAYERS_CFG2
    first, lay = meshgen.column_layers(m, top, SEED + 70 + rank, "bathymetry")
    mean_l = float(lay.mean())
    R, W, I = E.EXT_READ, E.EXT_WRITE, E.EXT_INC
    launches = 0
    clk = ClockSampler(local)
    clk.start()

    def timed(fn, pre=None, kernels=1):
        nonlocal launches
        fn()
        t = time_kernel(fn, reps, stream, flush, pre=pre)[0]
        launches += (reps + 1) * kernels
        return t

    def step_loops(gm):
        """RHS, mass, interpolation and two DG copies on one mesh."""
        cs = E.Space(gm, P1_DELTA, ncomp=3)
        p1 = E.Space(gm, P1_DELTA)
        dg = E.Space(gm, DG1_DELTA)
        d0 = E.Space(gm, (0, 0, 0, 0, 0, 1))
        X = E.extrude_coords(gm, cs)
        x = torch.rand(p1.ndofs, dtype=torch.float64, device=dev)
        b, out = p1.zeros(), dg.zeros()
        u0 = torch.rand(d0.ndofs, dtype=torch.float64, device=dev)
        o0 = d0.zeros()
        u1 = torch.rand(dg.ndofs, dtype=torch.float64, device=dev)
        nP1 = p1.ndofs
        cells_layers = dg.ndofs // 6
        items = int(cells_layers + C)  # (column, level) items of the P1 kernel: sum (lambda_c + 1)
        row = {}
        t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_MASS_P1P1, [(cs.handle, X, R), (p1.handle, x, R),
                                                                         (p1.handle, b, I)], s), pre=b.zero_,
                  kernels=p1_kernels(items, gm.layers, gm.variable, write=False))
        vb = 24 * nP1 + 16 * nP1 + 48 * C
        row["mass_p1p1"] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1),
                            "fp64_gops": round(p1_ops(nP1, items, C, gm.layers, gm.variable) / t / 1e6, 1),
                            "fp64_pct_nominal": round(100 * p1_ops(nP1, items, C, gm.layers, gm.variable) / t / 1e6
                                                      / nominal, 1)}
        t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_INTERP_DG1, [(p1.handle, x, R), (dg.handle, out, W)], s))
        vb = 8 * nP1 + 8 * dg.ndofs + 48 * C
        row["interp_dg1"] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1), "hbm_pct": round(100 * vb / t / 1e6 / hbm, 1)}
        for nm, sp, u, o in (("copy_dg0", d0, u0, o0), ("copy_dg1", dg, u1, out)):
            t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_COPY_DG, [(sp.handle, u, R), (sp.handle, o, W)], s))
            vb = 16 * sp.ndofs + 4 * C
            row[nm] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1), "hbm_pct": round(100 * vb / t / 1e6 / hbm, 1)}
        E.ext_sync_check(s)
        row["cell_layers"] = int(cells_layers)
        step_b = 2 * (24 * nP1 + 16 * nP1 + 48 * C) + 8 * nP1 + 8 * dg.ndofs + 48 * C
        row["step_gbs"] = round(step_b / (2 * row["mass_p1p1"]["ms"] + row["interp_dg1"]["ms"]) / 1e6, 1)
        return row, (cs, X)

    def facet_loops(gm, cs, X, cell_layers, vint_levels):
        """Facet mass on the (.)xCG1 spaces and the interior jump on five spaces."""
        row = {}
        for kind, spaces in (("facet_mass", FACET_SPACES), ("facet_jump", JUMP_SPACES)):
            for nm, delta, nh in spaces:
                sp = E.Space(gm, delta)
                u = torch.rand(sp.ndofs, dtype=torch.float64, device=dev)
                b = sp.zeros()
                kid = E.EXT_K_HFACET_MASS if kind == "facet_mass" else E.EXT_K_HFACET_JUMP
                t = timed(lambda: E.ext_par_loop(gm.handle, kid, [(cs.handle, X, R), (sp.handle, u, R),
                                                                  (sp.handle, b, I)], s), pre=b.zero_)
                if kind == "facet_mass":
                    facets = int(cell_layers + C)
                    coords = 24 * cs.ndofs
                    ops = FACET_MASS_OPS[nh]
                else:
                    facets = int(cell_layers - C)
                    coords = 24 * vint_levels
                    ops = FACET_JUMP_OPS[nh]
                vb = coords + 16 * sp.ndofs + 24 * C + 4 * sp.k * C
                row[f"{kind}:{nm}"] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1),
                                       "hbm_pct": round(100 * vb / t / 1e6 / hbm, 1),
                                       "facets": facets, "gfacets_per_s": round(facets / t / 1e6, 2),
                                       "fp64_pct_nominal": round(100 * ops * facets / t / 1e6 / nominal, 1)}
                del sp, u, b
        E.ext_sync_check(s)
        return row

    def padaptive(gm, cs, X, cell_layers):
        """p-adaptive DG (per-entity DoF counts): RHS and copy on a space with
        DG1xDG1 cells in a disk and DG0xDG0 cells elsewhere."""
        _, ne, _ = gm.N
        dent = meshgen.padaptive_dent(m, ne, SEED + 80, "disk")
        sp = E.Space(gm, dent=dent)
        f = torch.rand(sp.ndofs, dtype=torch.float64, device=dev)
        b, o = sp.zeros(), sp.zeros()
        kc = dent[-C:, 1].astype(np.int64)
        lay_c = cell_layers.astype(np.int64)
        ops = int(sum(DGP_OPS[k] * int(lay_c[kc == k].sum()) for k in (1, 2, 3, 6)))
        entries = int((kc).sum())
        t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_MASS_DGP, [(cs.handle, X, R), (sp.handle, f, R),
                                                                        (sp.handle, b, I)], s), pre=b.zero_)
        vb = 24 * cs.ndofs + 16 * sp.ndofs + 24 * C + 8 * (C + 1) + 4 * entries
        row = {"dg1_cells": int((kc == 6).sum()), "ndofs": int(sp.ndofs),
               "rhs": {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1), "hbm_pct": round(100 * vb / t / 1e6 / hbm, 1),
                       "fp64_pct_nominal": round(100 * ops / t / 1e6 / nominal, 1)}}
        t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_COPY_DG, [(sp.handle, f, R), (sp.handle, o, W)], s))
        vb = 16 * sp.ndofs + 8 * (C + 1) + 4 * entries
        row["copy"] = {"ms": round(t, 4), "gbs": round(vb / t / 1e6, 1), "hbm_pct": round(100 * vb / t / 1e6 / hbm, 1)}
        del b, o, f
        # the same right-hand side with one element everywhere, for reference
        for nm, delta in (("uniform_DG0xDG0", (0, 0, 0, 0, 0, 1)), ("uniform_DG1xDG1", (0, 0, 0, 0, 0, 6))):
            su = E.Space(gm, delta)
            fu = torch.rand(su.ndofs, dtype=torch.float64, device=dev)
            bu = su.zeros()
            t = timed(lambda: E.ext_par_loop(gm.handle, E.EXT_K_MASS_TP, [(cs.handle, X, R), (su.handle, fu, R),
                                                                           (su.handle, bu, I)], s), pre=bu.zero_)
            row[nm] = {"ms": round(t, 4)}
            del su, fu, bu
        E.ext_sync_check(s)
        return row

    results = {}
    # (a)+(b) variable layers
    gm = E.Mesh(m.cells, m.xy, cell_first=first, cell_layers=lay)
    vlo, vhi = vertex_hulls(m, first.astype(np.int64), lay.astype(np.int64))
    row, (cs, X) = step_loops(gm)
    row.update(facet_loops(gm, cs, X, int(lay.sum()), int(np.maximum(vhi - vlo - 1, 0).sum())))
    row["padaptive_dg"] = padaptive(gm, cs, X, lay)
    results["variable"] = row
    del gm, cs, X
    torch.cuda.empty_cache()
    # the same loops with constant layers: the rounded mean, and the top level
    for name, L in (("constant_mean", int(round(mean_l))), ("constant_top", top)):
        gm = E.Mesh(m.cells, m.xy, L)
        row, (cs, X) = step_loops(gm)
        if name == "constant_top":
            row.update(facet_loops(gm, cs, X, C * L, V * (L - 1)))
            row["padaptive_dg"] = padaptive(gm, cs, X, np.full(C, L))
        results[name] = row
        del gm, cs, X
        torch.cuda.empty_cache()
    clocks = clk.stop()
    if rank != 0:
        return None
    extra = {"results": results, "mean_layers": round(mean_l, 2), "top_level": top,
             "hbm_peak_gbs": hbm, "peak_kind": hbm_kind, "fp64_nominal_gops": round(nominal, 1),
             "fp64_rates_gops": {k: round(v, 1) for k, v in rates.items()},
             "timing": "min over reps, L2 flushed before every timed launch"}
    val = world * results["variable"]["step_gbs"]
    return _common(args, world, "valuable GB/s of the RHS + mass + DG1 interpolation step on a mesh with variable "
                   "layers per column (bathymetry, top level 100)", val, "GB/s",
                   {"workload": f"extruded prisms: {C} base triangles, column c spans levels 100 - l_c .. 100 with "
                                f"l_c = round(100 d(x_c, y_c)), d a smooth depth in [0.15, 0.95] (mean "
                                f"{mean_l:.1f} layers); facet loops at 100 layers; {args.order} base order",
                    "l2": "flushed"}, extra, clocks, launches)


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, all host cores (the
    coloured variant of its Algorithm 3), one pass over the CPU sample per
    step; W untimed passes, then K timed ones."""
    if rank != 0:
        return None
    m = meshgen.tri_mesh(N_CFG2, seed=SEED, order="rcm")
    L = LAYERS_CFG2
    cs = CpuSample(m, L)
    for _ in range(max(args.warmup, 1)):
        cs.run(True)
    ts = [cs.run(True) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    value = cs.bytes / t / 1e9
    C = m.ncells
    line = {
        "impl": "reference",
        "metric": "par_loop valuable HBM GB/s (P1xP1 RHS + mass action + DG1 interpolation, 100 layers, RCM)",
        "value": round(value, 4), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded perturbed structured triangulation, RCM)",
        "config": {"workload": f"extruded prisms: {C} base triangles x {L} layers, {args.order} base order, "
                               "P1xP1 RHS + P1xP1 mass action + DG1xDG1 interpolation (bounded sample)"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cs.threads, "kind": "oracle",
                         "sample": f"{cs.describe(m)}; mean of {args.steps} timed passes",
                         "nproc": os.cpu_count(), "host_cpu": host_cpu()},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def _node_cpus():
    """{NUMA node: CPUs of that node this process may run on}, nodes with CPUs only."""
    out = {}
    allowed = os.sched_getaffinity(0)
    base = "/sys/devices/system/node"
    for d in sorted(os.listdir(base)) if os.path.isdir(base) else []:
        if not d.startswith("node") or not d[4:].isdigit():
            continue
        try:
            with open(os.path.join(base, d, "cpulist")) as f:
                spec = f.read().strip()
        except OSError:
            continue
        cpus = set()
        for part in spec.split(","):
            if not part:
                continue
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= allowed
        if cpus:
            out[int(d[4:])] = sorted(cpus)
    return out


def run_hostlink(args, rank, world, local):
    """Host link rates of the end-to-end step's copies: pinned host buffers of
    1 GiB first touched from the CPUs of each NUMA node this process may use
    (so that their pages sit on that node), H2D and D2H alone and both
    directions at once, copy engines driven by cudaMemcpyAsync, best of 5."""
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prop = torch.cuda.get_device_properties(dev)
    bus = None
    for attr in ("pci_domain_id", "pci_bus_id", "pci_device_id"):
        if not hasattr(prop, attr):
            break
    else:
        bus = "%04x:%02x:%02x.0" % (prop.pci_domain_id, prop.pci_bus_id, prop.pci_device_id)
    gpu_node = None
    if bus:
        try:
            with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
                gpu_node = int(f.read().strip())
        except (OSError, ValueError):
            gpu_node = None
    nbytes = 1 << 30
    n = nbytes // 8
    d_a = torch.empty(n, dtype=torch.float64, device=dev)
    d_b = torch.empty(n, dtype=torch.float64, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    old = os.sched_getaffinity(0)
    rows = {}

    def rate(fn, streams, moved):
        best = 0.0
        for _ in range(5):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(streams[0])
            for st in streams[1:]:
                st.wait_event(a)
            fn()
            for st in streams[1:]:
                streams[0].wait_stream(st)
            b.record(streams[0])
            b.synchronize()
            best = max(best, moved / (a.elapsed_time(b) * 1e-3) / 1e9)
        return round(best, 1)

    nodes = _node_cpus()
    for node, cpus in (nodes.items() if nodes else [(-1, sorted(old))]):
        os.sched_setaffinity(0, cpus)
        h_a = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_b = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_a.fill_(1.0)  # first touch from this node's CPUs
        h_b.fill_(2.0)

        def h2d():
            with torch.cuda.stream(s1):
                d_a.copy_(h_a, non_blocking=True)

        def d2h():
            with torch.cuda.stream(s1):
                h_b.copy_(d_b, non_blocking=True)

        def both():
            with torch.cuda.stream(s1):
                d_a.copy_(h_a, non_blocking=True)
            with torch.cuda.stream(s2):
                h_b.copy_(d_b, non_blocking=True)

        rows[str(node)] = {"cpus": len(cpus), "h2d_gbs": rate(h2d, [s1], nbytes),
                           "d2h_gbs": rate(d2h, [s1], nbytes), "both_gbs": rate(both, [s1, s2], 2 * nbytes)}
        del h_a, h_b
    os.sched_setaffinity(0, old)
    if rank != 0:
        return None
    best = max(rows.values(), key=lambda r: r["h2d_gbs"] + r["d2h_gbs"])
    return {"metric": "host link: pinned host <-> GB300 copy rates per NUMA node of the host buffers",
            "value": best["both_gbs"], "unit": "GB/s", "n_gpus": world, "steps": 5, "warmup": 0,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic (1 GiB buffers)",
            "config": {"workload": "1 GiB H2D, D2H and both at once, copy engines, best of 5",
                       "gpu_pci": bus, "gpu_numa_node": gpu_node, "gpu": prop.name},
            "per_node": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-runs", type=int, default=10, help="runs of each CPU-baseline variant (minimum kept)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="base grid size (config 2: 707, config 4: 707)")
    ap.add_argument("--layers", type=int, default=None, help="layers (config 2: 100, config 4: 64)")
    ap.add_argument("--count", type=int, default=64, help="config 5: number of meshes")
    ap.add_argument("--cmax", type=float, default=5e5, help="config 5: largest base cell count")
    ap.add_argument("--cmin", type=float, default=1e4, help="config 5: smallest base cell count")
    ap.add_argument("--lmax", type=int, default=256, help="config 5: largest layer count (smallest: 8)")
    ap.add_argument("--order", choices=["rcm", "random"], default="rcm")
    ap.add_argument("--config", type=int, choices=[2, 3, 4, 5, 6, 7, 8], default=2,
                    help="2: 1M triangles x 100 layers (default); 3: layer sweep; 4: Q2/DG2 hexahedra; "
                         "5: 64-mesh batched vs plain; 6: the nine prism spaces at ~15M cells; "
                         "7: variable layers per column and horizontal-facet loops; 8: config 2 with "
                         "terrain-following levels (--geometry wavy: bent levels; tilted: leaning columns)")
    ap.add_argument("--geometry", choices=["flat", "terrain", "wavy", "tilted"], default=None,
                    help="levels of the config 2 step (config 8: terrain by default)")
    ap.add_argument("--no-forms", action="store_true", help="config 2: skip the per-form P1xP1 timings")
    ap.add_argument("--hostlink", action="store_true",
                    help="measure the host link (pinned buffers on each NUMA node) instead of a workload")
    ap.add_argument("--sweep", default=None, help="config 6: comma-separated layer counts")
    ap.add_argument("--spaces", default=None, help="config 6: comma-separated spaces (e.g. DG0xDG0); default all nine")
    ap.add_argument("--orders", default=None, help="config 6: comma-separated base orders (rcm, random); default both")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.geometry is None:
        args.geometry = "terrain" if args.config == 8 else "flat"
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build_library_only()
        runner = {2: run_ours, 3: run_cfg3, 4: run_cfg4, 5: run_cfg5, 6: run_cfg6, 7: run_cfg7,
                  8: run_ours}[args.config]
        if args.hostlink:
            runner = run_hostlink
        line = runner(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
