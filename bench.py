#!/usr/bin/env python3
"""Benchmark of the extruded-mesh par_loop on GB300: valuable HBM GB/s.

Default workload (one step = the three FP64 loops of the ~1M-triangle,
100-layer prism mesh, RCM-ordered): P1xP1 RHS assembly of int f v dx with
f = sin(x) cos(y) z (INC), P1xP1 mass-matrix action y += M x with x ~ U(-1,1)
(INC, outputs zeroed every step), and DG1xDG1 nodal interpolation of x
(WRITE).  Valuable bytes (each coordinate, input, output DoF and stencil-map
entry moved once) / device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 2|3|4|5]

--impl reference times the CPU oracle on a bounded sample of the same
workload (the reference arm: there is no reference GPU code).  Under torchrun
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
# FP64 operations (DADD/DMUL/DFMA instructions per item) of the straight-prism
# P1xP1 kernel: 2 (S) + 1 (h) + 2 (s, 2s) + 1 (sigma) + 3 (K) + 9 (three rows)
# = 18, of which 11 are FMAs: 29 flops.
MASS_OPS_PER_ITEM = 18
MASS_FLOPS_PER_ITEM = 29
MASS_FMA_PER_ITEM = 11


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
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- workload (config 2)
N_CFG2, LAYERS_CFG2, SEED = 707, 100, 1604


def valuable_bytes_cfg2(V, C, L, maps=True):
    nP1 = V * (L + 1)
    k1 = 24 * nP1 + 8 * nP1 + 8 * nP1 + (2 * 24 * C if maps else 0)        # coords, f, b (+ coords/P1 maps)
    k5 = 8 * nP1 + 48 * C * L + (2 * 24 * C if maps else 0)                 # x, out (+ P1/DG1 maps)
    return {"rhs": k1, "mass": k1, "interp": k5, "total": 2 * k1 + k5}


def run_ours(args, rank, world, local):
    import torch
    import paper_1604_05937_gb300 as E

    init_dist(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    m = meshgen.tri_mesh(args.n, seed=SEED + rank, order=args.order)
    L = args.layers
    gm = E.Mesh(m.cells, m.xy, L)
    cs = E.Space(gm, P1_DELTA, ncomp=3)
    p1 = E.Space(gm, P1_DELTA)
    dg = E.Space(gm, DG1_DELTA)
    X = E.extrude_coords(gm, cs)
    Xr = X.view(-1, 3)
    f = (torch.sin(Xr[:, 0]) * torch.cos(Xr[:, 1]) * Xr[:, 2]).contiguous()  # synthetic input data
    x = torch.from_numpy(meshgen.uniform_field(p1.ndofs, SEED + 10 + rank)).to(dev)
    b, y, out = p1.zeros(), p1.zeros(), dg.zeros()
    V, C = m.nverts, m.ncells
    vb = valuable_bytes_cfg2(V, C, L)
    vb_paper = valuable_bytes_cfg2(V, C, L, maps=False)
    READ, WRITE, INC = E.EXT_READ, E.EXT_WRITE, E.EXT_INC
    h = {"gm": gm.handle}
    a_rhs = [(cs.handle, X, READ), (p1.handle, f, READ), (p1.handle, b, INC)]
    a_mass = [(cs.handle, X, READ), (p1.handle, x, READ), (p1.handle, y, INC)]
    a_int = [(p1.handle, x, READ), (dg.handle, out, WRITE)]
    s = stream.cuda_stream

    def step(ev=None):
        b.zero_()
        y.zero_()
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

    if args.no_e2e:
        e2e_ms = None
    else:
        e2e_ms = e2e_time(args, world, stream, step, X, f, x, b, y, out)
    h2d = (X.numel() + f.numel() + x.numel()) * 8
    d2h = (b.numel() + y.numel() + out.numel()) * 8
    if rank != 0:
        return None
    return report(args, world, m, L, vb, vb_paper, ms, k_rhs, k_mass, k_int, clocks, e2e_ms, h2d, d2h)


def e2e_time(args, world, stream, step, X, f, x, b, y, out):
    """Same step through the public API with inputs copied from pinned host
    memory and results read back, copies inside the timed region."""
    import torch
    pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t.cpu())
    hX, hf, hx = pin(X), pin(f), pin(x)
    hb, hy, hout = (torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (b, y, out))
    def e2e_step():
        X.copy_(hX, non_blocking=True)
        f.copy_(hf, non_blocking=True)
        x.copy_(hx, non_blocking=True)
        step()
        hb.copy_(b, non_blocking=True)
        hy.copy_(y, non_blocking=True)
        hout.copy_(out, non_blocking=True)

    e2e_steps = max(3, min(args.steps, 10))
    e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    c1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(c0.elapsed_time(c1) / e2e_steps, world)


def report(args, world, m, L, vb, vb_paper, ms, k_rhs, k_mass, k_int, clocks, e2e_ms, h2d, d2h):
    hbm, hbm_kind, sm_max = peaks()
    V, C = m.nverts, m.ncells
    value = world * vb["total"] / (ms * 1e-3) / 1e9
    items = C * (L + 1)
    mass_ms = statistics.mean(k_rhs + k_mass)
    ops_peak = FP64_OPS_PER_CLK_PER_SM * SMS * sm_max * 1e6 / 1e9  # G FP64 ops/s
    achieved_ops = MASS_OPS_PER_ITEM * items / (mass_ms * 1e-3) / 1e9
    traffic = load_traffic("k_mass_p1")
    line = {
        "metric": "par_loop valuable HBM GB/s (P1xP1 RHS + mass action + DG1 interpolation, 100 layers, RCM)",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded perturbed structured triangulation, RCM; f = sin x cos y z; x ~ U(-1,1))",
        "config": {"workload": f"extruded prisms: {C} base triangles x {L} layers, {args.order} base order, "
                               "P1xP1 RHS + P1xP1 mass action + DG1xDG1 interpolation",
                   "base_cells": C, "base_vertices": V, "layers": L, "global_batch": world,
                   "l2": "inputs larger than L2 (7.5 GB working set per step, L2 129 MB)",
                   "valuable_bytes_per_step": vb["total"], "valuable_bytes_paper_definition": vb_paper["total"],
                   "parallelism": f"replicas x{world}"},
        "kernels_ms": {"rhs_p1p1": round(statistics.mean(k_rhs), 4), "mass_p1p1": round(statistics.mean(k_mass), 4),
                       "interp_dg1": round(statistics.mean(k_int), 4)},
        "kernels_gbs": {"rhs_p1p1": round(vb["rhs"] / statistics.mean(k_rhs) / 1e6, 1),
                        "mass_p1p1": round(vb["mass"] / statistics.mean(k_mass) / 1e6, 1),
                        "interp_dg1": round(vb["interp"] / statistics.mean(k_int) / 1e6, 1)},
        "hbm_frac": {"interp_dg1": round(vb["interp"] / statistics.mean(k_int) / 1e6 / hbm, 4),
                     "step": round(value / world / hbm, 4), "peak_gbs": hbm, "peak_kind": hbm_kind},
        "roofline": {"kernel": "k_mass_p1 (RHS and mass action)", "bound": "alu",
                     "achieved": round(achieved_ops, 2), "peak": round(ops_peak, 2), "unit": "G FP64 ops/s",
                     "frac": round(achieved_ops / ops_peak, 4), "traffic": traffic,
                     "algorithmic": f"{MASS_OPS_PER_ITEM} FP64 ops ({MASS_FLOPS_PER_ITEM} flops) per "
                                    f"(column, level) item x {items} items per launch",
                     "achieved_tflops": round(MASS_FLOPS_PER_ITEM * items / (mass_ms * 1e-3) / 1e12, 4),
                     "peak_note": "2 FP64 FMA/clk/SM x 152 SMs x max SM clock (nominal 1.25 TFLOP/s)"},
        "e2e": None if e2e_ms is None else {
            "value": round(world * vb["total"] / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, L, args.cpu_seconds)
    return line


def load_traffic(kernel: str):
    """dram bytes per launch of `kernel` from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        return t.get(kernel)
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle baseline
def cpu_baseline(m, L, seconds: float, steps: int = 1):
    """The oracle (serial C, one core) on the first S base columns of the same
    workload, all layers; S grows until one pass takes about `seconds`/steps."""
    import oracle as O
    X_sp, X = O.coords(m.cells, m.xy, L)
    p1 = O.number(m.cells, m.nverts, L, P1_DELTA)
    dg = O.number(m.cells, m.nverts, L, DG1_DELTA)
    Xr = X.reshape(-1, 3)
    f = np.sin(Xr[:, 0]) * np.cos(Xr[:, 1]) * Xr[:, 2]
    x = meshgen.uniform_field(p1.ndofs, SEED + 10)
    b = np.zeros(p1.ndofs)
    y = np.zeros(p1.ndofs)
    out = np.zeros(dg.ndofs)

    def one(S):
        t = time.perf_counter()
        O.par_loop(O.K_MASS, m.cells, L, [(X_sp, X, 3, O.READ), (p1, f, 1, O.READ), (p1, b, 1, O.INC)], ncells=S)
        O.par_loop(O.K_MASS, m.cells, L, [(X_sp, X, 3, O.READ), (p1, x, 1, O.READ), (p1, y, 1, O.INC)], ncells=S)
        O.par_loop(O.K_INTERP, m.cells, L, [(p1, x, 1, O.READ), (dg, out, 1, O.WRITE)], ncells=S)
        return time.perf_counter() - t

    S = 256
    dt = one(S)
    target = seconds / max(1, steps)
    while dt < 0.25 * target and S < m.ncells:
        S = min(m.ncells, S * 4)
        dt = one(S)
    S = min(m.ncells, max(1, int(S * target / max(dt, 1e-9))))
    times = [one(S) for _ in range(steps)]
    t = min(times)
    # valuable bytes of the sample: the touched vertex columns, the S cell
    # columns of DG1 output, S map rows per map (each counted once)
    Vs = np.unique(m.cells[:S]).size
    vb = 2 * (40 * Vs * (L + 1) + 48 * S) + (8 * Vs * (L + 1) + 48 * S * L + 48 * S)
    return {"value": round(vb / t / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {S} of {m.ncells} base columns x {L} layers, all three loops, "
                      f"min of {steps} run(s), {t:.2f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    m = meshgen.tri_mesh(N_CFG2, seed=SEED, order="rcm")
    L = LAYERS_CFG2
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    cb = cpu_baseline(m, L, per_step * args.steps, steps=args.steps)
    C = m.ncells
    line = {
        "impl": "reference",
        "metric": "par_loop valuable HBM GB/s (P1xP1 RHS + mass action + DG1 interpolation, 100 layers, RCM)",
        "value": cb["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded perturbed structured triangulation, RCM)",
        "config": {"workload": f"extruded prisms: {C} base triangles x {L} layers, {args.order} base order, "
                               "P1xP1 RHS + P1xP1 mass action + DG1xDG1 interpolation (bounded sample)"},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_CFG2, help="base grid size (2 n^2 triangles)")
    ap.add_argument("--layers", type=int, default=LAYERS_CFG2)
    ap.add_argument("--order", choices=["rcm", "random"], default="rcm")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build_library_only()
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
