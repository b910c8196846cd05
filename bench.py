"""Throughput of the Bessel-antenna FDTD hot path on GB300.

One bench "step" is one full Yee time step of the whole hot path (H update +
CPML, H soft source, fluence, E update + CPML, E soft source) over the
256 x 256 x 128-cell single-beam workload (dx = lambda/20, theta = 10 deg,
l = 0, ring radius 100 cells, 16-cell CPML), FP32 fields with FP64 source
phases and FP64 fluence.  The same workload is also timed in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle (the
baseline) on a bounded sample of the same workload.  Under torchrun each
rank runs its own replica of the workload (weak scaling, no collective on the
data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDTD Gcell-updates/s FP32 vs FP64 at stated L2 error; % HBM roofline; adjoint s/step"

NOMINAL_HBM_GBS = 8000.0   # GB300 HBM3e, nominal

# The timed block of --steps steps is repeated until this much GPU time has
# passed (at least MIN_REPEATS times); the reported time is the median block.
MIN_TIMED_S = 1.0
MIN_REPEATS = 5
MAX_REPEATS = 100000

# DRAM bytes (read + write) per launch of a kernel on the 256x256x128 FP32
# workload, from one ncu capture of the kernel as it stands (summary and
# command in profiles/); None where no capture of the current kernel exists.
TRAFFIC: dict[str, float | None] = {"yee_h_cell": 307.85e6, "yee_e_cell": 545.41e6, "yee_tb2": None}
UNIT = "Gcell-updates/s"

# FP64 instructions per cell of each FP64 pass (the cell pass and its antenna
# pass) on the 256x256x128 workload after 600 steps
# (smsp__inst_executed_pipe_fp64.sum x 32 / cells from one ncu capture of the
# kernels as they stand; summary and command in profiles/).  The FP64 passes
# are bound by GB300's FP64 pipe: 2 FP64 instructions per SM per clock,
# whatever the number of active lanes of the warp instruction.
FP64_INST_PER_CELL: dict[str, float | None] = {"yee_h_cell + antenna_add": 14.25 + 0.19,
                                               "yee_e_cell + antenna_add": 44.34 + 0.19}
# Steps run on the FP64 grid before its tiles are tuned and timed: the FP64
# norm of the fluence term costs less on cells whose fields are still zero,
# so the first steps of a run are cheaper than the rest of it.
FP64_PRESTEPS = 400
FP64_INST_PER_SM_CLK = 2.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def psi_per_cell(w) -> float:
    """Mean number of CPML psi values per cell (H and E sides together):
    4 on the x shells (2 npml / nx of the cells), 4 on the y shells, and on
    z-walled grids 4 on the z shells (2 npml_z / nz)."""
    return (4.0 * (2 * w.npml / w.nx) + 4.0 * (2 * w.npml / w.ny)
            + 4.0 * (2 * getattr(w, "npml_z", 0) / w.nz))


def algorithmic_bytes_per_cell(w, elem_bytes: int) -> float:
    """Bytes one whole step must move per cell-update at the least: read and
    write E and H once (12 words), read and write the 8-byte fluence
    accumulator (16 B), read and write every CPML psi value on the shells."""
    return 12 * elem_bytes + 16 + 2 * elem_bytes * psi_per_cell(w)


def launches_per_block(variant: int, steps: int) -> int:
    """Kernel launches of `steps` steps: two per step for the two-pass
    variants, one per two steps for variant 7 (plus one two-pass step for an
    odd count), one per step otherwise."""
    if variant == 7:
        return steps // 2 + 2 * (steps % 2)
    return steps * (2 if 3 <= variant <= 5 else 1)


def pass_bytes_per_cell(w, variant: int, b: int) -> list[tuple[str, float]]:
    """(kernel, algorithmic bytes per cell) of each kernel of a step: the
    distinct values that kernel itself must read and write.  Variant 7
    advances two steps per launch: its figure is per launch, the method's
    one-step minimum for each of the two cell-updates (the fluence, fields
    and psi it actually moves once per launch are half of that).
      one pass:            E, H in and out, fluence in and out, all psi;
      H pass (3, 5):       E^n, H^{n-1/2} in, H^{n+1/2} out, H-side psi;
      E pass + fluence:    E^n, H^{n+1/2}, H^{n-1/2} in, E^{n+1} out,
                           fluence in and out, E-side psi;
      H pass + fluence (4): E^n, H^{n-1/2} in, H^{n+1/2} out, fluence in and
                           out, H-side psi;  E pass (4): E^n, H^{n+1/2} in,
                           E^{n+1} out, E-side psi."""
    psi = psi_per_cell(w)
    one = 12 * b + 16 + 2 * b * psi
    h = 9 * b + b * psi
    if variant <= 2:
        name = {0: "yee_step_fused", 1: "yee_step_tma", 2: "yee_step_tma (2 rows/thread)"}[variant]
        return [(name, one)]
    if variant == 3:
        return [("yee_h_pass", h), ("yee_e_pass (with fluence)", 12 * b + 16 + b * psi)]
    if variant == 4:
        return [("yee_hflu_tma", h + 16), ("yee_e_pass", 9 * b + b * psi)]
    if variant == 5:
        if b == 8:   # FP64: each pass is followed by its antenna pass (antenna_add), timed with it
            return [("yee_h_cell + antenna_add", h), ("yee_e_cell + antenna_add", 12 * b + 16 + b * psi)]
        return [("yee_h_cell", h), ("yee_e_cell", 12 * b + 16 + b * psi)]
    if variant == 7:
        return [("yee_tb2", 2 * one)]
    return [("yee_step_cell", one)]


def kernel_roofline(w, tile, pass_ms, steps, b, peak, cells):
    """Per-kernel achieved bandwidth (algorithmic bytes / CUDA-event duration)
    and the dominant (longest) kernel.  pass_ms[p] sums kernel p over `steps`
    steps (variant 7: over its steps / 2 launches)."""
    table = pass_bytes_per_cell(w, tile[0], b)
    launches = steps // 2 if tile[0] == 7 else steps
    rows = []
    for (name, bpc), ms in zip(table, pass_ms):
        t = ms / launches
        ach = bpc * cells / (t * 1e-3) / 1e9
        rows.append({"kernel": name, "ms_per_launch": round(t, 5), "algorithmic_bytes_per_cell": round(bpc, 3),
                     "achieved_gbs": round(ach, 1), "frac": round(ach / peak, 4)})
    dom = max(rows, key=lambda r: r["ms_per_launch"])
    return rows, dom


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The slowest rank's time: every rank times its own replica; the job
    takes as long as the slowest one."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank: int, steps: int, ws: int, ms: float) -> float:
    """Whole-job Gcell-updates/s: the cell-updates of all ranks' replicas
    over the (max-over-ranks) time."""
    return cells_per_rank * steps * ws / (ms * 1e-3) / 1e9


def run_gpu(args):
    import torch
    import numpy as np
    from paper_2102_12978_gb300 import fdtd
    from paper_2102_12978_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def _barrier():
        barrier(ws)

    w = W.config2()
    cells = w.cells

    def make(prec):
        d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant,
                                precision=prec, fluence=True)
        g = fdtd.Grid(d, device=dev)
        g.set_source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness,
                     ramp=w.ramp)
        return g

    def timed(g, steps, warmup):
        """Median CUDA-event time of one block of `steps` steps: the block is
        repeated until at least MIN_TIMED_S of GPU time has passed (and at
        least MIN_REPEATS times), so that the clock sampler sees the load.
        Returns (max over ranks of the median ms, repeats, total timed ms)."""
        stream = g.stream
        g.step(warmup)
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = []
        while (sum(reps) < MIN_TIMED_S * 1e3 or len(reps) < MIN_REPEATS) and len(reps) < MAX_REPEATS:
            e0.record(stream)
            g.step(steps)
            e1.record(stream)
            e1.synchronize()
            reps.append(e0.elapsed_time(e1))
        torch.cuda.synchronize(dev)
        barrier(ws)
        return max_over_ranks(statistics.median(reps), ws, dev), len(reps), sum(reps)

    peak, peak_kind = _peaks()

    if args.only == "bessel_gauss":
        # profiling run: the Bessel-Gauss box, optionally shrunk, FP32
        wb = W.bessel_gauss()
        s = max(1, args.bg_shrink)
        wb = wb.scaled(nx=wb.nx // s, ny=wb.ny // s, nz=wb.nz // s, w0=wb.w0 / s)
        d = fdtd.make_grid_desc(wb.nx, wb.ny, wb.nz, wb.npml, wb.dx, wb.dx, wb.dz, courant=wb.courant,
                                precision="f32", fluence=True, z_walls=True, npml_z=wb.npml_z)
        g = fdtd.Grid(d, device=dev)
        g.set_wall_source(theta=wb.theta, w0=wb.w0, E0=wb.E0, envelope=wb.envelope, T=wb.T, T0=wb.T0,
                          plane=wb.plane)
        g.step(args.warmup)
        g.step(args.steps)
        g.sync()
        print(json.dumps({"only": "bessel_gauss", "grid": [wb.nx, wb.ny, wb.nz], "steps": args.steps,
                          "tile": list(g.tile())}))
        return

    if args.only != "all":
        g = make(args.only)
        if args.tile:
            g.set_tile(*[int(x) for x in args.tile.split(",")])
        if args.balance:
            apply_balance(g, [float(x) for x in args.balance.split(",")])
        g.step(args.warmup)
        g.step(args.steps)
        g.sync()
        print(json.dumps({"only": args.only, "steps": args.steps, "tile": list(g.tile())}))
        return

    # ---- FP32 (headline) ---------------------------------------------------
    g32 = make("f32")
    tile32 = g32.autotune(steps=60)   # 60 steps per candidate: the refined ranges differ by ~1 %
    balance32 = g32.balance()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    # variant 7 times its launches over an even number of steps
    steps_k = args.steps + (args.steps % 2 if tile32[0] == 7 else 0)
    with ClockSampler(gpu_id) as clk:
        ms32, reps32, timed_ms32 = timed(g32, args.steps, args.warmup)
        # the same steps again with CUDA events around every kernel launch
        # (each kernel's duration for the per-kernel rooflines)
        pass32 = g32.step_timed(steps_k)
    clocks = clk.summary()
    step_ms = ms32 / args.steps
    gcell32 = job_rate(cells, args.steps, ws, ms32)
    ab32 = algorithmic_bytes_per_cell(w, 4)
    step_achieved = ab32 * cells / (step_ms * 1e-3) / 1e9
    passes32, dom32 = kernel_roofline(w, tile32, pass32, steps_k, 4, peak, cells)
    traffic32 = step_traffic(tile32[0])

    # ---- FP64 (secondary) --------------------------------------------------
    g64 = make("f64")
    g64.step(FP64_PRESTEPS)
    tile64 = g64.autotune(steps=8)
    steps64 = max(10, args.steps // 4)
    ms64, reps64, _ = timed(g64, steps64, max(3, args.warmup // 4))
    pass64 = g64.step_timed(steps64)
    gcell64 = job_rate(cells, steps64, ws, ms64)
    ab64 = algorithmic_bytes_per_cell(w, 8)
    achieved64 = ab64 * cells / (ms64 / steps64 * 1e-3) / 1e9
    passes64, dom64 = kernel_roofline(w, tile64, pass64, steps64, 8, peak, cells)
    # the FP64 pipe roofline of the dominant FP64 kernel, against the FP64
    # FMA rate measured on this device (8 independent chains per thread,
    # 2048 threads per SM); the nominal rate beside it
    with ClockSampler(gpu_id) as clk64:
        fp64_rate, fp64_rate_ms = fdtd.measure_fp64_rate(chains=8, iters=60000)
    fp64_dep, _ = fdtd.measure_fp64_rate(chains=1, iters=20000)
    clocks64 = clk64.summary()
    sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fp64_nominal = props.multi_processor_count * FP64_INST_PER_SM_CLK * sm_mhz * 1e6 / 1e9   # G inst/s
    fp64_peak = fp64_rate / 1e9
    ipc = FP64_INST_PER_CELL.get(dom64["kernel"]) if tile64[0] == 5 else None
    fp64_alu = None
    if ipc is not None:
        ach = ipc * cells / (dom64["ms_per_launch"] * 1e-3) / 1e9
        fp64_alu = {"bound": "alu", "kernel": dom64["kernel"], "unit": "G fp64 inst/s", "achieved": round(ach, 1),
                    "peak": round(fp64_peak, 1), "frac": round(ach / fp64_peak, 4), "fp64_inst_per_cell": ipc,
                    "peak_kind": "measured: FP64 FMA microbenchmark (fdtd_measure_fp64_rate, 8 independent "
                                 f"chains x 2048 threads per SM, {fp64_rate_ms:.1f} ms)",
                    "peak_clocks": clocks64,
                    "dependent_chain_rate": round(fp64_dep / 1e9, 1),
                    "peak_nominal": round(fp64_nominal, 1),
                    "peak_nominal_from": f"{props.multi_processor_count} SMs x {FP64_INST_PER_SM_CLK:g} FP64 "
                                         f"inst/clk x {sm_mhz:g} MHz"}

    # FP32 against FP64 on the GPU over the workload's full run (both GPU
    # paths are parity-checked against the oracle in the test suite; FP64 is
    # the transfer standard at full length)
    l2_error = full_length_error(torch, make, w.steps if args.error_steps < 0 else args.error_steps, tile32,
                                 balance32)

    # ---- end to end through the public API with host buffers --------------
    e2e = run_e2e(torch, fdtd, w, dev, args.steps, _barrier, ws, tile32, balance32)

    # ---- batched sweep: 16 uneven grids advanced together ----------------
    batched = run_batched(torch, fdtd, W, dev, args.batch_steps) if args.batch_steps > 0 else None

    # ---- adjoint: 384x384x96 FP32 reverse steps ---------------------------
    adjoint = run_adjoint(torch, fdtd, W, dev, args.adjoint_steps) if args.adjoint_steps > 0 else None

    # ---- the Bessel-Gauss box of Section 2 (z walls, wall sheet) -----------
    bessel_gauss = (run_bessel_gauss(torch, fdtd, W, dev, args.bg_steps, peak)
                    if args.bg_steps > 0 else None)

    del g32, g64
    out = {
        "metric": METRIC, "value": round(gcell32, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "cells": cells, "grid": [w.nx, w.ny, w.nz], "npml": w.npml,
                   "dx_lambda": w.dx, "theta_deg": w.theta_deg, "m": w.m, "ring_radius_cells": w.r_center,
                   "fluence": "fp64", "source_phase": "fp64",
                   "l2_flush": "inputs larger than L2 (fields + fluence = %.0f MB/step)"
                               % (ab32 * cells / 1e6),
                   "tile_f32": list(tile32), "balance_f32": ("ranges refined on measured per-CTA times" if balance32[0] < 0
                                                  else [round(x, 3) for x in balance32]),
                   "tile_f64": list(tile64), "parallelism": f"replicas{ws}",
                   "timing": f"median of {reps32} repeats of the {args.steps}-step block (>= {MIN_TIMED_S:g} s "
                             f"of GPU time)"},
        "roofline": {"bound": "hbm", "achieved": round(step_achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_achieved / peak, 4), "traffic": traffic32,
                     "traffic_gbs": (round(traffic32 / (step_ms * 1e-3) / 1e9, 1)
                                     if traffic32 is not None else None),
                     "basis": "whole step: the method's bytes per cell-update (E, H, fluence, CPML psi in and "
                              "out once) x cells / ms_per_step; traffic = DRAM bytes per step (ncu); "
                              "traffic_gbs = traffic / ms_per_step",
                     "algorithmic_bytes_per_cell_update": ab32, "cell_updates_per_step": cells,
                     "peak_kind": peak_kind, "peak_nominal": NOMINAL_HBM_GBS,
                     "frac_nominal": round(step_achieved / NOMINAL_HBM_GBS, 4),
                     "dominant_kernel": dom32["kernel"], "kernels": passes32},
        "fp64": {"value": round(gcell64, 3), "unit": UNIT, "steps": steps64,
                 "ms_per_step": round(ms64 / steps64, 5), "tile": list(tile64),
                 "timed_after_steps": FP64_PRESTEPS,
                 "roofline": {"bound": "alu", "kernels": passes64, "dominant": dom64["kernel"],
                              "fp64_pipe": fp64_alu,
                              "step_achieved_gbs": round(achieved64, 1),
                              "step_frac_of_hbm": round(achieved64 / peak, 4),
                              "algorithmic_bytes_per_cell": ab64}},
        "l2_error": l2_error,
        "e2e": e2e,
        "batched": batched,
        "adjoint": adjoint,
        "bessel_gauss": bessel_gauss,
        "gpu_launches": reps32 * launches_per_block(tile32[0], args.steps),
        "timed_repeats": reps32, "timed_gpu_s": round(timed_ms32 * 1e-3, 3),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def step_traffic(variant: int):
    """DRAM bytes per step from the ncu captures in TRAFFIC (per launch):
    the sum over a step's kernels, half a launch of variant 7; None when a
    kernel of the step has no capture."""
    kernels = {5: ["yee_h_cell", "yee_e_cell"], 7: ["yee_tb2"]}.get(variant)
    if not kernels or any(TRAFFIC.get(k) is None for k in kernels):
        return None
    t = sum(TRAFFIC[k] for k in kernels)
    return round(t / 2 if variant == 7 else t)


def rel_l2_t(torch, x, y) -> float:
    x = x.double(); y = y.double()
    den = float(torch.linalg.vector_norm(y))
    return float(torch.linalg.vector_norm(x - y)) / den if den > 0 else float(torch.linalg.vector_norm(x))


def apply_balance(g, balance):
    """The variant-7 balance the autotuner chose: weights, or (-1, -1) for
    ranges refined on measured per-CTA times (refined again on g; the grid's
    antenna must be set)."""
    if balance[0] < 0:
        g.measure_balance()
    else:
        g.set_balance(*balance)


def full_length_error(torch, make, steps, tile32, balance32):
    """Relative L2 of the FP32 fields and fluence against the FP64 GPU run
    after `steps` steps of the workload (its full run by default), per field
    component and for the fluence, in the bench's FP32 launch configuration."""
    a = make("f32")
    a.set_tile(*tile32)
    apply_balance(a, balance32)
    b = make("f64")
    a.step(steps)
    b.step(steps)
    per = {}
    for c, name in enumerate(("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")):
        per[name] = rel_l2_t(torch, a.field(c), b.field(c))
    per["fluence"] = rel_l2_t(torch, a.fluence(), b.fluence())
    num = den = 0.0
    for c in range(6):
        x = a.field(c).double(); y = b.field(c)
        num += float(torch.sum((x - y) ** 2)); den += float(torch.sum(y ** 2))
    a.close(); b.close()
    return {"f32_vs_f64_gpu": {k: float(f"{v:.3e}") for k, v in per.items()},
            "f32_vs_f64_gpu_rel_l2_fields": float(f"{(num / den) ** 0.5:.3e}"), "after_steps": steps,
            "f64_vs_oracle_tol": 1e-11, "f32_vs_oracle_tol": 1e-4}


def run_batched(torch, fdtd, W, dev, steps):
    """The 16-configuration sweep (l in 0..3 x theta in 5, 10, 20, 30 deg,
    N^2 x 64 grids with N = 96 .. 640), all grids advanced together: the
    graph engine with every grid on the cell passes (its default), the
    persistent cell engine (one cooperative launch per 64 steps), and the
    batch as fdtd_batch_autotune leaves it (each grid's mode, then the
    engine).  Against the same grids stepped one grid at a time, with the
    default tile and with each grid's tuned tile."""
    ws_ = W.config4()

    def make(wl):
        d = fdtd.make_grid_desc(wl.nx, wl.ny, wl.nz, wl.npml, wl.dx, wl.dx, wl.dz, courant=wl.courant,
                                precision="f32", fluence=True)
        g = fdtd.Grid(d, device=dev)
        g.set_source(m=wl.m, theta=wl.theta, pol=wl.pol, r_center=wl.r_center, thickness=wl.thickness,
                     ramp=wl.ramp)
        return g

    cells = sum(wl.cells for wl in ws_)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)

    def sequential(tiles):
        seq = [make(wl) for wl in ws_]
        for g, t in zip(seq, tiles):
            if t is not None:
                g.set_tile(*t)
        for g in seq:
            g.step(2)
        torch.cuda.synchronize(dev)
        stream = seq[0].stream
        e0.record(stream)
        for _ in range(steps // 2):
            for g in seq:
                g.step(2)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        for g in seq:
            g.close()
        return ms

    def batched(engine=None, tune=False):
        bat = [make(wl) for wl in ws_]
        b = fdtd.Batch(bat, engine=engine)
        tuned = b.autotune(steps=8) if tune else None
        if tune:
            tuned = (*tuned, [b.grid_ctas(q) for q in range(len(bat))])
        b.step(64)                 # warm-up, builds the graph
        b.sync()
        e0.record(bat[0].stream)
        b.step(steps)
        e1.record(bat[0].stream)
        torch.cuda.synchronize(dev)
        b.sync()
        ms = e0.elapsed_time(e1)
        b.close()
        for g in bat:
            g.close()
        return ms, tuned

    ms_seq = sequential([None] * len(ws_))
    ms_cell, _ = batched(fdtd.BATCH_CELL)
    ms_pc, _ = batched(fdtd.BATCH_PERSISTENT_CELL)
    ms_tuned, (engine, modes, ctas) = batched(tune=True)
    mode_tile = {0: (5, 4, 1), 1: (5, 8, 1), 2: (5, 16, 1), 3: (7, 16, 1)}
    ms_seq_tuned = sequential([mode_tile[m] for m in modes])
    rate = lambda ms: round(cells * steps / (ms * 1e-3) / 1e9, 3)
    return {"value": rate(ms_tuned), "unit": UNIT, "engine": "graph" if engine == fdtd.BATCH_CELL else "persistent_cell",
            "grid_modes": {wl.name: ["cell4", "cell8", "cell16", "two_step"][m] for wl, m in zip(ws_, modes)},
            "two_step_ctas": {wl.name: c for wl, m, c in zip(ws_, modes, ctas) if m == 3},
            "tuned_by": "fdtd_batch_autotune (each grid's mode alone, then the engine over the batch)",
            "cell_value": rate(ms_cell), "persistent_cell_value": rate(ms_pc),
            "sequential_value": rate(ms_seq), "sequential_tuned_tiles_value": rate(ms_seq_tuned),
            "speedup_vs_sequential": round(ms_seq / ms_tuned, 3),
            "speedup_vs_sequential_same_kernels": round(ms_seq_tuned / ms_tuned, 3),
            "grids": len(ws_), "cells": cells, "steps": steps,
            "ms_per_step": round(ms_tuned / steps, 4), "sequential_ms_per_step": round(ms_seq / steps, 4)}


def run_bessel_gauss(torch, fdtd, W, dev, steps, peak):
    """Section 2's Bessel-Gauss box (411 x 411 x 738 cells with the CPML, z
    walls, the Gaussian-axicon E_x sheet), FP32 on the cell passes: `steps`
    of its 3635 steps timed with CUDA events (the fields and fluence, 7.6 GB,
    exceed L2), then the same number with events around each kernel."""
    w = W.bessel_gauss()
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant,
                            precision="f32", fluence=True, z_walls=True, npml_z=w.npml_z)
    g = fdtd.Grid(d, device=dev)
    g.set_wall_source(theta=w.theta, w0=w.w0, E0=w.E0, envelope=w.envelope, T=w.T, T0=w.T0, plane=w.plane)
    g.step(5)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(steps)
    e1.record(g.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    pass_ms = g.step_timed(steps)
    rows, dom = kernel_roofline(w, g.tile(), pass_ms, steps, 4, peak, w.cells)
    for r in rows:   # z-walled grids run the *_w instantiations of the cell passes
        r["kernel"] += "_w"
    out = {"workload": w.name, "cells": w.cells, "grid": [w.nx, w.ny, w.nz], "npml": w.npml,
           "npml_z": w.npml_z, "theta_deg": w.theta_deg, "w0_lambda": w.w0, "steps_timed": steps,
           "steps_full_run": w.steps, "value": round(job_rate(w.cells, steps, 1, ms), 3), "unit": UNIT,
           "ms_per_step": round(ms / steps, 5),
           "full_run_s": round(ms / steps * w.steps / 1e3, 3), "dtype": "f32", "tile": list(g.tile()),
           "kernels": rows, "dominant": dom["kernel"], "dominant_frac": dom["frac"]}
    del g
    torch.cuda.empty_cache()
    return out


def run_adjoint(torch, fdtd, W, dev, steps):
    """Seconds per reverse (adjoint) step and per forward step on the
    384 x 384 x 96 FP32 adjoint workload (3-cell ring, 16-cell CPML); one
    checkpointed gradient costs a forward, a recomputing forward and an
    adjoint step per step."""
    import numpy as np
    wl = W.config5()
    d = fdtd.make_grid_desc(wl.nx, wl.ny, wl.nz, wl.npml, wl.dx, wl.dx, wl.dz, courant=wl.courant,
                            precision="f32", fluence=False)
    g = fdtd.Grid(d, device=dev)
    g.set_source(m=wl.m, theta=wl.theta, pol=wl.pol, r_center=wl.r_center, thickness=wl.thickness,
                 ramp=wl.ramp)
    g.autotune(steps=3)
    g.step(steps + 8)
    i = np.arange(wl.nx)[None, :]
    j = np.arange(wl.ny)[:, None]
    r0 = 0.383 / np.sin(wl.theta) / wl.dx
    cols = np.flatnonzero((np.hypot(i - wl.nx / 2, j + 0.5 - wl.ny / 2) < 3 * r0).ravel())
    probes = (np.arange(wl.nz)[:, None] * (wl.nx * wl.ny) + cols[None, :]).ravel()
    adj = fdtd.Adjoint(g, fdtd.EY, probes)
    adj.reset(g.n)
    stream = g.stream
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    adj.step(4)
    torch.cuda.synchronize(dev)
    e0.record(stream); adj.step(steps); e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_adj = e0.elapsed_time(e1) / steps
    e0.record(stream); g.step(steps); e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_fwd = e0.elapsed_time(e1) / steps
    adj.close(); g.close()
    # one whole gradient over the workload's 5000 steps: the autograd forward
    # (checkpoints every 250 steps, the steps before the 250-step loss window on
    # the two-step kernel) and backward (segment replays and reverse steps)
    from paper_2102_12978_gb300.adjoint import BeamProblem, beam_loss
    tgt = torch.ones(probes.size, dtype=torch.float64, device=dev)
    src = dict(m=wl.m, theta=wl.theta, pol=wl.pol, r_center=wl.r_center, thickness=wl.thickness, ramp=wl.ramp)
    prob = BeamProblem(d, src, fdtd.EY, probes, tgt, wl.steps, 250, 250, tile=(7, 16, 1))
    wa = torch.ones((wl.ny, wl.nx), dtype=torch.float64, requires_grad=True)
    wp = torch.zeros((wl.ny, wl.nx), dtype=torch.float64, requires_grad=True)
    prob.context()
    grad_runs = []
    for _ in range(2):   # the first call also makes the checkpoints' device buffers
        wa.grad = None
        wp.grad = None
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        beam_loss(wa, wp, prob).backward()
        torch.cuda.synchronize(dev)
        grad_runs.append(time.perf_counter() - t0)
    grad_s = grad_runs[-1]
    return {"s_per_step": round(ms_adj * 1e-3, 7), "forward_s_per_step": round(ms_fwd * 1e-3, 7),
            "gradient_s_per_step": round(grad_s / wl.steps, 7), "gradient_s": round(grad_s, 3),
            "gradient_first_call_s": round(grad_runs[0], 3),
            "gradient_steps": wl.steps, "gradient_what": "one autograd forward + backward over all 5000 steps "
                                                          "(wall clock, host included; the second of two "
                                                          "calls, the first beside it)",
            "grid": [wl.nx, wl.ny, wl.nz],
            "probes": int(probes.size), "steps_timed": steps, "dtype": "f32",
            "adjoint_gcell_per_s": round(wl.cells / (ms_adj * 1e-3) / 1e9, 3)}


def run_e2e(torch, fdtd, w, dev, steps, barrier, ws, tile, balance):
    """Whole job through the public API with host buffers: the initial state
    (6 field arrays) and the source description go host -> device, `steps`
    Yee steps run (in the tile configuration the autotuner chose), and the
    fluence plus the dominant field come back to pinned host memory, all
    inside the timed region."""
    import numpy as np
    shape = (w.nz, w.ny, w.nx)
    init = [torch.zeros(shape, dtype=torch.float32).pin_memory() for _ in range(6)]
    flu_h = torch.empty(shape, dtype=torch.float64).pin_memory()
    fld_h = torch.empty(shape, dtype=torch.float32).pin_memory()
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant,
                            precision="f32", fluence=True)
    g = fdtd.Grid(d, device=dev)
    g.set_tile(*tile)
    if balance[0] < 0:   # measured costs: measured with the antenna the timed region sets again
        g.set_source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness, ramp=w.ramp)
    apply_balance(g, balance)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for c in range(6):
        fdtd.fdtd_set_field(g.handle, c, init[c].data_ptr(), False)
    g.set_source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness, ramp=w.ramp)
    g.step(steps)
    fdtd.fdtd_fluence(g.handle, flu_h.data_ptr(), False, False)
    fdtd.fdtd_get_field(g.handle, 1 if w.pol == "y" else 0, fld_h.data_ptr(), False)
    torch.cuda.synchronize(dev)
    barrier()
    dt = max_over_ranks((time.perf_counter() - t0) * 1e3, ws, dev) * 1e-3
    h2d = 6 * init[0].numel() * 4 + (16 * 6 + 1) * w.nx * w.ny + 32 * w.nz
    d2h = flu_h.numel() * 8 + fld_h.numel() * 4
    g.close()
    return {"value": round(w.cells * steps * ws / dt / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / steps, 1), "d2h_bytes_per_step": round(d2h / steps, 1),
            "seconds": round(dt, 4),
            "what": "host state + source description in, K steps, fluence + E_pol out (pinned host)"}


def cpu_baseline(w, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the same workload: the full 256x256x128 grid with its antenna, for as many
    steps as fit in about `budget_s` seconds on all cores, then one step on
    one thread."""
    import oracle
    og = oracle.Grid(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant)
    os_ = oracle.Source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness,
                        ramp=w.ramp)
    st = oracle.State(og)
    cores = oracle.threads()
    oracle.run(og, os_, st, 1)                  # antenna build + first step
    t0 = time.perf_counter()
    oracle.run(og, os_, st, 1)                  # calibration step
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(og, os_, st, n)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.run(og, os_, st, 1)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": round(w.cells * n / dt / 1e9, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": round(w.cells / dt1 / 1e9, 5),
            "sample": f"{n} steps of the full {w.nx}x{w.ny}x{w.nz} workload (FP64 C, OpenMP), "
                      f"{dt:.1f} s on {cores} threads; 1 step on 1 thread, {dt1:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2102_12978_gb300 import workloads as W
    import oracle
    w = W.config2()
    og = oracle.Grid(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant)
    os_ = oracle.Source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness,
                        ramp=w.ramp)
    st = oracle.State(og)
    # each reference "step" is one oracle Yee step of the full workload
    oracle.run(og, os_, st, max(1, min(args.warmup, 3)))
    n = max(1, min(args.steps, 20))
    t0 = time.perf_counter()
    oracle.run(og, os_, st, n)
    dt = time.perf_counter() - t0
    cores = oracle.threads()
    v = w.cells * n / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": ws,
        "steps": n, "warmup": args.warmup, "ms_per_step": round(dt / n * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "cells": w.cells},
        "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} steps of the full workload, {dt:.1f} s"},
        "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--only", default="all", choices=["all", "f32", "f64", "bessel_gauss"],
                    help="time only one precision (profiling runs)")
    ap.add_argument("--tile", default=None, help="variant,ty,lz for --only runs")
    ap.add_argument("--balance", default=None, help="w_shell,w_antenna (variant 7 work split) for --only runs")
    ap.add_argument("--batch-steps", type=int, default=128,
                    help="steps of the 16-grid batched sweep (0 skips it)")
    ap.add_argument("--bg-steps", type=int, default=200,
                    help="steps of the Bessel-Gauss box timed (0: skip)")
    ap.add_argument("--bg-shrink", type=int, default=1,
                    help="--only bessel_gauss: divide the box's nx, ny, nz by this (profiling runs)")
    ap.add_argument("--error-steps", type=int, default=-1,
                    help="steps of the FP32-vs-FP64 comparison (default: the workload's full run)")
    ap.add_argument("--adjoint-steps", type=int, default=100,
                    help="reverse steps timed on the adjoint workload (0 skips it)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
