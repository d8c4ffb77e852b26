#!/usr/bin/env python3
"""Throughput of the SIMPLE-TS time step (arXiv:1802.04243) on GB300.

One benchmark step = one time step of the whole hot path: loop-2 iterations
of face densities, energy, pseudo velocities, pressure, velocity correction,
equation of state and residual reduction (plus the explicit convective terms
for the explicit scheme).  The default workload is the paper-scale channel:
4864 x 1216 cells (5.9 M control volumes, the size the paper fits in 1 GB,
Section 5) with one square obstacle, implicit upwind, Mach 2, Re 300, 2
loop-2 iterations per step; `value` is its FP64 throughput and the same line
carries the mixed-precision and double-float runs of the same workload with
their error against FP64.  Metric: Mcell-steps/s = nx * ny * steps / second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision fp64|mixed|df64] [--only-main]

Under torchrun (N > 1) every rank advances its own replica of the channel
(the method needs no exchange between independent problems): weak scaling.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s FP64 vs FP32/FP64 mixed at stated error; % of HBM roofline"
UNIT = "Mcell-steps/s"

# The dominant kernel of every FP64 scheme, k_assemble, is bound by GB300's
# FP64 pipe.  Its work per cell and loop-2 iteration is the number of FP64
# arithmetic thread instructions (DFMA, DADD, DMUL) ncu counts on one launch,
# divided by the cells of that launch; its DRAM traffic per cell likewise
# (dram__bytes_read.sum + dram__bytes_write.sum).  Each entry names the case
# it was counted on; the bench scales it by the cells of its own workload.
# The commands are in profiles/.
_C4HALF = "2432x608 channel (the 4864x1216 channel at half resolution, 1,478,656 cells)"
ASSEMBLE_FP64_COUNTS = {
    "implicit-upwind": {"dfma": 51.15, "dadd": 43.90, "dmul": 33.52, "dram_bytes": 223.3, "fp64_pipe": 0.865,
                        "case": _C4HALF},
    "implicit-tvd": {"dfma": 66.88, "dadd": 43.90, "dmul": 33.52, "dram_bytes": 281.8, "fp64_pipe": 0.873,
                     "case": _C4HALF},
    "explicit-upwind": {"dfma": 41.31, "dadd": 25.21, "dmul": 37.45, "dram_bytes": 214.1, "fp64_pipe": 0.860,
                        "case": _C4HALF},
    "explicit-tvd": {"dfma": 41.31, "dadd": 25.21, "dmul": 37.45, "dram_bytes": 214.1, "fp64_pipe": 0.860,
                     "case": _C4HALF},
}
# Algorithmic HBM bytes of k_assemble per cell: the previous iterate's u, v,
# p, T, rho, Gamma, level n-1's u, v, T, rho, and the face arrays F^x, F^y,
# D^T_x, D^T_y, B Gamma (corner) and its two control-volume conductances,
# B Gamma dy/dx, B Gamma dx/dy, the two cell-centre mass fluxes, the two cell
# pair sums and rho^u dy, rho^v dx (25 doubles read); T, u^, d^u, v^, d^v and
# the pressure equation's face terms a^px, a^py, b^px, b^py written (9
# doubles).
ASSEMBLE_BYTES_PER_CELL = 34 * 8
# Algorithmic HBM bytes of the method per cell (the sweep's own minimum with
# perfect neighbour reuse): each loop-2 iteration reads u, v, p, T of the
# previous iterate and of level n-1 and writes u, v, p, T (12 doubles); the
# explicit scheme reads its three explicit terms as well (15 doubles) and
# computes them once per step from 4 reads and 3 writes (7 doubles).
def method_bytes_per_step(case) -> int:
    per_iter = 15 * 8 if not case.implicit else 12 * 8
    return case.cells * (case.iters * per_iter + (0 if case.implicit else 7 * 8))


# GB300 FP64 pipe: 2 FP64 thread instructions per cycle per SM (ncu's
# peak_sustained for DFMA), 152 SMs.
FP64_INST_PER_CYCLE_PER_SM = 2


def hbm_peak_gbs() -> float:
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batched measurement")
    ap.add_argument("--batch-steps", type=int, default=40)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c4",
                    help="c4 (default: the paper-scale 4864x1216 channel, the benchmark line); the others "
                         "are for profiling and sweeps")
    ap.add_argument("--precision", choices=["fp64", "mixed", "df64"], default="fp64",
                    help="arithmetic of the main timed run (default fp64, the bench value)")
    ap.add_argument("--only-main", action="store_true",
                    help="time the main run only (no per-kernel pass, no other precisions, no e2e, batch or "
                         "CPU baseline): the command the profiler captures")
    ap.add_argument("--sweep", choices=["paper", "plans"], default=None,
                    help="paper: the paper's experiment (Section 4) -- the four schemes on the 4032 x "
                         "{200, 400, 2000, 4000} meshes with 1, 2, 10, 20 particles, FP64, against the "
                         "oracle on one core, and the tile-height sweep that stands in for its rows per "
                         "work-group; plans: every work distribution of the equation kernels (tile shape, "
                         "CTA count) on --workload for each precision")
    return ap.parse_args()


def _c4_half(W):
    """The paper-scale channel at half resolution (2432x608, square of side
    152 at a quarter of the length): the C4 geometry on a case small enough
    for a detailed profiler capture, with a state (about 0.6 GB FP64) well
    above L2."""
    return W.channel(2432, 608, 152, name="c4half_2432x608_implicit_upwind", mach_in=2.0, reynolds=300.0,
                     implicit=True, tvd=False, seed=4, steps=2000)


_SCHEMES = {"implicit-upwind": (True, False), "implicit-tvd": (True, True), "explicit-upwind": (False, False),
            "explicit-tvd": (False, True)}


def _with_scheme(case, scheme):
    implicit, tvd = _SCHEMES[scheme]
    name = case.name.rsplit("_", 2)[0] + "_" + scheme.replace("-", "_")
    return case.replace(implicit=implicit, tvd=tvd, name=name)


WORKLOADS = {
    "c2": lambda W: W.c2_medium(),
    "c3": lambda W: W.c3_large(implicit=True),
    "c3-explicit": lambda W: W.c3_large(implicit=False),
    "c4": lambda W: W.c4_paper_scale(),
    "profile": lambda W: W.profile_channel(),
    "c2-implicit-tvd": lambda W: W.c2_medium().replace(tvd=True, name="c2_1024x256_implicit_tvd"),
    "c2-explicit-upwind": lambda W: W.c2_medium().replace(implicit=False, name="c2_1024x256_explicit_upwind"),
    "c2-explicit-tvd": lambda W: W.c2_medium().replace(implicit=False, tvd=True, name="c2_1024x256_explicit_tvd"),
    "paper": lambda W: W.paper_channel(ny=400),
    "paper-4000": lambda W: W.paper_channel(ny=4000),
    **{f"c4-{s}": (lambda s: lambda W: _with_scheme(W.c4_paper_scale(), s))(s) for s in _SCHEMES if s != "implicit-upwind"},
    **{f"c4half-{s}": (lambda s: lambda W: _with_scheme(_c4_half(W), s))(s) for s in _SCHEMES},
}
_ARGS = None


def workload():
    import workloads as W
    return WORKLOADS[_ARGS.workload if _ARGS else "c4"](W)


def small_case():
    import workloads as W
    return W.c1_small()


def device_bytes_of(make):
    """(object, device bytes its creation took): the drop in the driver's
    free-memory count around make(), which allocates through cudaMalloc."""
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    obj = make()
    torch.cuda.synchronize()
    return obj, free0 - torch.cuda.mem_get_info()[0]


def config_of(case):
    """The workload description, identical in both arms of the benchmark."""
    scheme = ("implicit" if case.implicit else "explicit") + ("-tvd" if case.tvd else "-upwind")
    state_mb = case.cells * 3 * 6 * 8 / 1e6       # three FP64 levels of six fields
    l2 = ("state larger than L2" if state_mb > 126 else "state smaller than L2") + \
         f" ({state_mb:.0f} MB of FP64 levels vs 126 MB); the GPU arm also writes 256 MB between timed steps"
    return {"workload": f"{case.name}: {case.nx}x{case.ny} channel, {len(case.rects)} square obstacle(s), "
                        f"{scheme}, Mach {case.mach_in}, Re {case.reynolds:g}, "
                        f"{case.iters} loop-2 iterations per step",
            "nx": case.nx, "ny": case.ny, "cells": case.cells, "scheme": scheme,
            "loop2_iters": case.iters, "l2": l2}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------ cross-rank helpers

def reduce_max(x: float, dist, device) -> float:
    """Maximum of a per-rank value over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(cells: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job Mcell-steps/s: every rank advances its own replica of `cells`."""
    return cells * steps * world / seconds / 1e6


def timed_steps(sim_obj, steps, stream, flush, starts, ends):
    """Time `steps` single time steps with CUDA events on `stream`, writing a
    buffer larger than L2 before each step (outside the events); returns ms."""
    import torch
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        sim_obj.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts[:steps], ends[:steps]))


# ------------------------------------------------------------------ batches

def run_batch(args, stream):
    """64 independent channels of uneven size (256x64 .. 2048x512), mixed
    precision, advanced together with the autotuned work distribution (tile
    shape and CTA count of the per-phase kernels in a CUDA graph per step, or
    one persistent cooperative kernel per step); both forms are also timed at
    the tuned tile shape.  Compared with the same problems stepped one after
    another, and with an FP64 batch for the error."""
    import numpy as np
    import torch

    import paper_1802_04243_gb300 as sim
    import workloads as W
    cases = W.c5_batch(64, precision=W.MIXED)
    cells = sum(c.cells for c in cases)
    steps = max(1, min(args.batch_steps, args.steps))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(step_all):
        ms = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            e0.record(stream)
            step_all()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms

    b = sim.Batch(cases, stream=stream.cuda_stream)
    b.tune()
    plan = b.plan_info()
    for _ in range(args.warmup):
        b.step(1)
    batch_ms = timed(lambda: b.step(1))
    mixed_fields = [b.fields(q) for q in range(len(cases))]
    b.close()

    # the two step forms at the tuned tile shape, each timed: one launch per
    # phase in a captured graph, and one persistent cooperative kernel per step
    forms = {}
    for name, persistent in (("per_phase", False), ("persistent", True)):
        with sim.Batch(cases, stream=stream.cuda_stream) as fb:
            fb.set_tiles(plan[0], plan[1], plan[2])
            fb.set_persistent(persistent)
            for _ in range(args.warmup):
                fb.step(1)
            ms = timed(lambda: fb.step(1))
            forms[name] = {"value": round(throughput(cells, steps, 1, ms * 1e-3), 3),
                           "ms_per_step": round(ms / steps, 4)}

    singles = [sim.Simulation(c, stream=stream.cuda_stream) for c in cases]
    for _ in range(args.warmup):
        for h in singles:
            h.step(1)

    def step_each():
        for h in singles:
            h.step(1)
    seq_ms = timed(step_each)
    for h in singles:
        h.close()

    fb = sim.Batch([c.replace(precision=W.FP64) for c in cases], stream=stream.cuda_stream)
    fb.step(args.warmup + steps)
    err = {k: 0.0 for k in "uvpT"}
    for q in range(len(cases)):
        f64 = fb.fields(q)
        for k in "uvpT":
            err[k] = max(err[k], float(np.abs(mixed_fields[q][k] - f64[k]).max() / np.abs(f64[k]).max()))
    fb.close()
    return {"workload": "64 channels, nx ~ U{256..2048} (multiples of 32), ny = nx/4, Mach U[1.5,3], Re U[50,400], "
                        "1-4 squares, implicit upwind, mixed precision, seeds 1000..1063",
            "cells": cells, "steps": steps, "value": round(throughput(cells, steps, 1, batch_ms * 1e-3), 3),
            "unit": UNIT, "ms_per_step": round(batch_ms / steps, 4),
            "tuned": {"tile": list(plan[:2]), "ctas": plan[2], "persistent": bool(plan[3])},
            "forms_at_tuned_tiles": forms,
            "one_by_one": {"value": round(throughput(cells, steps, 1, seq_ms * 1e-3), 3),
                           "ms_per_step": round(seq_ms / steps, 4)},
            "max_rel_err_vs_fp64_batch": {k: float(f"{v:.3e}") for k, v in err.items()},
            "error_after_steps": args.warmup + steps}


# ------------------------------------------------------------- cpu baseline

def oracle_throughput(case, target_s: float = 12.0, max_steps: int = 400, rows: bool = False):
    """Time the reference oracle (serial FP64 C, or with rows=True its
    row-parallel OpenMP build on all host threads) on the host on a bounded
    number of time steps of the same workload; returns (Mcell-steps/s, steps, seconds)."""
    import oracle
    state = oracle.init(case)
    t0 = time.perf_counter()
    state = oracle.run(case, state, nsteps=1, rows=rows)[0]
    t1 = time.perf_counter() - t0
    n = max(1, min(max_steps, int(target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(case, state, nsteps=n, rows=rows)
    dt = time.perf_counter() - t0
    return case.cells * n / dt / 1e6, n, dt


def cpu_rows_baseline(case):
    """The same oracle source built with OpenMP: its row loops split across
    all host threads (same bits as the serial build).  A second, multi-core
    CPU figure beside the one-core baseline."""
    import oracle
    try:
        v, n, secs = oracle_throughput(case, target_s=6.0, rows=True)
        cores = oracle.threads(rows=True)
    except (OSError, subprocess.CalledProcessError) as e:
        return {"unavailable": f"row-parallel oracle build failed: {e}".splitlines()[0]}
    return {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle, row-parallel (OpenMP)",
            "sample": f"{n} time steps of the same {case.nx}x{case.ny} channel from its seeded start "
                      f"({secs:.1f} s on {cores} threads)"}


# ------------------------------------------------------------ paper sweep

PAPER_HEIGHTS = (200, 400, 2000, 4000)
PAPER_SCHEMES = (("explicit-tvd", False, True), ("explicit-upwind", False, False),
                 ("implicit-tvd", True, True), ("implicit-upwind", True, False))
PAPER_TILES = ((256, 1), (128, 2), (64, 4), (32, 8), (16, 16))


def run_paper_sweep(args, local_rank):
    """The paper's experiment (Section 4): every scheme on the four meshes of
    its test case, FP64 Mcell-steps/s and the speedup over the serial oracle on
    one host core on the same case; then, for the implicit upwind scheme, the
    throughput of every tile shape of 256 threads (tile height 1 to 16 rows),
    which plays the part of the paper's rows per work-group."""
    import torch

    import paper_1802_04243_gb300 as sim
    import workloads as W
    from paper_1802_04243_gb300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    steps = max(1, args.steps)

    def timed(step_fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            step_fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    rows, tiles = [], []
    with ClockSampler(local_rank) as clocks:
        for ny in PAPER_HEIGHTS:
            base = W.paper_channel(ny=ny)
            for name, implicit, tvd in PAPER_SCHEMES:
                case = base.replace(implicit=implicit, tvd=tvd)
                with sim.Simulation(case, stream=stream.cuda_stream) as s:
                    for _ in range(args.warmup):
                        s.step(1)
                    ms = timed(lambda: s.step(1), steps)
                v = throughput(case.cells, steps, 1, ms * 1e-3)
                row = {"ny": ny, "particles": len(case.rects), "scheme": name, "fp64": round(v, 2)}
                if not args.no_cpu_baseline:
                    # one time step of the serial oracle on the same case
                    import oracle
                    state = oracle.init(case)
                    t0 = time.perf_counter()
                    oracle.run(case, state, nsteps=1)
                    dt = time.perf_counter() - t0
                    o = case.cells / dt / 1e6
                    row.update({"oracle_1core": round(o, 3), "speedup": round(v / o, 1),
                                "oracle_sample": f"1 step, {dt:.1f} s"})
                rows.append(row)
            case = base.replace(implicit=True, tvd=False)
            with sim.Batch([case], stream=stream.cuda_stream) as b:
                for tx, ty in PAPER_TILES:
                    b.set_tiles(tx, ty, 0)
                    for _ in range(max(2, args.warmup)):
                        b.step(1)
                    ms = timed(lambda: b.step(1), steps)
                    tiles.append({"ny": ny, "tile": [tx, ty],
                                  "fp64": round(throughput(case.cells, steps, 1, ms * 1e-3), 2)})
    top = next(r for r in rows if r["ny"] == PAPER_HEIGHTS[-1] and r["scheme"] == "implicit-upwind")
    line = {"metric": METRIC, "value": top["fp64"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper sweep: 4032 x {200, 400, 2000, 4000} channels with 1, 2, 10, 20 "
                                   "square particles (side 20 cells, one per 10 a of height), hard-sphere gas "
                                   "Kn 0.001, Mach 2.43, moving slip/jump walls; value = 4032x4000 implicit "
                                   "upwind",
                       "l2": "state larger than L2 on every mesh", "parallelism": "single GPU"},
            "sweep": rows, "tiles": tiles, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ plan sweep

PLAN_CANDIDATES = [(32, 8, 0, 0), (32, 4, 0, 0), (64, 2, 0, 0), (64, 4, 0, 0), (32, 4, 0, 1216), (32, 8, 0, 608),
                   (32, 8, 0, 1216), (32, 8, 0, 912), (32, 2, 0, 0), (128, 1, 0, 0)]


def run_plan_sweep(args, local_rank):
    """Time every candidate work distribution of the equation kernels
    (sim_set_plan: tile shape, CTA count) on the
    workload, for each precision: graph-replayed steps with the L2 flush
    between them, and per-kernel means from the event-timed pass.  Every plan
    gives the same bits (tests/test_batch_gpu.py)."""
    import torch

    import paper_1802_04243_gb300 as sim
    from paper_1802_04243_gb300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    base = workload()
    steps = max(1, args.steps)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    rows = []
    with ClockSampler(local_rank) as clocks:
        for prec in ("fp64", "mixed", "df64"):
            with sim.Simulation(base.replace(precision=PRECISIONS[prec]), stream=stream.cuda_stream) as s:
                for plan in PLAN_CANDIDATES:
                    s.set_plan(*plan)
                    for _ in range(args.warmup):
                        s.step(1)
                    ms = timed_steps(s, steps, stream, flush, starts, ends)
                    s.profile(True, timing=True)
                    timed_steps(s, min(steps, 10), stream, flush, starts, ends)
                    prof = s.profile_read()
                    s.profile(False)
                    rows.append({"precision": prec, "plan": list(plan),
                                 "value": round(throughput(base.cells, steps, 1, ms * 1e-3), 2),
                                 "kernel_ms_avg": {k: round(t / n, 5) for k, (t, n) in prof.items() if n}})
    print(json.dumps({"sweep": "plans", "config": config_of(base), "steps": steps, "warmup": args.warmup,
                      "rows": rows, "clocks": clocks.summary()}), flush=True)


# ------------------------------------------------------------------- ours

PRECISIONS = {"fp64": 0, "mixed": 1, "df64": 2}
DTYPE_OF = {"fp64": "f64",
            "mixed": "f32 assembly / f64 pressure, EOS, residuals",
            "df64": "df64 (float pairs, about 48 bits) in every kernel; f64 state on read-out"}


def scheme_key(case) -> str:
    return ("implicit" if case.implicit else "explicit") + ("-tvd" if case.tvd else "-upwind")


def fp64_roofline(case, asm_avg_s, clocks, n_sm, probe_gflops):
    """Roofline of k_assemble, FP64: achieved FP64 instructions per second
    (ncu's per-cell count for the scheme x cells / event-timed launch) against
    the FP64 pipe's peak at the sampled clock; None when the scheme has no
    count."""
    cnt = ASSEMBLE_FP64_COUNTS.get(scheme_key(case))
    if cnt is None:
        return None
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    per_cell = cnt["dfma"] + cnt["dadd"] + cnt["dmul"]
    inst = per_cell * case.cells                                               # per launch
    flops = (2 * cnt["dfma"] + cnt["dadd"] + cnt["dmul"]) * case.cells
    peak_inst = FP64_INST_PER_CYCLE_PER_SM * n_sm * sm_mhz * 1e6              # per second
    ach = inst / asm_avg_s
    return {"bound": "alu", "achieved": round(ach / 1e9, 2), "peak": round(peak_inst / 1e9, 2),
            "unit": "G FP64 inst/s", "frac": round(ach / peak_inst, 4),
            "traffic": round(cnt["dram_bytes"] * case.cells), "kernel": "k_assemble",
            "kernel_ms_avg": round(asm_avg_s * 1e3, 5),
            "peak_source": f"{FP64_INST_PER_CYCLE_PER_SM} FP64 instructions/cycle/SM x {n_sm} SMs x "
                           f"{sm_mhz:.0f} MHz (median SM clock sampled in the timed region)",
            "work_source": f"ncu DFMA+DADD+DMUL thread instructions per cell of one {scheme_key(case)} "
                           f"k_assemble launch on the {cnt['case']}: {per_cell:.1f} per cell, x {case.cells} cells",
            "traffic_source": f"ncu dram__bytes_read.sum + dram__bytes_write.sum of that launch, "
                              f"{cnt['dram_bytes']:.1f} B per cell, scaled to {case.cells} cells",
            "time_source": "mean event-timed k_assemble launch of the per-kernel pass",
            "fp64_pipe_active_ncu": cnt["fp64_pipe"],
            "flops": {"achieved_tflops": round(flops / asm_avg_s / 1e12, 4),
                      "peak_tflops": round(2 * peak_inst / 1e12, 4),
                      "probe_tflops": round(probe_gflops / 1e3, 4)},
            "hbm": {"algorithmic_gbs": round(ASSEMBLE_BYTES_PER_CELL * case.cells / asm_avg_s / 1e9, 1),
                    "peak_gbs": hbm_peak_gbs(), "unit": "GB/s"}}


def step_hbm(case, ms_per_step):
    """The whole step against HBM: the method's algorithmic bytes per step
    (method_bytes_per_step) over the graph-timed step."""
    b = method_bytes_per_step(case)
    ach = b / (ms_per_step * 1e-3) / 1e9
    peak = hbm_peak_gbs()
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "bytes_per_step": b,
            "bytes_source": ("12 doubles per cell and loop-2 iteration (u, v, p, T of the previous iterate and "
                             "of level n-1 read, u, v, p, T written)" if case.implicit else
                             "15 doubles per cell and loop-2 iteration (12 plus the three explicit terms) and "
                             "7 per step for the explicit terms"),
            "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


# ncu figures of the mixed path's loop-2 kernels (one launch each, one
# kernel per capture, implicit upwind): pipe and occupancy percentages and
# DRAM bytes per cell, from the case named; the commands are in profiles/.
MIXED_KERNEL_NCU = {
    "case": _C4HALF + ", ncu --metrics (one kernel per capture)",
    "faces": {"fma_pct": 19.2, "lsu_pct": 34.5, "fp64_pct": 0.0, "warps_active_pct": 86.2, "dram_bytes": 20.1},
    "assemble": {"fma_pct": 25.1, "lsu_pct": 43.0, "fp64_pct": 0.0, "warps_active_pct": 46.4, "dram_bytes": 68.0},
    "pressure": {"fma_pct": 12.5, "lsu_pct": 24.3, "fp64_pct": 76.7, "warps_active_pct": 92.7, "dram_bytes": 57.8},
    "velocity": {"fma_pct": 12.2, "lsu_pct": 37.2, "fp64_pct": 27.9, "warps_active_pct": 90.2, "dram_bytes": 34.4},
}


def mixed_roofline(case, ms_per_step, kernel_ms):
    """Roofline block of the mixed path: the step against HBM (the method's
    bytes, and the DRAM bytes ncu counted), and per kernel its measured time
    and the pipe that bounds it."""
    r = step_hbm(case, ms_per_step)
    dram = sum(MIXED_KERNEL_NCU[k]["dram_bytes"] for k in ("faces", "assemble", "pressure", "velocity"))
    r["traffic"] = round(dram * case.cells * case.iters)
    r["traffic_source"] = (f"sum of the four kernels' ncu DRAM bytes per cell ({dram:.1f} B) x cells x loop-2 "
                           f"iterations; counted on the {MIXED_KERNEL_NCU['case']}")
    per = {}
    for k in ("faces", "assemble", "pressure", "velocity"):
        n = MIXED_KERNEL_NCU[k]
        pipes = {"fma": n["fma_pct"], "lsu": n["lsu_pct"], "fp64": n["fp64_pct"]}
        top = max(pipes, key=pipes.get)
        per[k] = {**n, "ms_avg": kernel_ms.get(k),
                  "bound": ("fp64 pipe" if top == "fp64" and pipes["fp64"] > 60 else
                            "latency (no pipe above 60 %, LSU the busiest)" if top == "lsu" else f"{top} pipe")}
    r["kernels"] = per
    return r


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1802_04243_gb300 as sim
    import workloads as W
    from paper_1802_04243_gb300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    base = workload()
    case = base.replace(precision=PRECISIONS[args.precision])
    stream = torch.cuda.current_stream()
    sim.Simulation(small_case(), stream=stream.cuda_stream).close()   # loads the GPU code first
    s, dev_bytes = device_bytes_of(lambda: sim.Simulation(case, stream=stream.cuda_stream))
    for _ in range(args.warmup):
        s.step(1)
    peak_fp64 = 0.0 if args.only_main else sim.alu_peak_gflops("fp64", 30.0, stream.cuda_stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2 (126 MB)
    n_ev = max(args.steps, 1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]

    s.profile(True, timing=False)                  # count launches; step graphs stay on
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks:
        total_ms = timed_steps(s, args.steps, stream, flush, starts, ends)
    if dist:
        dist.barrier()
    launches = sum(n for _, n in s.profile_read().values())
    res, iters, st = s.residuals()
    total_ms = reduce_max(total_ms, dist, "cuda")
    value = throughput(case.cells, args.steps, world, total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    csum = clocks.summary()

    if args.only_main:
        s.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "dtype": DTYPE_OF[args.precision], "data": "synthetic", "config": config_of(case),
                              "gpu_launches": int(launches), "clocks": csum, "impl": "ours",
                              "note": "--only-main: the main timed run alone (profiling command)"}), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    main_state = s.fields()

    # per-kernel durations: the same steps again, kernels launched one by one
    # between CUDA events on the same stream
    prof_steps = min(args.steps, 50)

    def kernel_pass(h):
        h.profile(True, timing=True)
        timed_steps(h, prof_steps, stream, flush, starts, ends)
        p = h.profile_read()
        h.profile(False)
        return p

    prof = kernel_pass(s)
    kernel_ms = {k: ms / n for k, (ms, n) in prof.items() if n}
    event_ms_per_step = sum(ms for ms, _ in prof.values()) / prof_steps

    # the same workload and timing protocol with the other precisions of the
    # sweep, and their per-field error against the main run after the same
    # number of steps from the same start
    def variant(prec_name):
        sv, v_bytes = device_bytes_of(lambda: sim.Simulation(base.replace(precision=PRECISIONS[prec_name]),
                                                             stream=stream.cuda_stream))
        for _ in range(args.warmup):
            sv.step(1)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as vclocks:
            v_ms = timed_steps(sv, args.steps, stream, flush, starts, ends)
        v_state = sv.fields()
        vprof = kernel_pass(sv)
        sv.close()
        v_ms = reduce_max(v_ms, dist, "cuda")
        err = {k: float(np.abs(v_state[k] - main_state[k]).max() / np.abs(main_state[k]).max())
               for k in ("u", "v", "p", "T")}
        vk = {k: ms / n for k, (ms, n) in vprof.items() if n}
        out = {"value": round(throughput(case.cells, args.steps, world, v_ms * 1e-3), 3),
               "ms_per_step": round(v_ms / args.steps, 5), "dtype": DTYPE_OF[prec_name],
               f"max_rel_err_vs_{args.precision}": {k: float(f"{x:.3e}") for k, x in err.items()},
               "error_after_steps": args.warmup + args.steps,
               "device_bytes_per_cell": round(v_bytes / case.cells, 1),
               "kernel_ms_avg": {k: round(x, 5) for k, x in vk.items()}, "clocks": vclocks.summary()}
        if prec_name == "mixed":
            out["roofline"] = mixed_roofline(case, v_ms / args.steps, vk)
        else:
            out["step_hbm"] = step_hbm(case, v_ms / args.steps)
        return out

    others = {p: variant(p) for p in ("fp64", "mixed", "df64") if p != args.precision}

    # the same workload decomposed into x-strips on this device (halo of 4
    # columns recomputed per loop-2 iteration, one halo-copy kernel per
    # iteration): the cost of the decomposition against the whole problem
    strips = {}
    for n_strips in (2, 4):
        with sim.Strips(case, n_strips, stream=stream.cuda_stream) as sp:
            for _ in range(args.warmup):
                sp.step(1)
            torch.cuda.synchronize()
            sp_ms = timed_steps(sp, min(args.steps, 50), stream, flush, starts, ends)
            sp_ms = reduce_max(sp_ms, dist, "cuda")
            nst = min(args.steps, 50)
            strips[str(n_strips)] = {"value": round(throughput(case.cells, nst, world, sp_ms * 1e-3), 3),
                                     "ms_per_step": round(sp_ms / nst, 5),
                                     "vs_whole": round((total_ms / args.steps) / (sp_ms / nst), 4)}

    # end to end through the C ABI with host buffers: every step uploads its
    # input state from pinned host memory (sim_set_state), advances one step
    # and reads the new state and the residuals back (sim_get_state)
    host = {k: torch.from_numpy(v).pin_memory() for k, v in s.fields().items()}
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = h2d + 4 * 8
    views = {k: v.numpy() for k, v in host.items()}
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    for _ in range(2):
        s.set_state(views); s.step(1); s.get_state(views)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(views)
        s.step(1)
        s.get_state(views)
    e2e_s = time.perf_counter() - t0
    e2e_value = throughput(case.cells, e2e_steps, world, reduce_max(e2e_s, dist, "cuda"))
    s.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    roof = None
    if args.precision == "fp64" and "assemble" in kernel_ms:
        roof = fp64_roofline(case, kernel_ms["assemble"] * 1e-3, csum, n_sm, peak_fp64)
    elif args.precision == "mixed":
        roof = mixed_roofline(case, ms_per_step, kernel_ms)

    batched = None if args.no_batch else run_batch(args, stream)

    cpu = cpu_rows = None
    if not args.no_cpu_baseline:
        v, n, secs = oracle_throughput(case)
        cpu = {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} time steps of the same {case.nx}x{case.ny} channel from its seeded start "
                         f"({secs:.1f} s, serial FP64 C oracle); Mcell-steps/s = cells x steps / seconds"}
        cpu_rows = cpu_rows_baseline(case)

    steps_per_iter_kernels = {k: n / (prof_steps * case.iters) for k, (_, n) in prof.items() if n}
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_OF[args.precision], "data": "synthetic",
            "config": config_of(case),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "path": "sim_set_state (pinned host -> device), sim_step, sim_get_state (device -> pinned "
                            "host, residuals)"},
            "mcell_iterations_per_s": round(value * case.iters, 3),
            "device_bytes_per_cell": round(dev_bytes / case.cells, 1),
            "gpu_launches": int(launches),
            "roofline": roof, "step_hbm": step_hbm(case, ms_per_step),
            "kernel_ms_avg": {k: round(x, 5) for k, x in kernel_ms.items()},
            "kernel_timing": {
                "how": f"separate pass of {prof_steps} steps, every kernel launched on its own between two "
                       "CUDA events on the library's stream (the timed steps replay one CUDA graph per step, "
                       "which has no per-kernel events)",
                "event_pass_ms_per_step": round(event_ms_per_step, 5), "graph_ms_per_step": round(ms_per_step, 5),
                "note": "the per-launch events and the direct launches add overhead, so the event pass's sum "
                        "exceeds the graph-timed step; shares between kernels and each kernel's mean are what "
                        "it gives (the roofline's k_assemble time comes from it)",
                "launches_per_iteration": {k: round(x, 3) for k, x in steps_per_iter_kernels.items()}},
            **others, "strips": {"note": "the same workload as x-strips on this device, value and ratio to the "
                                         "whole-problem step time", **strips},
            "batched": batched, "cpu_baseline": cpu,
            "cpu_baseline_rows": cpu_rows, "clocks": csum,
            "residuals_last_step": [float(x) for x in res], "impl": "ours"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# -------------------------------------------------------------- reference

def run_reference(args, rank, world):
    """The reference arm: the serial FP64 oracle on the host cores."""
    if rank != 0:
        return
    import oracle
    case = workload()
    state = oracle.init(case)
    for _ in range(args.warmup):
        t0 = time.perf_counter()
        state = oracle.run(case, state, nsteps=1)[0]
        t_step = time.perf_counter() - t0
    budget = 150.0
    n = args.steps if args.warmup == 0 or args.steps * t_step <= budget else max(1, int(budget / t_step))
    t0 = time.perf_counter()
    oracle.run(case, state, nsteps=n)
    secs = time.perf_counter() - t0
    value = case.cells * n / secs / 1e6
    sample = (f"{n} of the {args.steps} requested time steps of the {case.nx}x{case.ny} channel "
              f"({secs:.1f} s, serial FP64 C oracle on one host core)")
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs / n * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(case), "parallelism": "host, one core", "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "kind": "oracle", "cores": 1, "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global _ARGS
    args = parse()
    _ARGS = args
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sweep == "paper":
        if rank == 0:
            run_paper_sweep(args, local_rank)
    elif args.sweep == "plans":
        if rank == 0:
            run_plan_sweep(args, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
