"""Benchmark of the GB300 GRMHD finite-volume hot path: zone-updates per second.

Workload (N = 1): the 3-D GRMHD blob in a fixed capped-Schwarzschild spacetime, 192^3 cells
on [-20, 20]^3, FP64, divergence cleaning on, seed 1102 (the paper's rotating-neutron-star
runs of §4.1 need the external rns code; this seeded blob has their shape).  One "step" is
one full RK3 step (three fused substep launches plus the device time-step clock) over the
whole grid.  The state (about 2.6 GB) is larger than L2, so no flush is needed between steps.

Lines printed (one JSON line on rank 0):
  default          the CUDA path: device-timed value, roofline of the substep kernel, the
                   oracle's CPU baseline on a bounded sample, an end-to-end number through
                   the C-ABI with host buffers, SM clocks sampled during the timed region;
  --impl reference the FP64 oracle on the host cores on a bounded sample of the same
                   workload (the reference arm: a deliberately slow, plain program).
Under torchrun (N > 1) every rank advances its own independent replica (the path is not
sharded across GPUs): value = all ranks' zone updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-updates/s"
UNIT = "ZU/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA throughput measured on this machine's GB300 with an in-register DFMA loop
# (profiles/fp64_alu_peak.md): 2 DFMA per clock per SM x 152 SMs.
FP64_PEAK_TFLOPS = 1.194
FP32_PEAK_TFLOPS = 72.98  # FFMA loop of the same probe, 8 blocks per SM
# Double-word (pair-of-FP32) multiply-add loop of the same probe: 1.98e12 per second, two flops
# each -- the rate of the double-word path's face arithmetic.
DW_PEAK_TFLOPS = 3.96
# Algorithmic flops per zone update (one cell, one RK3 step) of the method on the blob
# workload at 192^3 (MC, cleaning on, CFL 0.5), from the op-counting oracle
# (oracle/opcount_blob3d.json, written by oracle/write_counts.py): the floating-point operations
# (+, -, *, /, sqrt) that each face's and each cell's results and decisions depend on, each
# counted once, operations on structural zeros of the diagonal spacetime and the static
# geometry excluded.  The roofline's achieved rate is this count over the measured time.
FP64_ALG_FLOPS_PER_ZU = 3898.8812772962783
# The part of it in the phases the mixed path keeps in FP64 (RK update, recovery, CFL maximum);
# the rest (reconstruction, face states, fluxes, speeds, HLLE, divergence, sources) runs in FP32
# there.
ALG_FLOPS_PER_ZU_FP64_PHASES = 308.66399468315973
# FP64 operations per cell per substep executed by the fused substep kernel (3-D, cleaning
# on, diagonal metric with its geometry tables), from ncu instruction counters on the 128^3
# blob (profiles/k_substep_blob3d.md): DFMA counted as 2 flops, DADD/DMUL as 1.  Reported
# beside the algorithmic rate: the kernel's own arithmetic (reciprocal refinements, the
# recovery's corrections) differs from the method's count.
FP64_FLOPS_PER_CELL_SUBSTEP = 1502.6
# FP64 instructions (DFMA + DMUL + DADD) per cell per substep from the same capture, and the
# FP64 instruction rate of the pipe measured by the probe (1.91 DFMA per clock per SM at
# 2070 MHz): DMUL and DADD occupy the pipe like a DFMA, so this fraction is the pipe's use.
FP64_INST_PER_CELL_SUBSTEP = 1171.8
FP64_INST_PEAK_PER_S = 6.0e11
# DRAM bytes per cell per substep of the same kernel from the same capture (read + write,
# 2180 MB per launch at 128^3, the geometry tables included), scaled by the cell count.
DRAM_BYTES_PER_CELL_SUBSTEP = 1039.6
# The same two figures for the mixed-precision substep kernel at 192^3
# (profiles/k_substep_mixed_blob3d.md): FP64 flops (recovery, update) per cell per substep,
# and DRAM bytes per cell per substep.
MIXED_FP64_FLOPS_PER_CELL_SUBSTEP = 52.3
MIXED_DRAM_BYTES_PER_CELL_SUBSTEP = 304.9
# Algorithmic HBM bytes per zone update (three substeps, FP64, nine fields): read P, U_k, U0,
# metric and write U_{k+1}, P_{k+1} once per substep; stage 1 reads U0 once.
HBM_BYTES_PER_ZU = (46 + 55 + 55) * 8
# Mixed precision: primitives and metric stored in FP32 (4 B), conserved state in FP64 (8 B):
# stage 1 reads P, metric, U0 and writes U, P; stages 2-3 also read U_k.
HBM_BYTES_PER_ZU_MIXED = (9 * 4 + 10 * 4 + 9 * 8 + 9 * 8 + 9 * 4) + 2 * (9 * 4 + 10 * 4 + 2 * 9 * 8 + 9 * 8 + 9 * 4)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=192, help="cells per axis of the blob")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-dw", action="store_true", help="skip the double-word face leg")
    ap.add_argument("--adjoint-reps", type=int, default=3, help="timed repetitions of the adjoint leg")
    ap.add_argument("--no-mixed-error", action="store_true",
                    help="skip the mixed error statement (100 FP64 and 100 mixed steps at the mixed size, about a minute)")
    ap.add_argument("--ensemble-tubes", type=int, default=512)
    ap.add_argument("--n-mixed", type=int, default=384, help="cells per axis of the mixed line")
    ap.add_argument("--sweep", default="",
                    help="comma-separated cells per axis: instead of the benchmark line, print one JSON line "
                         "of FP64 and mixed ZU/s of the blob at each size (cost per zone update against grid size)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def aggregate(units_local: float, seconds_local: float, dist, device=None):
    """Whole-job throughput: sum of units over ranks / max of time over ranks."""
    if dist is None:
        return units_local, seconds_local
    import torch

    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to $HZN_CLOCKS_DIR (default: the temporary directory)
        self.path = os.path.join(os.environ.get("HZN_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"hzn_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm = float(parts[1].split()[0])
                smax = float(parts[2].split()[0])
            except ValueError:
                continue
            rows.append((sm, smax, parts[5], parts[6], parts[7], parts[8]))
        if not rows:
            return None
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------------- GPU arm
def fp64_roofline(cells: int, substep_s: float) -> dict:
    """ALU roofline of the FP64 substep kernel: the method's algorithmic flops per launch over
    the mean launch duration against the measured DFMA peak, with the kernel's executed FP64
    flops and instructions beside it."""
    ach = FP64_ALG_FLOPS_PER_ZU / 3.0 * cells / substep_s / 1e12
    impl = FP64_FLOPS_PER_CELL_SUBSTEP * cells / substep_s / 1e12
    inst = FP64_INST_PER_CELL_SUBSTEP * cells / substep_s
    return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS,
            "traffic": DRAM_BYTES_PER_CELL_SUBSTEP * cells if DRAM_BYTES_PER_CELL_SUBSTEP else None,
            "kernel": "k_substep<32,4,3-D,cleaning,diag,FP64,MC>", "peak_source": "measured FP64 DFMA loop",
            "algorithmic_flops_per_zu": FP64_ALG_FLOPS_PER_ZU,
            "implemented_fp64_flops": {"per_cell_substep": FP64_FLOPS_PER_CELL_SUBSTEP, "achieved": impl,
                                       "frac": impl / FP64_PEAK_TFLOPS},
            "fp64_instructions": {"per_cell_substep": FP64_INST_PER_CELL_SUBSTEP, "achieved_per_s": inst,
                                  "peak_per_s": FP64_INST_PEAK_PER_S, "frac": inst / FP64_INST_PEAK_PER_S}}


def mixed_roofline(cells: int, substep_s: float) -> dict:
    """ALU roofline of the mixed-precision substep kernel: the algorithmic flops of the phases
    it keeps in FP64 against the DFMA peak, those of its FP32 phases against the FFMA peak."""
    fl = ALG_FLOPS_PER_ZU_FP64_PHASES / 3.0 * cells / substep_s / 1e12
    fl32 = (FP64_ALG_FLOPS_PER_ZU - ALG_FLOPS_PER_ZU_FP64_PHASES) / 3.0 * cells / substep_s / 1e12
    impl = MIXED_FP64_FLOPS_PER_CELL_SUBSTEP * cells / substep_s / 1e12
    return {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": fl / FP64_PEAK_TFLOPS,
            "traffic": MIXED_DRAM_BYTES_PER_CELL_SUBSTEP * cells if MIXED_DRAM_BYTES_PER_CELL_SUBSTEP else None,
            "kernel": "k_substep<32,4,3-D,cleaning,diag,mixed> (FP64 recovery and update)",
            "algorithmic_flops_per_zu_fp64_phases": ALG_FLOPS_PER_ZU_FP64_PHASES,
            "implemented_fp64_flops": {"per_cell_substep": MIXED_FP64_FLOPS_PER_CELL_SUBSTEP,
                                       "achieved": impl, "frac": impl / FP64_PEAK_TFLOPS},
            "fp32_phases": {"achieved": fl32, "peak": FP32_PEAK_TFLOPS, "frac": fl32 / FP32_PEAK_TFLOPS}}


def dw_roofline(cells: int, substep_s: float) -> dict:
    """ALU roofline of the double-word face path: the algorithmic flops of its face phases
    (reconstruction to sources, in pair-of-FP32 arithmetic) against the measured double-word
    multiply-add rate, those of its FP64 phases (update, recovery, CFL) against the DFMA peak."""
    f64 = ALG_FLOPS_PER_ZU_FP64_PHASES / 3.0 * cells / substep_s / 1e12
    fdw = (FP64_ALG_FLOPS_PER_ZU - ALG_FLOPS_PER_ZU_FP64_PHASES) / 3.0 * cells / substep_s / 1e12
    return {"bound": "alu", "achieved": fdw, "peak": DW_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": fdw / DW_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_substep<32,4,3-D,cleaning,diag,FP64 state,double-word faces>",
            "peak_source": "measured double-word multiply-add loop (2 flops each)",
            "fp64_phases": {"achieved": f64, "peak": FP64_PEAK_TFLOPS, "frac": f64 / FP64_PEAK_TFLOPS}}


def run_gpu(args, rank, world, local):
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    P = W.blob3d(args.n)
    s = hzn.Solver.for_problem(P)
    stream = s.stream
    cells = P.ncell

    for _ in range(args.warmup):
        s.step_cfl(0.5, 1e30)
    torch.cuda.synchronize()
    st0 = s.stats()
    if st0.c2p_failures:
        print(f"[rank {rank}] warning: {st0.c2p_failures} recovery failures in warm-up", file=sys.stderr)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            s.step_cfl(0.5, 1e30)
            ev[k][1].record(stream)
        t_stop.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_stop) * 1e-3
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = s.stats()
    units, seconds = aggregate(float(cells) * args.steps, elapsed, dist, device=torch.device("cuda", local))
    value = units / seconds

    # roofline of the dominant kernel (the fused substep): three launches per step
    substep_s = statistics.mean(step_ms) * 1e-3 / 3.0
    roof = fp64_roofline(cells, substep_s)
    hbm_peak = json.load(open(MEASURED_PEAKS))["hbm_gbs"] if os.path.exists(MEASURED_PEAKS) else 6800.0
    hbm_ach = HBM_BYTES_PER_ZU / 3.0 * cells / substep_s / 1e9
    hbm = {"bytes_per_zu": HBM_BYTES_PER_ZU, "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_ach / hbm_peak, "roofline_zu_per_s": hbm_peak * 1e9 / HBM_BYTES_PER_ZU,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if os.path.exists(MEASURED_PEAKS) else "fallback"}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(s, P, args, dist, local)

    mixed = None
    if not args.no_mixed:
        del s
        torch.cuda.empty_cache()
        mixed = run_mixed(args, dist, local, hbm_peak)

    ensemble = None
    if not args.no_ensemble:
        ensemble = run_ensemble(args, dist, local)

    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, dist, local, reps=args.adjoint_reps)

    variants = None
    if not args.no_variants:
        variants = run_variants(args, dist, local, base_zu_per_s=value)

    dw = None
    if not args.no_dw:
        dw = run_dw(args, dist, local, base_zu_per_s=value)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = run_cpu_baseline(P, seconds_target=15.0)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": seconds / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"blob3d_{args.n}^3_fp64_cleaning", "cells": cells,
                       "domain": "[-20,20]^3", "metric": "capped isotropic Schwarzschild M=1.4",
                       "cfl": 0.5, "courant": "sum over axes", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state larger than L2 (no flush)"},
            "roofline": roof,
            "hbm_roofline": hbm,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "ensemble": ensemble,
            "adjoint": adjoint,
            "variants": variants,
            "fp64_dw_faces": dw,
            "gpu_launches": 4 * args.steps,
            "clocks": clk,
            "c2p_failures": int(st.c2p_failures),
            "sim_time": st.t,
            # last, so that a reader of the line's tail sees the mixed configuration's figures
            "mixed": mixed,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_mixed(args, dist, local, hbm_peak):
    """The mixed-precision configuration: the same blob at 384^3 (FP32 faces and sources,
    FP64 conserved state, update, recovery and CFL), timed like the FP64 line."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    P = W.blob3d(args.n_mixed)
    s = hzn.Solver.for_problem(P, precision=hzn.HZ_MIXED)
    for _ in range(args.warmup):
        s.step_cfl(0.5, 1e30)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s.stream):
        a.record(s.stream)
        for _ in range(args.steps):
            s.step_cfl(0.5, 1e30)
        b.record(s.stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    st = s.stats()
    units, seconds = aggregate(float(P.ncell) * args.steps, sec, dist, device=torch.device("cuda", local))
    value = units / seconds
    ach = HBM_BYTES_PER_ZU_MIXED * value / world_size(dist) / 1e9
    substep_s = sec / args.steps / 3.0
    del s
    torch.cuda.empty_cache()
    err = None if args.no_mixed_error else mixed_error(P)
    # the headline figures come last (a reader of the line's tail sees them first)
    return {"error_vs_fp64_gpu_100_steps": err, "roofline": mixed_roofline(P.ncell, substep_s),
            "workload": f"blob3d_{args.n_mixed}^3_mixed_cleaning", "cells": P.ncell,
            "dtype": "f32/f64", "c2p_failures": int(st.c2p_failures), "gpu_launches": 4 * args.steps,
            "ms_per_step": seconds / args.steps * 1e3,
            "hbm_roofline": {"bytes_per_zu": HBM_BYTES_PER_ZU_MIXED, "achieved": ach, "peak": hbm_peak,
                             "unit": "GB/s", "roofline_zu_per_s": hbm_peak * 1e9 / HBM_BYTES_PER_ZU_MIXED,
                             "frac": ach / hbm_peak},
            "unit": UNIT, "value": value}


def mixed_error(P, steps: int = 100):
    """Relative L1 per field of the mixed run against the FP64 GPU run of the same blob after
    `steps` CFL steps (the FP64 run's time steps replayed), whole grid and star bulk."""
    import torch

    from paper_1102_5202_gb300 import hzn

    s = hzn.Solver.for_problem(P)
    dts = []
    for _ in range(steps):
        s.step_cfl(0.5, 1e30)
        dts.append(s.stats().dt)
    a = s.primitives().cpu().numpy()
    del s
    torch.cuda.empty_cache()
    s = hzn.Solver.for_problem(P, precision=hzn.HZ_MIXED)
    for dt in dts:
        s.step(dt)
    b = s.primitives().cpu().numpy()
    fails = int(s.stats().c2p_failures)
    del s
    torch.cuda.empty_cache()

    def rel(x, y):
        den = np.array([np.abs(y[g, ...]).sum() if len(g) == 1 else
                        np.sqrt((y[list(g)] ** 2).sum(axis=0)).sum() for g in
                        ((0,), (1,), (2, 3, 4), (2, 3, 4), (2, 3, 4), (5, 6, 7), (5, 6, 7), (5, 6, 7), (8,))])
        return [float(np.abs(x[f] - y[f]).sum() / max(den[f], 1e-300)) for f in range(9)]

    star = a[0] > 0.1 * a[0].max()
    return {"fields": ["rho", "p", "utx", "uty", "utz", "Bx", "By", "Bz", "psi"], "steps": steps,
            "whole_grid": rel(b, a), "star_bulk": rel(b[:, star], a[:, star]), "mixed_c2p_failures": fails}


def run_adjoint(args, dist, local, reps: int = 3):
    """The gradient configurations: the 1-D tube (N=800, 1000 fixed steps, textured base point)
    and the 2-D cylindrical blast wave (256^2, 200 fixed steps).  Each rep times, with CUDA
    events on the solver's stream: the plain forward run (hz_step x n), the forward pass with
    sqrt(n) checkpoints (hz_adjoint_forward) and the reverse sweep (hz_adjoint_backward, which
    recomputes each segment).  adjoint_over_forward = reverse sweep / plain forward (median of
    the reps)."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    out = {}
    for P in (W.adjoint_tube(800), W.blast2d(256)):
        steps, dt = P.steps, W.fixed_dt(P)
        s = hzn.Solver.for_problem(P)
        A = hzn.Adjoint(s, steps, dt)
        st = s.stream
        g = torch.zeros((9,) + P.prim.shape[1:], dtype=torch.float64, device="cuda")
        g[0] = 1.0
        prim0 = s._dev(P.prim)
        rows = []
        for rep in range(reps + 1):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            with torch.cuda.stream(st):
                s.set_primitives(prim0)
                ev[0].record(st)
                for _ in range(steps):
                    s.step(dt)
                ev[1].record(st)
                A.forward(prim0)
                ev[2].record(st)
                A.backward(g)
                ev[3].record(st)
            ev[3].synchronize()
            if rep:  # the first rep warms up
                rows.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
        rows = np.array(rows)
        fwd, ckf, bwd = (float(np.median(rows[:, k])) for k in range(3))
        zu = float(P.ncell) * steps
        units, seconds = aggregate(zu, bwd * 1e-3, dist, device=torch.device("cuda", local))
        key = "tube1d" if P.n[1] == 1 else "blast2d"
        out[key] = {"workload": f"{P.name}_{'x'.join(str(k) for k in P.n if k > 1)}_{steps}steps_fp64",
                    "cells": P.ncell, "steps": steps, "dt": dt, "checkpoint_every": A.checkpoint_every,
                    "segments": A.segments, "forward_ms": fwd, "forward_checkpointed_ms": ckf,
                    "backward_ms": bwd, "adjoint_over_forward": bwd / fwd,
                    "forward_and_backward_over_forward": (ckf + bwd) / fwd,
                    "backward_zone_updates_per_s": units / seconds,
                    "gpu_launches_backward": 9 * steps + A.segments + 3}
        A.close()
        s.close()
    return out


def run_variants(args, dist, local, base_zu_per_s: float, steps: int = 5, warmup: int = 2):
    """The scheme variants of §3.2 on the FP64 blob at the benchmark size, each timed like the
    main line (CUDA events on the solver's stream, CFL 0.5 steps): PPM reconstruction, the 1D
    recovery scheme, and the toroidal-field initial data of §5.2."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    out = {}
    for name in ("ppm", "c2p_1d", "toroidal"):
        P = W.blob3d(args.n, field="toroidal" if name == "toroidal" else "poloidal")
        if name == "ppm":
            P.recon = hzn.HZ_RECON_PPM
        if name == "c2p_1d":
            P.c2p = hzn.HZ_C2P_1D
        s = hzn.Solver.for_problem(P)
        for _ in range(warmup):
            s.step_cfl(0.5, 1e30)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(s.stream):
            a.record(s.stream)
            for _ in range(steps):
                s.step_cfl(0.5, 1e30)
            b.record(s.stream)
        b.synchronize()
        sec = a.elapsed_time(b) * 1e-3
        st = s.stats()
        units, seconds = aggregate(float(P.ncell) * steps, sec, dist, device=torch.device("cuda", local))
        out[name] = {"workload": f"{P.name}_fp64" + ("_ppm" if name == "ppm" else "") +
                     ("_c2p1d" if name == "c2p_1d" else ""), "value": units / seconds, "unit": UNIT,
                     "steps": steps, "ms_per_step": seconds / steps * 1e3,
                     "relative_to_mc_2d_poloidal": units / seconds / base_zu_per_s,
                     "c2p_failures": int(st.c2p_failures), "gpu_launches": 4 * steps}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def run_dw(args, dist, local, base_zu_per_s: float, steps: int = 10, warmup: int = 2):
    """The benchmark blob with the double-word face path (FP64 state, update, recovery and CFL
    maximum; faces, fluxes and sources in pair-of-FP32 arithmetic), timed like the main line,
    and its per-field relative L1 distance from the FP64 path after the same steps."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    P = W.blob3d(args.n)
    s = hzn.Solver.for_problem(P, precision=hzn.HZ_FP64_DW)
    for _ in range(warmup):
        s.step_cfl(0.5, 1e30)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(s.stream):
        a.record(s.stream)
        for _ in range(steps):
            s.step_cfl(0.5, 1e30)
        b.record(s.stream)
    b.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    st = s.stats()
    units, seconds = aggregate(float(P.ncell) * steps, sec, dist, device=torch.device("cuda", local))
    dw_prim = s.primitives().cpu().numpy()
    s.close()
    del s
    torch.cuda.empty_cache()
    # the FP64 path over the same steps from the same state
    r = hzn.Solver.for_problem(P)
    for _ in range(warmup + steps):
        r.step_cfl(0.5, 1e30)
    ref = r.primitives().cpu().numpy()
    r.close()
    del r
    torch.cuda.empty_cache()
    num = np.abs(dw_prim - ref).reshape(9, -1).sum(1)
    den = np.abs(ref).reshape(9, -1).sum(1)
    rel = {W.PRIM_FIELDS[f]: float(num[f] / den[f]) if den[f] > 0 else float(num[f]) for f in range(9)}
    return {"workload": f"{P.name}_fp64_dw_faces", "value": units / seconds, "unit": UNIT,
            "steps": steps, "ms_per_step": seconds / steps * 1e3,
            "relative_to_fp64": units / seconds / base_zu_per_s,
            "rel_l1_vs_fp64_gpu": rel, "c2p_failures": int(st.c2p_failures),
            "roofline": dw_roofline(P.ncell, seconds / steps / 3.0),
            "dtype": "f64 state / f32x2 faces", "gpu_launches": 4 * steps}


def world_size(dist):
    return 1 if dist is None else dist.get_world_size()


def run_ensemble(args, dist, local):
    """The batched configuration: 512 independent magnetised tubes (cells U{200..4000}, seed
    1103) advanced to t = 0.4 at CFL 0.5 in one persistent, graph-captured launch whose block
    shape the library's autotuner picks.  Zone updates = sum over tubes of cells x steps."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    tubes = W.ensemble(args.ensemble_tubes, seed=1103)
    E = hzn.Ensemble(tubes)
    threads, ctas, probe_ms = E.autotune(t_probe=0.02)
    E.set_primitives()
    E.run(0.4, 0.5, use_graph=True)  # warm-up: captures and runs the graph
    E.stream.synchronize()
    E.set_primitives()
    E.stream.synchronize()
    if dist is not None:
        dist.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(E.stream)
    E.run(0.4, 0.5, use_graph=True)
    b.record(E.stream)
    b.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    t, steps, fails = E.results()
    zu = float((E.n.astype(np.float64) * steps).sum())
    units, seconds = aggregate(zu, sec, dist, device=torch.device("cuda", local))
    E.close()
    return {"value": units / seconds, "unit": UNIT, "workload": f"ensemble_{len(tubes)}_tubes_fp64",
            "tubes": len(tubes), "cells": int(E.n.sum()), "zone_updates": zu, "seconds": seconds,
            "t_reached_min": float(t.min()), "steps_min": int(steps.min()), "steps_max": int(steps.max()),
            "c2p_failures": int(fails.sum()), "launch": {"threads": threads, "ctas_per_sm": ctas,
                                                         "autotune_probe_ms": [round(m, 3) for m in probe_ms]},
            "graph": True, "gpu_launches": 1}


def run_e2e(s, P, args, dist, local):
    """Same metric through the C-ABI with the state in pinned host memory: every step copies
    the primitive state host->device, converts it, advances one RK3 step and copies the new
    primitive state back.  Two solver contexts on two streams take the steps in turn, so that
    one step's host<->device copies run on the copy engines while the other step computes."""
    import torch

    from paper_1102_5202_gb300 import hzn

    host_in = torch.from_numpy(np.ascontiguousarray(P.prim)).pin_memory()
    s2 = hzn.Solver.for_problem(P, stream=torch.cuda.Stream(device=s.device))
    lanes = []
    for sol in (s, s2):
        lanes.append({
            "sol": sol,
            "dev_in": torch.empty(host_in.shape, dtype=torch.float64, device=s.device),
            "dev_out": torch.empty(host_in.shape, dtype=torch.float64, device=s.device),
            "host_out": torch.empty_like(host_in).pin_memory(),
        })
    nsteps = max(4, min(args.steps, 20))
    nsteps += nsteps % 2

    def one(L):
        st = L["sol"].stream
        with torch.cuda.stream(st):
            L["dev_in"].copy_(host_in, non_blocking=True)
            hzn.hz_set_primitives(L["sol"].ctx, L["dev_in"].data_ptr())
            hzn.hz_step_cfl(L["sol"].ctx, 0.5, 1e30)
            hzn.hz_get_primitives(L["sol"].ctx, L["dev_out"].data_ptr())
            L["host_out"].copy_(L["dev_out"], non_blocking=True)

    sa, sb = lanes[0]["sol"].stream, lanes[1]["sol"].stream
    one(lanes[0])
    one(lanes[1])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(sa)
    sb.wait_event(a)
    for k in range(nsteps):
        one(lanes[k % 2])
    done_b = torch.cuda.Event()
    done_b.record(sb)
    sa.wait_event(done_b)
    b.record(sa)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    units, seconds = aggregate(float(P.ncell) * nsteps, sec, dist, device=torch.device("cuda", local))
    nbytes = host_in.numel() * 8
    s2.close()
    # restore the benchmark state
    s.set_primitives(P.prim)
    return {"value": units / seconds, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": nsteps,
            "pipeline": "2 solver contexts on 2 streams, steps alternate; copies overlap the other context's compute"}


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(P, m: int):
    """Central m^3 sub-box of the workload with its metric (the sample the oracle times)."""
    lo = (P.n[0] - m) // 2
    return P.subbox((lo,) * 3, (lo + m,) * 3, name=f"{P.name}_sample{m}")


def _time_oracle_steps(O, Q, seconds_target):
    grid = O.make_grid(Q.n, Q.dx, Q.bc)
    opts = O.make_opts(Q.gamma, cleaning=Q.cleaning, ch=Q.ch, kappa=Q.kappa, rho_floor=Q.rho_floor,
                       p_floor=Q.p_floor, atm_K=Q.atm_K, rho_atm=Q.rho_atm)
    U = O.grid_prim2cons(grid, opts, Q.metric, Q.prim)
    dt = 0.5 / O.max_speed(grid, opts, Q.metric, Q.prim)
    prim, cons = Q.prim, U
    steps = 0
    t0 = time.perf_counter()
    while True:
        prim, cons, _ = O.step(grid, opts, Q.metric, prim, cons, dt)
        steps += 1
        if time.perf_counter() - t0 >= seconds_target or steps >= 1000:
            break
    return steps, time.perf_counter() - t0


def run_cpu_baseline(P, seconds_target=15.0, m=48, m_single=24, seconds_single=6.0):
    """The oracle on the host cores (OpenMP over all of them) on the central m^3 sub-box of the
    benchmark blob, and on one core on a smaller sub-box."""
    import oracle as O

    Q = oracle_sample(P, m)
    cores = O.num_threads()
    steps, sec = _time_oracle_steps(O, Q, seconds_target)
    out = {"value": Q.ncell * steps / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{steps} RK3 step(s) of the central {m}^3 sub-box of the {P.n[0]}^3 blob, "
                     f"{sec:.1f} s"}
    Q1 = oracle_sample(P, m_single)
    O.set_num_threads(1)
    try:
        steps1, sec1 = _time_oracle_steps(O, Q1, seconds_single)
    finally:
        O.set_num_threads(cores)
    v1 = Q1.ncell * steps1 / sec1
    out["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{steps1} RK3 step(s) of the central {m_single}^3 sub-box, "
                                      f"{sec1:.1f} s"}
    out["cpu_model"] = cpu_model()
    # the one-core figure and the CPU also in the sample text, which every reader of the line keeps
    out["sample"] += (f"; one core: {v1:.3g} {UNIT} on {steps1} RK3 step(s) of the central "
                      f"{m_single}^3 sub-box; CPU {out['cpu_model']}, {cores} threads")
    return out


def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    import subprocess

    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_1102_5202_gb300 import workloads as W

    import oracle as O

    P = W.blob3d(args.n)
    m = 32
    Q = oracle_sample(P, m)
    grid = O.make_grid(Q.n, Q.dx, Q.bc)
    opts = O.make_opts(Q.gamma, cleaning=Q.cleaning, ch=Q.ch, kappa=Q.kappa, rho_floor=Q.rho_floor,
                       p_floor=Q.p_floor, atm_K=Q.atm_K, rho_atm=Q.rho_atm)
    U = O.grid_prim2cons(grid, opts, Q.metric, Q.prim)
    dt = 0.5 / O.max_speed(grid, opts, Q.metric, Q.prim)
    prim, cons = Q.prim, U
    for _ in range(args.warmup):
        prim, cons, _ = O.step(grid, opts, Q.metric, prim, cons, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prim, cons, _ = O.step(grid, opts, Q.metric, prim, cons, dt)
    sec = time.perf_counter() - t0
    value = Q.ncell * args.steps / sec
    sample = f"each step: one RK3 step of the central {m}^3 sub-box of the {args.n}^3 blob"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"blob3d_{args.n}^3_fp64_cleaning", "cells": P.ncell,
                       "domain": "[-20,20]^3", "metric": "capped isotropic Schwarzschild M=1.4",
                       "cfl": 0.5, "courant": "sum over axes", "sample_cells": Q.ncell,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def run_sweep(args):
    """Zone updates per second of the blob against its size, FP64 and mixed: each size `warmup`
    untimed CFL steps, then `steps` steps timed with CUDA events on the solver's stream."""
    import torch

    from paper_1102_5202_gb300 import hzn
    from paper_1102_5202_gb300 import workloads as W

    rows = []
    for n in (int(x) for x in args.sweep.split(",") if x):
        P = W.blob3d(n)
        row = {"n": n, "cells": P.ncell}
        for name, prec in (("fp64", hzn.HZ_FP64), ("mixed", hzn.HZ_MIXED)):
            s = hzn.Solver.for_problem(P, precision=prec)
            for _ in range(args.warmup):
                s.step_cfl(0.5, 1e30)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s.stream):
                a.record(s.stream)
                for _ in range(args.steps):
                    s.step_cfl(0.5, 1e30)
                b.record(s.stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) * 1e-3
            row[name] = P.ncell * args.steps / sec
            row[name + "_ms_per_step"] = sec / args.steps * 1e3
            s.close()
            del s
            torch.cuda.empty_cache()
        rows.append(row)
    print(json.dumps({"sweep": "blob3d", "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "rows": rows}))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweep:
        run_sweep(args)
        return
    run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
