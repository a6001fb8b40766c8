"""Writes ``opcount_blob3d.json``: the op count (``opcount.py``) of one RK3 step of the oracle on
the 3-D blob in its curved diagonal spacetime (MC reconstruction, divergence cleaning, CFL 0.5),
at the size the benchmark's FP64 line runs (192^3) and at the sizes the CPU tests recount.

    python -m oracle.write_counts            # from the repository root; ~15 min on 8 cores

Calls nothing but ``oracle/`` and the seeded input generators.  TEST AND MEASUREMENT
INFRASTRUCTURE, NOT PRODUCT CODE.
"""
from __future__ import annotations

import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle as O  # noqa: E402
from oracle import opcount as OC  # noqa: E402
from paper_1102_5202_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "opcount_blob3d.json")
SIZES = (16, 32, 192)


def count_blob(n: int, check_rhs: bool) -> dict:
    P = W.blob3d(n)
    grid = O.make_grid(P.n, P.dx, P.bc)
    opts = O.make_opts(P.gamma, cleaning=P.cleaning, ch=P.ch, kappa=P.kappa, rho_floor=P.rho_floor,
                       p_floor=P.p_floor, atm_K=P.atm_K, rho_atm=P.rho_atm, recon=P.recon)
    dt = P.cfl / O.max_speed(grid, opts, P.metric, P.prim)
    t0 = time.time()
    r = OC.count_step(grid, opts, P.metric, P.prim, dt, check_rhs=check_rhs)
    return {
        "n": n,
        "seconds": round(time.time() - t0, 1),
        "dt": dt,
        "flops_per_zu": OC.step_flops_per_zu(r),
        "per_zu": r["per_zu"],
        "raw_per_zu": r["raw_per_zu"],
        "ops_per_zu": {op: float(r["tally"][1:, q].sum()) / r["ncell"] for q, op in enumerate(OC.OPS)},
        "recovery_iterations": r["iters"],
        "recovery_calls": r["calls"],
        "check": [int(c) for c in r["check"]],
        "vdiff": r["vdiff"],
    }


def main():
    out = {"workload": "blob3d (curved diagonal spacetime, MC, cleaning on, kappa 1, CFL 0.5)",
           "unit": "flops per zone update (one cell, one RK3 step)",
           "counts": {}}
    for n in SIZES:
        out["counts"][str(n)] = count_blob(n, check_rhs=n <= 32)
        print(n, out["counts"][str(n)]["flops_per_zu"], out["counts"][str(n)]["seconds"], "s", flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
