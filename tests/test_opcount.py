"""Pins of the op-counting oracle (``oracle/opcount.cpp``), which fixes the algorithmic flops per
zone update behind the FP64 path's ALU roofline.

What pins it, besides itself: the phased driver's raw count and values equal those of the
oracle's own rhs() run with the counting scalar; closed forms of the phases whose operation
count the method's formulas fix exactly (the RK3 update of §3.2: 2 + 5 + 5 flops per conserved
field; the flux divergence: a difference, a scaling and an accumulation per axis and field; the
MC reconstruction of a uniform state: only its three differences, every slope being zero);
invariants of the counting conventions (a diagonal spacetime costs less than a general one in
the metric-dependent phases and the same elsewhere; the distinct count never exceeds the raw
one); and the stored counts that the benchmark uses, recomputed."""
import json
import os

import numpy as np
import pytest

import oracle as O
import parity
from oracle import opcount as OC
from paper_1102_5202_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
NCONS = 9


def _count(P, dt=1e-3, check_rhs=True):
    grid, opts = parity.oracle_setup(P)
    return OC.count_step(grid, opts, P.metric, P.prim, dt, check_rhs=check_rhs)


@pytest.fixture(scope="module")
def blob():
    return _count(W.blob3d(12))


@pytest.fixture(scope="module")
def general():
    P = W.with_periodic_metric(W.smooth_periodic((8, 6, 5), seed=3), parity.general_metric)
    P.cleaning, P.ch, P.kappa = True, 0.6, 0.3
    return _count(P)


@pytest.fixture(scope="module")
def diag_twin():
    """The same periodic data in the diagonal part of the same metric."""
    P = W.with_periodic_metric(W.smooth_periodic((8, 6, 5), seed=3), parity.general_metric)
    P.metric[1:4] = 0.0
    P.metric[[5, 6, 8]] = 0.0
    P.cleaning, P.ch, P.kappa = True, 0.6, 0.3
    return _count(P)


def test_phased_rhs_is_the_oracles_rhs(blob, general):
    for r in (blob, general):
        assert r["check"].tolist() == [0, 0, 0]
        assert r["vdiff"] == 0.0


def test_rk3_update_costs_twelve_flops_per_field(blob, general):
    for r in (blob, general):
        assert r["per_zu"]["update"] == 12 * NCONS
        assert r["raw_per_zu"]["update"] == 12 * NCONS


@pytest.mark.parametrize("n,ndim", [((40, 1, 1), 1), ((10, 8, 1), 2), ((8, 6, 5), 3)])
def test_divergence_cost_per_axis_and_field(n, ndim):
    r = _count(W.smooth_periodic(n, seed=4), check_rhs=False)
    want = 3 * NCONS * (3 * ndim - 1)  # the first axis accumulates into zero
    assert r["per_zu"]["divergence"] == want
    assert r["raw_per_zu"]["divergence"] == want


def test_mc_reconstruction_of_a_uniform_state_is_three_differences():
    """Uniform periodic 1-D state: every MC slope vanishes, so a face costs the differences of
    its four-cell stencil, three distinct (four as written) per field; n + 1 faces per axis."""
    P = W.smooth_periodic((24, 1, 1), seed=5, amp=0.0)
    r = _count(P, check_rhs=False)
    faces_per_cell = 25 / 24
    assert r["per_zu"]["recon"] == pytest.approx(3 * NCONS * 3 * faces_per_cell, rel=1e-12)
    assert r["raw_per_zu"]["recon"] == pytest.approx(3 * NCONS * 4 * faces_per_cell, rel=1e-12)


def test_diagonal_spacetime_costs_less_where_the_metric_enters(general, diag_twin):
    for ph in ("face_state", "sources", "geometry"):
        assert diag_twin["per_zu"][ph] < general["per_zu"][ph], ph
    for ph in ("update", "divergence"):
        assert diag_twin["per_zu"][ph] == general["per_zu"][ph], ph
    # the limiter's branches follow the data, which the two metrics evolve differently after
    # the first stage
    for ph in ("recon", "hlle"):
        assert diag_twin["per_zu"][ph] == pytest.approx(general["per_zu"][ph], rel=0.01), ph


def test_distinct_count_never_exceeds_raw(blob, general):
    for r in (blob, general):
        assert np.all(r["tally"] <= r["raw"])
        assert r["tally"].sum() > 0.5 * r["raw"].sum()


def test_recovery_count_includes_the_root_solve(blob):
    assert blob["calls"] > 0 and blob["iters"] >= blob["calls"]
    assert blob["per_zu"]["c2p"] * blob["ncell"] > blob["iters"] * 10


def test_stored_blob_counts_and_benchmark_constant():
    """The stored counts (oracle/write_counts.py) recompute exactly at the small sizes, vary
    little with resolution, and the benchmark's constant is the 192^3 figure."""
    path = os.path.join(ROOT, "oracle", "opcount_blob3d.json")
    stored = json.load(open(path))["counts"]
    r = OC.step_flops_per_zu(_count(W.blob3d(16), dt=stored["16"]["dt"], check_rhs=False))
    assert r == stored["16"]["flops_per_zu"]
    big = stored["192"]["flops_per_zu"]
    assert abs(stored["32"]["flops_per_zu"] / big - 1.0) < 0.02
    import bench
    assert bench.FP64_ALG_FLOPS_PER_ZU == pytest.approx(big, rel=1e-9)
    ph = stored["192"]["per_zu"]
    assert bench.ALG_FLOPS_PER_ZU_FP64_PHASES == pytest.approx(ph["update"] + ph["c2p"] + ph["cfl"], rel=1e-9)


def test_benchmark_roofline_objects():
    """The roofline objects the benchmark prints, from a measured launch duration: the
    algorithmic rate is the op count per cell-substep times the cells over the duration, and
    the kernel's executed figures sit beside it (captured 128^3 launch: 5.56 ms)."""
    import bench
    cells, t = 128 ** 3, 5.56e-3
    r = bench.fp64_roofline(cells, t)
    json.dumps(r)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.FP64_ALG_FLOPS_PER_ZU / 3 * cells / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert 0.35 < r["frac"] < 0.45
    assert 0.43 < r["implemented_fp64_flops"]["frac"] < 0.53  # 0.58 TFLOP/s in the capture
    assert r["traffic"] == pytest.approx(bench.DRAM_BYTES_PER_CELL_SUBSTEP * cells)
    m = bench.mixed_roofline(cells, t / 8)
    json.dumps(m)
    assert m["achieved"] + m["fp32_phases"]["achieved"] == pytest.approx(
        bench.FP64_ALG_FLOPS_PER_ZU / 3 * cells / (t / 8) / 1e12)
    d = bench.dw_roofline(cells, t / 1.5)
    json.dumps(d)
    assert d["achieved"] + d["fp64_phases"]["achieved"] == pytest.approx(
        bench.FP64_ALG_FLOPS_PER_ZU / 3 * cells / (t / 1.5) / 1e12)
    assert d["frac"] == pytest.approx(d["achieved"] / bench.DW_PEAK_TFLOPS)
