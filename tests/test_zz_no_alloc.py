"""hz_step_noalloc: the whole update for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: a solver embedded as a plug-in in a host
framework that owns all device memory through its own pool, or a thin foreign-function layer
that only passes pointers it was given.  hz_step_noalloc runs the same kernels on a static
device scratch array instead of a caller-provided workspace.  These tests call it through the
C-ABI and check it against the workspace path (hz_create + hz_step) on two calls in a row.
This file is collected last so that a run stopping at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from parity import TOL_ONE_STEP, assert_parity
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1102_5202_gb300 import build
    build.build_library()
    hzn.lib()


def _reference(P, dt, nsteps):
    s = hzn.Solver.for_problem(P)
    for _ in range(nsteps):
        s.step(dt)
    out = s.primitives().cpu().numpy()
    return out, s


def _noalloc(P, opts, dt, nsteps, stream):
    import torch

    met = torch.from_numpy(np.ascontiguousarray(P.metric)).cuda()
    pin = torch.from_numpy(np.ascontiguousarray(P.prim)).cuda()
    pout = torch.full_like(pin, float("nan"))
    grid = hzn.make_grid(P.n, P.dx, P.bc)
    torch.cuda.synchronize()
    code = hzn.hz_step_noalloc(grid, opts, met.data_ptr(), pin.data_ptr(), pout.data_ptr(), dt,
                               nsteps, stream.cuda_stream)
    # the call returns once its result is written: nothing of it is left on the stream, and no
    # recovery failed on these problems
    assert stream.query()
    assert code == hzn.HZ_OK
    return pout.cpu().numpy()


@pytest.mark.parametrize("case", ["blob24", "balsara400"])
def test_noalloc_matches_workspace_path_twice(case):
    import torch

    P = W.blob3d(24) if case == "blob24" else W.balsara1(400)
    nsteps = 2 if case == "blob24" else 3
    ref_solver = hzn.Solver.for_problem(P)
    dt = 0.5 / ref_solver.max_speed()
    ref, s = _reference(P, dt, nsteps)
    stream = torch.cuda.current_stream()
    for call in range(2):
        got = _noalloc(P, s.options, dt, nsteps, stream)
        assert np.all(np.isfinite(got))
        assert_parity(got, ref, TOL_ONE_STEP, what=f"{case} no-alloc call {call + 1}")


def test_noalloc_interleaved_problems_do_not_leak_state():
    """A different problem in between leaves nothing behind that changes the next result."""
    import torch

    A, B = W.blob3d(16), W.balsara1(128)
    sa = hzn.Solver.for_problem(A)
    dta = 0.5 / sa.max_speed()
    refA, s = _reference(A, dta, 1)
    stream = torch.cuda.current_stream()
    first = _noalloc(A, s.options, dta, 1, stream)
    sb = hzn.Solver.for_problem(B)
    _noalloc(B, sb.options, 0.5 / sb.max_speed(), 2, stream)
    second = _noalloc(A, s.options, dta, 1, stream)
    assert_parity(first, refA, TOL_ONE_STEP, what="A before B")
    assert_parity(second, refA, TOL_ONE_STEP, what="A after B")


def test_noalloc_rejects_grids_beyond_the_scratch():
    opts = hzn.make_options(2.0, cleaning=True, ch=0.5, kappa=1.0)
    big = hzn.make_grid((64, 64, 64), (0.1, 0.1, 0.1), (0, 0, 0))
    assert hzn.hz_workspace_bytes(big, opts) > hzn.HZ_NOALLOC_SCRATCH_BYTES
    with pytest.raises(hzn.HznError) as e:
        hzn.hz_step_noalloc(big, opts, 256, 256, 256, 0.1, 1, 0)
    assert e.value.code == hzn.HZ_ERR_TOO_LARGE
    fits = hzn.make_grid((24, 24, 24), (0.1, 0.1, 0.1), (0, 0, 0))
    assert hzn.hz_workspace_bytes(fits, opts) <= hzn.HZ_NOALLOC_SCRATCH_BYTES
