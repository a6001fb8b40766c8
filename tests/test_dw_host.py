"""The double-word operations of the HZ_FP64_DW path built for the host (the product's headers
with a stand-in for cuda_runtime.h, tests/host_build/) against exact decimal arithmetic: the same
bounds as the GPU self-test, without a GPU."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from dw_check import NRESULTS, check_pair_results, pair_inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1102_5202_gb300", "csrc")


@pytest.fixture(scope="module")
def host_lib():
    out = os.path.join(tempfile.mkdtemp(prefix="dw_host_"), "dw_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-I", os.path.join(HERE, "host_build"), "-I", CSRC, os.path.join(HERE, "host_build", "dw_host.cpp"),
           "-o", out]
    subprocess.run(cmd, check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    L.dw_selftest_host.argtypes = [dp, dp, dp, ctypes.c_long]
    L.dw_selftest_host.restype = None
    return L


def test_pair_arithmetic_error_bounds_host(host_lib):
    a, b, m = pair_inputs()
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    out = np.zeros((NRESULTS, 2, len(a)))
    dp = ctypes.POINTER(ctypes.c_double)
    host_lib.dw_selftest_host(a.ctypes.data_as(dp), b.ctypes.data_as(dp), out.ctypes.data_as(dp), len(a))
    check_pair_results(a, out, m)


def test_split_is_exact_for_24_bit_values(host_lib):
    """A double with at most 24 significant bits splits into (itself, 0)."""
    rng = np.random.Generator(np.random.PCG64(7))
    a = (rng.integers(1, 2 ** 24, 256) * 2.0 ** rng.integers(-100, 100, 256)).astype(np.float64)
    out = np.zeros((NRESULTS, 2, len(a)))
    dp = ctypes.POINTER(ctypes.c_double)
    host_lib.dw_selftest_host(a.ctypes.data_as(dp), np.ones_like(a).ctypes.data_as(dp),
                              out.ctypes.data_as(dp), len(a))
    assert np.array_equal(out[0, 0], a) and np.all(out[0, 1] == 0.0)
