"""The C-ABI library builds for sm_103a, loads, exports every entry point include/hzn.h
declares, and validates arguments before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1102_5202_gb300 import build, hzn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hzn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return hzn.lib()


def test_header_declares_binding_names():
    assert set(declared_functions()) == set(hzn.EXPORTED) | set(hzn.ENSEMBLE_EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert hzn.hz_version() == 1


def test_strerror_names_every_code(lib):
    for code in (0, 1, -1, -2, -3, -4, -5):
        assert hzn.hz_strerror(code) != "unknown code"
    assert hzn.hz_strerror(-99) == "unknown code"


def test_workspace_bytes_and_argument_checks(lib):
    g = hzn.make_grid((192, 192, 192), (0.2, 0.2, 0.2), (0, 0, 0))
    o = hzn.make_options(2.0, cleaning=True, ch=0.5, kappa=1.0)
    nb = hzn.hz_workspace_bytes(g, o)
    # 10 padded metric fields + 4 state arrays of 9 padded fields, FP64
    assert nb >= (10 * 194 ** 3 + 4 * 9 * 192 ** 3) * 8
    assert nb < (10 * 208 * 194 * 194 + 4 * 9 * 192 ** 3 + 4096) * 8
    bad = [
        (hzn.make_grid((1, 4, 4), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_UNSUPPORTED),
        (hzn.make_grid((8, 1, 4), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_UNSUPPORTED),
        (hzn.make_grid((8, 8, 8), (1, 0, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((8, 8, 8), (1, 1, 1), (0, 2, 0)), o, hzn.HZ_ERR_ARG),
        (g, hzn.make_options(1.0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, cleaning=True, ch=0.0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, c2p_maxit=0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, rho_floor=0.0), hzn.HZ_ERR_ARG),
    ]
    for gg, oo, code in bad:
        n = ctypes.c_size_t(0)
        assert lib.hz_workspace_bytes(ctypes.byref(gg), ctypes.byref(oo), ctypes.byref(n)) == code
    # null pointers
    assert lib.hz_workspace_bytes(None, None, None) == hzn.HZ_ERR_ARG
    assert lib.hz_step(None, ctypes.c_double(1.0)) == hzn.HZ_ERR_ARG
    assert lib.hz_set_metric(None, None) == hzn.HZ_ERR_ARG
    h = ctypes.c_void_p(0)
    # misaligned / missing workspace is rejected before any device work
    assert lib.hz_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(o), ctypes.c_void_p(8), nb,
                         None) == hzn.HZ_ERR_WORKSPACE
    assert lib.hz_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(o), ctypes.c_void_p(4096),
                         nb - 8, None) == hzn.HZ_ERR_WORKSPACE
