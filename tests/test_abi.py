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
    assert set(declared_functions()) == (set(hzn.EXPORTED) | set(hzn.ENSEMBLE_EXPORTED) |
                                         set(hzn.ADJOINT_EXPORTED))


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert hzn.hz_version() == 1


def test_strerror_names_every_code(lib):
    for code in (0, 1, -1, -2, -3, -4, -5):
        assert hzn.hz_strerror(code) != "unknown code"
    assert hzn.hz_strerror(-99) == "unknown code"


def test_cuda_error_query(lib):
    """hz_last_cuda_error starts at 0 on a thread that met no CUDA error (argument errors are
    not CUDA errors), and hz_cuda_error_string describes CUDA runtime codes."""
    import threading

    seen = []

    def probe():
        seen.append(int(lib.hz_last_cuda_error()))
        g = hzn.make_grid((0, 1, 1), (0.1, 1.0, 1.0), (0, 0, 0))
        o = hzn.make_options(2.0)
        n = ctypes.c_size_t(0)
        seen.append(int(lib.hz_workspace_bytes(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n))))
        seen.append(int(lib.hz_last_cuda_error()))

    t = threading.Thread(target=probe)
    t.start()
    t.join()
    assert seen == [0, hzn.HZ_ERR_ARG, 0]
    assert lib.hz_cuda_error_string(0).decode() == "no error"
    assert "argument" in lib.hz_cuda_error_string(1).decode()


def test_workspace_bytes_and_argument_checks(lib):
    g = hzn.make_grid((192, 192, 192), (0.2, 0.2, 0.2), (0, 0, 0))
    o = hzn.make_options(2.0, cleaning=True, ch=0.5, kappa=1.0)
    nb = hzn.hz_workspace_bytes(g, o)
    # 10 padded metric fields + 4 state arrays of 9 padded fields + the geometry tables of a
    # DIAG metric (centre 11 fields, faces 3 x 11, source differences 3 x 4; metric layout), FP64
    msize = 208 * 194 * 194
    assert nb >= (10 * 194 ** 3 + 4 * 9 * 192 ** 3 + 56 * 194 ** 3) * 8
    assert nb < (10 * msize + 4 * 9 * 192 ** 3 + 56 * msize + 4096) * 8
    bad = [
        (hzn.make_grid((1, 4, 4), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_UNSUPPORTED),
        # degenerate grids: empty, negative, a single cell (no active axis)
        (hzn.make_grid((0, 1, 1), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((8, 0, 1), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((-4, 1, 1), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((1, 1, 1), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_UNSUPPORTED),
        # sizes whose index arithmetic or workspace would overflow
        (hzn.make_grid((2 ** 31 - 1, 1, 1), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((2 ** 20, 2 ** 20, 2 ** 20), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((8, 1, 4), (1, 1, 1), (0, 0, 0)), o, hzn.HZ_ERR_UNSUPPORTED),
        (hzn.make_grid((8, 8, 8), (1, 0, 1), (0, 0, 0)), o, hzn.HZ_ERR_ARG),
        (hzn.make_grid((8, 8, 8), (1, 1, 1), (0, 2, 0)), o, hzn.HZ_ERR_ARG),
        (g, hzn.make_options(1.0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, cleaning=True, ch=0.0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, c2p_maxit=0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, rho_floor=0.0), hzn.HZ_ERR_ARG),
        (g, hzn.make_options(2.0, precision=3), hzn.HZ_ERR_ARG),
        # the double-word face path has MC reconstruction only
        (g, hzn.make_options(2.0, precision=hzn.HZ_FP64_DW, recon=hzn.HZ_RECON_PPM), hzn.HZ_ERR_UNSUPPORTED),
    ]
    # the double-word face path keeps the FP64 layout
    assert hzn.hz_workspace_bytes(g, hzn.make_options(2.0, cleaning=True, ch=0.5, kappa=1.0,
                                                      precision=hzn.HZ_FP64_DW)) == nb
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


def test_adjoint_workspace_and_argument_checks(lib):
    g = hzn.make_grid((800, 1, 1), (1.0 / 800, 1, 1), (0, 0, 0))
    o = hzn.make_options(2.0)
    nb = hzn.hz_adjoint_workspace_bytes(g, o, 1000, 0)
    # 32 checkpoints of (P, U) + a tape of 3*32+1 states + 7 cell arrays + 2 face arrays
    per = 9 * 832 * 8  # 800 cells padded to a field stride of 832
    assert nb >= (32 * 2 + 97 + 7) * per
    assert nb < (32 * 2 + 97 + 7 + 4) * per + 300 * 256
    n = ctypes.c_size_t(0)
    L = hzn._adj_lib()
    mixed = hzn.make_options(2.0, precision=hzn.HZ_MIXED)
    assert L.hz_adjoint_workspace_bytes(ctypes.byref(g), ctypes.byref(mixed), 10, 0,
                                        ctypes.byref(n)) == hzn.HZ_ERR_UNSUPPORTED
    assert L.hz_adjoint_workspace_bytes(ctypes.byref(g), ctypes.byref(o), 0, 0,
                                        ctypes.byref(n)) == hzn.HZ_ERR_ARG
    h = ctypes.c_void_p(0)
    assert L.hz_adjoint_create(ctypes.byref(h), None, 10, 0.1, 0, None, 0) == hzn.HZ_ERR_ARG
    assert L.hz_adjoint_backward(None, None, None, None) == hzn.HZ_ERR_ARG
