"""The C ABI library builds, loads and exports every function declared in
include/hps.h; argument checks answer before any device work (no GPU)."""

import ctypes
import math

import numpy as np
import pytest

from paper_2112_02211_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    return N.load()


def test_exports_every_declared_function(lib):
    names = N.header_functions()
    assert "hps_setup" in names and "hps_gmres_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    assert set(names) == set(N.SIGNATURES)


def test_default_options(lib):
    o = N.Options()
    lib.hps_default_options(ctypes.byref(o))
    assert o.restart == 50 and o.cluster == 2 and o.forms == 3 and o.max_rhs == 1


def _setup(lib, grid, kappa=10.0, eta=10.0, b=None, opt=None):
    h = ctypes.c_void_p()
    bp = None if b is None else b.ctypes.data_as(ctypes.c_void_p)
    rc = lib.hps_setup(ctypes.byref(grid), kappa, eta, bp, None if opt is None else ctypes.byref(opt),
                       ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("grid", [N.Grid(2, 2, 2, 8, 5), N.Grid(0, 2, 2, 8, 6), N.Grid(2, 2, 2, 3, 1),
                                  N.Grid(2, 2, 2, 17, 15)])
def test_setup_rejects_bad_grids(lib, grid):
    rc, h = _setup(lib, grid)
    assert rc == N.HPS_EINVAL
    assert not h.value
    assert lib.hps_last_error()


def test_setup_rejects_zero_eta_and_nan_medium(lib):
    g = N.Grid(1, 1, 1, 6, 4)
    rc, _ = _setup(lib, g, eta=0.0)
    assert rc == N.HPS_EINVAL
    rc, _ = _setup(lib, g, kappa=math.nan)
    assert rc == N.HPS_EINVAL
    b = np.zeros(4 ** 3, dtype=np.complex128)
    b[5] = np.nan
    rc, _ = _setup(lib, g, b=b)
    assert rc == N.HPS_EINVAL and b"NaN" in lib.hps_last_error()


def test_setup_rejects_bad_options(lib):
    g = N.Grid(1, 1, 1, 6, 4)
    o = N.Options()
    lib.hps_default_options(ctypes.byref(o))
    o.restart = 100
    rc, _ = _setup(lib, g, opt=o)
    assert rc == N.HPS_EINVAL
    lib.hps_default_options(ctypes.byref(o))
    o.cluster = 3
    rc, _ = _setup(lib, g, opt=o)
    assert rc == N.HPS_EINVAL


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.hps_apply(None, 0, None, None, 1, None) == N.HPS_EINVAL
    assert lib.hps_precond(None, 0, None, None, 1, None) == N.HPS_EINVAL
    assert lib.hps_gmres_solve(None, 1, None, None, 1, 1e-6, None, None, None) == N.HPS_EINVAL
    assert lib.hps_export(None, 0, 0, None) == N.HPS_EINVAL
    assert lib.hps_destroy(None) == N.HPS_OK
    assert lib.hps_memory_bytes(None) == 0
