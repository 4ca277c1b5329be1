"""The host eigen-decomposition behind Algorithm 3 (Sec. 4.1: L1 = V E V^{-1} per axis, used by
the global-system preconditioner) through the C ABI, without a GPU, against numpy's general
eigensolver on the oracle's L1 for every supported order, plus special cases with known answers."""

import ctypes

import numpy as np
import pytest

from oracle.kron import interior_L1
from paper_2112_02211_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    return N.load()


def _eig(lib, M):
    M = np.ascontiguousarray(M, dtype=np.float64)
    n = M.shape[0]
    V, Vi, E = np.zeros((n, n)), np.zeros((n, n)), np.zeros(n)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = lib.hps_axis_eig(n, ptr(M), ptr(V), ptr(Vi), ptr(E))
    return rc, V, Vi, E


@pytest.mark.parametrize("p", range(4, 17))
@pytest.mark.parametrize("h", [1.0, 1.0 / 3.0, 1.0 / 32.0])
def test_l1_factorization_matches_numpy(lib, p, h):
    M = interior_L1(p, h)
    rc, V, Vi, E = _eig(lib, M)
    assert rc == N.HPS_OK
    ref = np.linalg.eigvals(M)
    assert np.max(np.abs(ref.imag)) == 0.0  # real spectrum: the premise of Algorithm 3
    assert np.allclose(np.sort(E), np.sort(ref.real), rtol=1e-12, atol=0)
    scale = np.max(np.abs(M))
    assert np.max(np.abs(M @ V - V * E)) <= 1e-9 * scale
    assert np.max(np.abs(V @ Vi - np.eye(len(E)))) <= 1e-9
    # the factorization reproduces M, as Algorithm 3's mode products use it
    assert np.max(np.abs(V @ np.diag(E) @ Vi - M)) <= 1e-9 * scale


def test_diagonal_and_triangular(lib):
    rc, V, Vi, E = _eig(lib, np.diag([3.0, -1.0, 2.0]))
    assert rc == N.HPS_OK and sorted(E) == [-1.0, 2.0, 3.0]
    T = np.array([[1.0, 5.0, -2.0], [0.0, 4.0, 7.0], [0.0, 0.0, -3.0]])
    rc, V, Vi, E = _eig(lib, T)
    assert rc == N.HPS_OK
    assert np.allclose(np.sort(E), [-3.0, 1.0, 4.0], rtol=1e-13)
    rc, V, Vi, E = _eig(lib, np.array([[5.0]]))
    assert rc == N.HPS_OK and E[0] == 5.0 and abs(V[0, 0] * Vi[0, 0] - 1.0) < 1e-15


def test_complex_pair_is_refused(lib):
    rc, *_ = _eig(lib, np.array([[0.0, 1.0], [-1.0, 0.0]]))
    assert rc == N.HPS_EBREAKDOWN
    assert b"eigen" in lib.hps_last_error()


def test_bad_arguments(lib):
    M = np.eye(3)
    M[1, 2] = np.nan
    rc, *_ = _eig(lib, M)
    assert rc == N.HPS_EINVAL
    assert lib.hps_axis_eig(0, None, None, None, None) == N.HPS_EINVAL
