"""hps_setup_bytes, the admission estimate of the serving loop (no GPU): it covers the arrays a
handle must hold, computed here from their definitions (leaf maps R, H per leaf, cluster inverses
per cluster, the Krylov basis), stays within a bounded margin above them, and orders the forms as
their contents do."""

import ctypes

import pytest

from paper_2112_02211_gb300 import _native as N

GiB = 1 << 30


@pytest.fixture(scope="module")
def lib():
    return N.load()


def _bytes(lib, L, p, forms=3, lean=0, nrhs=1, restart=50, cluster=2, lambda_bin=0.0):
    o = N.Options()
    lib.hps_default_options(ctypes.byref(o))
    o.forms, o.lean, o.max_rhs, o.restart, o.cluster, o.lambda_bin = forms, lean, nrhs, restart, cluster, lambda_bin
    g = N.Grid(L, L, L, p, p - 2)
    return lib.hps_setup_bytes(ctypes.byref(g), ctypes.byref(o), nrhs)


def _rup4(n):
    return (n + 3) // 4 * 4


def _arrays(L, p, r_bytes, h_bytes, k_bytes, nrhs=1, restart=50, cluster=True):
    """Leaf maps R (6q^2 x 6q^2), H (6q^2 x n1^3), cluster inverses (24q^2 square per 2x2x2
    cluster), Krylov basis (restart + 1 vectors of N_f complex, 16 bytes per entry)."""
    q = n1 = p - 2
    nb, ni, nl = 6 * q * q, n1 ** 3, L ** 3
    total = nl * nb * _rup4(nb) * r_bytes + nl * nb * _rup4(ni) * h_bytes
    if cluster:
        total += (L // 2) ** 3 * (24 * q * q) * _rup4(24 * q * q) * k_bytes
    total += (restart + 1) * nrhs * nl * nb * 16
    return total


@pytest.mark.parametrize("L,p", [(4, 8), (16, 10), (32, 10)])
def test_lean_covers_its_arrays(lib, L, p):
    # FP32 maps and their FP16 remainders, FP16 cluster inverses
    need = _arrays(L, p, r_bytes=12, h_bytes=12, k_bytes=4)
    got = _bytes(lib, L, p, forms=N.HPS_FORM_MIXED, lean=1, lambda_bin=0.01)
    assert need <= got <= 1.15 * need + 24 * GiB + 4 * GiB


@pytest.mark.parametrize("L,p", [(4, 8), (16, 10)])
def test_both_forms_cover_their_arrays(lib, L, p):
    # FP64 and FP32 maps with the FP16 remainders of the FP32 ones (R and H), cluster inverses in
    # FP64, FP32 and FP16
    need = _arrays(L, p, r_bytes=16 + 8 + 4, h_bytes=16 + 8 + 4, k_bytes=16 + 8 + 4)
    got = _bytes(lib, L, p)
    assert need <= got <= 1.15 * need + 24 * GiB


def test_forms_are_ordered(lib):
    both = _bytes(lib, 16, 10)
    mixed = _bytes(lib, 16, 10, forms=N.HPS_FORM_MIXED)
    lean = _bytes(lib, 16, 10, forms=N.HPS_FORM_MIXED, lean=1)
    fp64 = _bytes(lib, 16, 10, forms=N.HPS_FORM_FP64)
    assert lean < mixed < both and fp64 < both
    assert _bytes(lib, 16, 10, cluster=0) < both


def test_right_hand_sides_grow_the_krylov_space(lib):
    one, four = _bytes(lib, 8, 10, nrhs=1), _bytes(lib, 8, 10, nrhs=4)
    nf = 8 ** 3 * 6 * 64
    assert four - one >= 3 * 51 * nf * 16  # three more basis columns of 51 vectors


def test_invalid_arguments_give_zero(lib):
    o = N.Options()
    lib.hps_default_options(ctypes.byref(o))
    assert lib.hps_setup_bytes(ctypes.byref(N.Grid(2, 2, 2, 8, 5)), ctypes.byref(o), 1) == 0
    assert lib.hps_setup_bytes(ctypes.byref(N.Grid(2, 2, 2, 8, 6)), ctypes.byref(o), 0) == 0
    o.restart = 0
    assert lib.hps_setup_bytes(ctypes.byref(N.Grid(2, 2, 2, 8, 6)), ctypes.byref(o), 1) == 0
