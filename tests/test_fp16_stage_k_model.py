"""CPU model of the FP16 tensor-core stage K (z_int = K_c t on tcgen05 kind::f16), from which the
bars of its GPU test (tests/test_gpu_multi_rhs.py::test_fp16_tensor_core_stage_k) follow.

What the kernel computes, per cluster block K_c (n x n complex) and member t (n complex):
* A = K_c with every row divided by its largest |re|, |im| (the FP32 row scale s_row) and rounded
  to FP16, read as the real n x 2n matrix of interleaved (re, im) columns;
* x = t / t_max (t_max = the largest |re|, |im| of the cluster's t, 0 below 2^-126), split into
  two FP16 terms hi = fp16(x), lo = fp16(x - hi), each laid out as the B rows conj and re/im swap;
* per K chunk of 16 halves two MMAs into one FP32 accumulator, D += A B_hi then D += A B_lo, each
  modelled as the truncating block FMA of tests/tc_model.py;
* z = D s_row t_max.

Checks: the error against the exact K_c t is the FP16 rounding of K_c (~2^-12 relative per
entry), far inside the GPU test's 5e-3; the result is linear in t to ~1e-6 (the GPU test's bar
is 3e-5), while one FP16 rounding of t (no lo term) breaks linearity at ~1e-4, above that bar; a
cluster whose t is all subnormal yields 0."""

import numpy as np
import pytest

import tc_model as T


def _fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def _quantize_rows(K):
    s = np.maximum(np.abs(K.real), np.abs(K.imag)).max(axis=1).astype(np.float32)
    s = np.where(s > 0, s, 1.0).astype(np.float32)
    inv = (np.float32(1.0) / s).astype(np.float32)
    Kq = _fp16(K.real.astype(np.float32) * inv[:, None]) + 1j * _fp16(K.imag.astype(np.float32) * inv[:, None])
    return Kq, s


def _split_t(t, two_terms=True):
    tf = t.astype(np.complex64)
    tmax = np.float32(max(np.abs(tf.real).max(), np.abs(tf.imag).max()))
    if not tmax >= np.float32(2.0 ** -126):
        return None, None, np.float32(0.0)
    sc = np.float32(1.0) / tmax
    xr, xi = tf.real.astype(np.float32) * sc, tf.imag.astype(np.float32) * sc
    hr, hi_ = _fp16(xr), _fp16(xi)
    if two_terms:
        lr, li = _fp16(xr - hr), _fp16(xi - hi_)
    else:
        lr, li = np.zeros_like(hr), np.zeros_like(hi_)
    return hr + 1j * hi_, lr + 1j * li, tmax


def model_stage_k(K, t, two_terms=True, kblk=8, extra=2):
    """z = K t as the kernel computes it (one member), under the block-FMA model."""
    Kq, s = _quantize_rows(K)
    th, tl, tmax = _split_t(t, two_terms)
    if th is None:
        return np.zeros(K.shape[0], dtype=np.complex128)
    A = T.complex_as_real(Kq).astype(np.float64)
    Bh = T.operands(th[:, None]).astype(np.float64)
    Bl = T.operands(tl[:, None]).astype(np.float64)
    n2 = A.shape[1]
    D = np.zeros((A.shape[0], 2))
    for k0 in range(0, n2, 16):
        for B in (Bh, Bl):
            for j0 in range(k0, min(k0 + 16, n2), kblk):
                p = A[:, None, j0:j0 + kblk] * B.T[None, :, j0:j0 + kblk]
                D = T.block_fma(D, p, extra)
    f = s.astype(np.float64) * np.float64(tmax)
    return (D[:, 0] + 1j * D[:, 1]) * f


def _case(n, seed):
    rng = np.random.default_rng(seed)
    # a well-scaled dense block with rows of different magnitudes (the row scales matter)
    K = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * np.exp(rng.uniform(-3, 3, n))[:, None]
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return K, x, y


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,kblk", [(96, 8), (96, 16), (384, 8)])
def test_error_is_the_fp16_rounding_of_the_block(n, kblk):
    K, x, _ = _case(n, n + kblk)
    z = model_stage_k(K, x, kblk=kblk)
    exact = K @ x
    e = _rel(z, exact)
    # K_c rounded to FP16 (2^-12 relative per entry, random signs): ~2^-12 overall, well inside
    # the GPU test's 5e-3 against the oracle
    assert 1e-5 < e < 1e-3, e
    # with an exact K_c what is left is the two-term t (~2^-23) and the accumulation: each of the
    # 2 (2n / 8) block additions truncates toward zero by less than one FP32 unit of |D|
    Kq, s = _quantize_rows(K)
    zq = model_stage_k(Kq * s[:, None], x, kblk=kblk)
    assert _rel(zq, (Kq * s[:, None]) @ x) < (n / 2) * 2.0 ** -23


@pytest.mark.parametrize("n", [96, 384])
def test_two_fp16_terms_keep_it_linear(n):
    K, x, y = _case(n, 7 * n)
    lin = {}
    for two in (True, False):
        zx, zy = model_stage_k(K, x, two), model_stage_k(K, y, two)
        zxy = model_stage_k(K, x + 0.5 * y, two)
        lin[two] = _rel(zx + 0.5 * zy, zxy)
    assert lin[True] < 3e-5 / 10, lin       # the GPU test's bar, with a margin of 10
    assert lin[False] > 3e-5, lin           # one FP16 term would fail that bar


def test_subnormal_cluster_gives_zero():
    K, x, _ = _case(96, 3)
    tiny = (x / np.abs(x).max() * 3e-40).astype(np.complex64)
    assert np.abs(tiny).max() > 0  # subnormal, not flushed
    assert np.all(model_stage_k(K, tiny) == 0)
    # a normal but small scale still works
    small = (x * 1e-30).astype(np.complex64)
    assert _rel(model_stage_k(K, small), K @ small.astype(np.complex128)) < 1e-3
