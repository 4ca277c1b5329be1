"""The error bounds the tensor-core tolerances rest on, derived on the CPU by emulating the operand
rounding of kind::tf32 products (10 explicit mantissa bits, round to nearest with ties away from
zero) in numpy.  Accumulation is exact here (FP64), so what is measured is the rounding of the
operands alone: about 2^-22 relative per term with three products (A_hi B_hi + A_hi B_lo +
A_lo B_hi), about 2^-11 with one.  The GPU bars (1e-5 for the three-product multi-RHS apply, 5e-3
for the one-product shared preconditioner blocks) sit above these with room for FP32
accumulation."""

import numpy as np


def tf32(x):
    """Round float32 values to TF32 (1 + 8 + 10 bits), to nearest, ties away from zero."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000  # add half an ulp of the 10-bit mantissa, then truncate
    return u.astype(np.uint32).view(np.float32)


def split(x):
    hi = tf32(x)
    lo = tf32(np.asarray(x, dtype=np.float32) - hi)
    return hi, lo


def _complex_as_real(R):
    """Complex n x n as the real n x 2n matrix of interleaved (re, im) columns."""
    A = np.empty((R.shape[0], 2 * R.shape[1]))
    A[:, 0::2], A[:, 1::2] = R.real, R.imag
    return A


def _operands(F):
    """B^T rows conj(f) and the re/im swap of f, so that A B = [Re(R F) | Im(R F)]."""
    n, k = F.shape
    B = np.empty((2 * n, 2 * k))
    B[0::2, :k], B[1::2, :k] = F.real, -F.imag
    B[0::2, k:], B[1::2, k:] = F.imag, F.real
    return B


def test_tf32_rounding_is_to_nearest():
    x = np.array([1.0, 1.0 + 2.0 ** -11, 1.0 + 2.0 ** -10, 1.0 + 3 * 2.0 ** -11, -1.0 - 2.0 ** -11,
                  3.0e-20], dtype=np.float32)
    y = tf32(x)
    assert y[0] == 1.0 and y[2] == np.float32(1.0 + 2.0 ** -10)
    assert y[1] == np.float32(1.0 + 2.0 ** -10)  # tie: away from zero
    assert y[3] == np.float32(1.0 + 2.0 ** -9)
    assert y[4] == np.float32(-1.0 - 2.0 ** -10)
    r = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    assert np.max(np.abs(tf32(r) - r) / np.abs(r)) <= 2.0 ** -11


def test_complex_as_real_product_is_exact_algebra():
    rng = np.random.default_rng(1)
    R = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    F = rng.standard_normal((12, 4)) + 1j * rng.standard_normal((12, 4))
    G = _complex_as_real(R) @ _operands(F)
    ref = R @ F
    assert np.allclose(G[:, :4], ref.real, atol=1e-12) and np.allclose(G[:, 4:], ref.imag, atol=1e-12)


def test_three_and_one_product_bounds():
    # a leaf map of the multi-RHS size (n_b = 600) against 64 right-hand sides
    rng = np.random.default_rng(2)
    n, k = 600, 64
    R = ((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)).astype(np.complex64)
    F = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))).astype(np.complex64)
    A = _complex_as_real(R.astype(np.complex128)).astype(np.float32)
    B = _operands(F.astype(np.complex128)).astype(np.float32)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    ah, al = split(A)
    bh, bl = split(B)
    f64 = np.float64
    three = ah.astype(f64) @ bh.astype(f64) + ah.astype(f64) @ bl.astype(f64) + al.astype(f64) @ bh.astype(f64)
    one = ah.astype(f64) @ bh.astype(f64)
    err3 = np.linalg.norm(three - exact) / np.linalg.norm(exact)
    err1 = np.linalg.norm(one - exact) / np.linalg.norm(exact)
    assert err3 < 2.0 ** -19  # ~2^-22 per term, random signs
    assert 2.0 ** -16 < err1 < 2.0 ** -10
    # the GPU bars leave room above the operand rounding for FP32 accumulation
    assert err3 < 1e-5 / 10 and err1 < 5e-3 / 5
