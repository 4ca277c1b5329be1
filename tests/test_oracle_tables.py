"""Pins of the oracle's 1D tables, sizes and Kronecker forms against facts the
paper or mathematics fix (no GPU)."""

import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = int(v)
    return vals


@pytest.mark.parametrize("p", [4, 6, 8, 10, 12, 16])
def test_chebyshev_diff_exact_on_polynomials(p):
    x = O.chebyshev_lobatto(p)
    D = O.chebyshev_diff(p)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(p)  # degree p-1 polynomial
    poly = np.polynomial.Polynomial(c)
    err = np.max(np.abs(D @ poly(x) - poly.deriv()(x)))
    assert err < 1e-11 * p ** 2 * np.max(np.abs(c)) * p


@pytest.mark.parametrize("p", [5, 8, 13])
def test_chebyshev_points_are_extrema(p):
    x = O.chebyshev_lobatto(p)
    assert x[0] == -1.0 and abs(x[-1] - 1.0) < 1e-15
    # interior points are the zeros of U_{p-2}, i.e. extrema of T_{p-1}
    T = np.polynomial.chebyshev.Chebyshev.basis(p - 1)
    assert np.max(np.abs(T.deriv()(x[1:-1]))) < 1e-9 * p ** 2


@pytest.mark.parametrize("q", [4, 6, 8, 10, 14])
def test_gauss_legendre_exact_degree(q):
    x, w = O.gauss_legendre(q)
    for m in range(2 * q):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x ** m) - exact) < 1e-13
    # degree 2q is not integrated exactly: the rule really has q points
    assert abs(np.sum(w * x ** (2 * q)) - 2.0 / (2 * q + 1)) > 1e-8


def test_lagrange_matrix_exact_and_invertible():
    for p in (6, 8, 10, 12):
        xc = O.chebyshev_lobatto(p)[1:-1]
        xg, _ = O.gauss_legendre(p - 2)
        Q = O.lagrange_matrix(xc, xg)
        poly = np.polynomial.Polynomial(np.random.default_rng(p).standard_normal(p - 2))
        assert np.max(np.abs(Q @ poly(xc) - poly(xg))) < 1e-12
        assert np.linalg.cond(Q) < 1e4


def test_face_interp_is_2d_tensor_interpolation():
    p = 8
    Pf = O.face_interp(p)
    xc = O.chebyshev_lobatto(p)[1:-1]
    xg, _ = O.gauss_legendre(p - 2)
    # f(a, b) = a^2 b^3 - b, a the first (fastest) in-face coordinate
    f = lambda a, b: a ** 2 * b ** 3 - b
    src = np.array([f(xc[j1], xc[j2]) for j2 in range(p - 2) for j1 in range(p - 2)])
    dst = np.array([f(xg[j1], xg[j2]) for j2 in range(p - 2) for j1 in range(p - 2)])
    assert np.max(np.abs(Pf @ src - dst)) < 1e-12


def test_printed_sizes():
    g = _golden("paper_sizes.txt")
    L = O.LeafLayout(16)
    assert L.nb == g["n_b@n_c=16"]
    assert L.ni == g["n_i@n_c=16"]
    assert O.Grid(4, 4, 4, 16).paper_unknowns() == g["N@4x4x4"]
    assert O.Grid(64, 64, 64, 16).paper_unknowns() == g["N@64x64x64"]


def test_layout_is_a_bijection():
    p = 6
    L = O.LeafLayout(p)
    seen = set()
    for k in range(p):
        for j in range(p):
            for i in range(p):
                if sum(a in (0, p - 1) for a in (i, j, k)) <= 1:
                    seen.add(L.index(i, j, k))
    assert seen == set(range(L.n))


def test_lemma1_kron():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    N = rng.standard_normal((5, 5))
    x = rng.standard_normal(25) + 1j * rng.standard_normal(25)
    assert np.allclose(O.lemma1_apply(M, N, x), np.kron(M, N) @ x, atol=1e-13, rtol=0)


def test_L1_eigenvalues_approach_dirichlet_laplacian():
    # 1D Dirichlet Laplacian on an interval of width h: eigenvalues -(m pi/h)^2.
    h = 0.25
    ev = np.linalg.eigvals(O.interior_L1(16, h))
    assert np.max(np.abs(ev.imag)) < 1e-8 * np.max(np.abs(ev.real))
    ev = np.sort(ev.real)[::-1]
    assert np.all(ev < 0)
    for m in (1, 2, 3):
        exact = -(m * np.pi / h) ** 2
        assert abs(ev[m - 1] - exact) / abs(exact) < 1e-6


@pytest.mark.parametrize("p", [6, 9])
def test_interior_block_three_ways(p):
    """leaf_matrix interior block == np.kron form of eq. (leafmat) == Algorithm 1."""
    h = (0.25, 0.5, 1.0 / 3.0)
    rng = np.random.default_rng(p)
    n1 = p - 2
    c = rng.standard_normal(n1 ** 3) + 1j * rng.standard_normal(n1 ** 3)
    A = O.leaf_matrix(p, h, 3.0, c)[: n1 ** 3, : n1 ** 3]
    Ak = O.dense_Aii(p, h, c)
    assert np.max(np.abs(A - Ak)) < 1e-9 * np.max(np.abs(A))
    v = rng.standard_normal(n1 ** 3) + 1j * rng.standard_normal(n1 ** 3)
    assert np.max(np.abs(O.alg1_apply_Aii(p, h, c, v) - A @ v)) < 1e-9 * np.max(np.abs(A @ v))


def test_alg3_homogenized_inverse():
    p = 8
    h = (0.25, 0.25, 0.25)
    lam = 1600.0 * (1 - 0.2) + 5j
    rng = np.random.default_rng(3)
    v = rng.standard_normal((p - 2) ** 3) + 1j * rng.standard_normal((p - 2) ** 3)
    ref = np.linalg.solve(O.dense_Aii_homog(p, h, lam), v)
    got = O.alg3_apply_Aii_homog_inv(p, h, lam, v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
