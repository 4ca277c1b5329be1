"""Pins of the locally homogenized constant lambda^tau of Sec. 4.1 in the oracle (no GPU).

The paper replaces the leaf's varying C_ii = kappa^2 (1 - b) by one constant: the average of
the largest and the smallest diagonal entry.  For complex C (Im b > 0) the reading taken is the
midrange of the real parts plus i times the midrange of the imaginary parts.  The values below
are worked by hand; the brute-force pin characterizes the midrange without its formula (it is
the constant that minimizes the largest deviation max_i |C_ii - lambda| over real C), so a mean,
a missing 1/2 or a swapped real/imaginary part fails at least one of them.
"""

import numpy as np

import oracle as O


def test_real_diagonal_midrange_by_hand():
    # max 7, min -1: (7 + (-1)) / 2 = 3; the mean (3.5) and max + min (6) are different
    assert O.homogenized_lambda(np.array([3.0, 7.0, -1.0, 5.0])) == 3.0
    # an even count where mean and median differ from the midrange too: (10 + 0) / 2 = 5
    assert O.homogenized_lambda(np.array([0.0, 1.0, 2.0, 10.0])) == 5.0


def test_complex_diagonal_takes_real_and_imaginary_extremes_separately():
    # Re in {1, 5, 3}: (5 + 1)/2 = 3; Im in {10, 2, 4}: (10 + 2)/2 = 6.  The entry with the
    # largest real part (5+2j) is not the one with the largest imaginary part (1+10j).
    lam = O.homogenized_lambda(np.array([1 + 10j, 5 + 2j, 3 + 4j]))
    assert lam == 3 + 6j
    # negative imaginary parts: Im in {-3, 1}: (1 - 3)/2 = -1; Re in {2, 2}: 2
    assert O.homogenized_lambda(np.array([2 - 3j, 2 + 1j])) == 2 - 1j


def test_constant_diagonal_is_its_own_constant():
    for c in (7.0 - 2.0j, -40.5 + 0.0j, 1600.0 + 0.25j):
        assert O.homogenized_lambda(np.full(27, c)) == c


def test_helmholtz_constant_for_the_bump_medium():
    # C = kappa^2 (1 - b): b in [0, 1.5] at kappa = 40 gives C in [1600 (1 - 1.5), 1600] =
    # [-800, 1600], so lambda = (1600 - 800) / 2 = 400; b = 0 gives kappa^2.
    kappa = 40.0
    b = np.array([0.0, 0.3, 1.5, 0.9])
    assert O.homogenized_lambda(O.cdiag_from_b(kappa, b)) == 400.0
    assert O.homogenized_lambda(O.cdiag_from_b(kappa, np.zeros(8))) == kappa * kappa


def test_midrange_minimizes_the_largest_deviation():
    """For real values the midrange is the unique minimizer of max_i |c_i - lambda| (the
    Chebyshev centre of the interval [min c, max c]); found here by brute force over a fine grid,
    with no reference to the formula."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        c = rng.uniform(-50.0, 120.0, 9)
        grid = np.linspace(-60.0, 130.0, 190001)  # spacing 1e-3
        dev = np.max(np.abs(c[None, :] - grid[:, None]), axis=1)
        best = grid[np.argmin(dev)]
        assert abs(O.homogenized_lambda(c) - best) <= 1e-3
