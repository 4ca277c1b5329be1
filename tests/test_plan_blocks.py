"""Host planning of the shared preconditioner blocks (Sec. 4.1 remark: one local solver for leaves
with nearly the same medium), the step of hps_setup between binning the homogenized constants and
building the blocks, through the C ABI without a GPU.  Integer work, so bit-exact: the block of
every leaf and every cluster equals the partition the oracle's keys give (binned constant and
internal-face mask per leaf; the sequence of its leaves' keys per cluster), numbered in order of
first appearance on both sides."""

import numpy as np
import pytest

import oracle as O
from paper_2112_02211_gb300 import _native as N

hps = pytest.importorskip("paper_2112_02211_gb300")


def _oracle_plan(grid, lam):
    leaf_key = {}
    cl_key = []
    for leaves in O.clusters(grid):
        members = set(leaves)
        key = []
        for leaf in leaves:
            mask = sum(1 << f for f in range(6) if grid.neighbor(leaf, f) in members)
            leaf_key[leaf] = (complex(lam[leaf]), mask)
            key.append(leaf_key[leaf])
        cl_key.append(tuple(key))

    def number(keys):
        seen = {}
        return np.array([seen.setdefault(k, len(seen)) for k in keys], dtype=np.int32)

    return number([leaf_key[i] for i in range(grid.nleaves)]), number(cl_key)


def _lambdas(n, seed, distinct):
    """Constants drawn from `distinct` values (so that many leaves share one), with signed zeros."""
    rng = np.random.default_rng(seed)
    pool = rng.uniform(-2.0, 2.0, distinct) + 1j * rng.choice([0.0, -0.0, 0.5], distinct)
    return pool[rng.integers(0, distinct, n)]


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 2, 5), (1, 1, 1), (5, 3, 2), (2, 7, 1)])
@pytest.mark.parametrize("distinct", [1, 3, 40])
def test_plan_matches_oracle_partition(shape, distinct):
    grid = O.Grid(*shape, 6)
    lam = _lambdas(grid.nleaves, sum(shape) + distinct, distinct)
    leaf_b, cl_k = hps.plan_blocks(*shape, 6, lam)
    ref_b, ref_k = _oracle_plan(grid, lam)
    assert np.array_equal(leaf_b, ref_b)
    assert np.array_equal(cl_k, ref_k)


def test_binned_constants_of_a_smooth_medium():
    """The binning the setup applies (oracle.binned_lambdas) on a smooth field: coarser bins give
    fewer blocks, and the plan follows the oracle's keys at every width."""
    grid = O.Grid(6, 6, 6, 6)
    x = (np.arange(6) + 0.5) / 6
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    # no symmetry, so no two leaves share a constant before binning
    field = (1600.0 * (1.0 - 0.3 * np.sin(2.1 * X + 0.3) * np.cos(1.3 * Y + 0.2) * (Z + 0.37))
             + 25.0j * (1 + np.cos(2.9 * Z + 0.4 * X)))
    lam = np.transpose(field, (2, 1, 0)).reshape(-1)  # leaf id ix + nx (iy + ny iz)
    counts = []
    for delta in (0.0, 0.01, 0.05, 0.2, 10.0):
        lq = O.binned_lambdas(lam, delta)
        leaf_b, cl_k = hps.plan_blocks(6, 6, 6, 6, lq)
        ref_b, ref_k = _oracle_plan(grid, lq)
        assert np.array_equal(leaf_b, ref_b) and np.array_equal(cl_k, ref_k), delta
        counts.append((cl_k.max() + 1, leaf_b.max() + 1))
    assert counts[0] == (27, 216)  # every cluster and leaf distinct
    assert all(a[0] >= b[0] and a[1] >= b[1] for a, b in zip(counts, counts[1:]))
    assert counts[-1] == (1, 8)  # one constant: one cluster block, one B block per mask


def test_signed_zero_is_one_key():
    lam = np.array([1.0 + 0.0j] * 8)
    lam_neg = lam.copy()
    lam_neg[3] = complex(1.0, -0.0)
    a = hps.plan_blocks(2, 2, 2, 6, lam)
    b = hps.plan_blocks(2, 2, 2, 6, lam_neg)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rejects_non_finite_and_bad_sizes():
    lam = np.ones(8, dtype=np.complex128)
    lam[2] = np.nan
    with pytest.raises(N.HPSError):
        hps.plan_blocks(2, 2, 2, 6, lam)
    with pytest.raises(ValueError):
        hps.plan_blocks(2, 2, 2, 6, np.ones(7))
    with pytest.raises(N.HPSError):
        hps.plan_blocks(2, 2, 2, 3, np.ones(8))
