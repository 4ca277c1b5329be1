"""The benchmark workload at its full size (16^3 leaves, p = 10, kappa = eta = 40, the bump
medium and Gaussian source; the handle bench.py times: both forms, shared preconditioner blocks at
lambda_bin 0.01) against the oracle on sampled outputs that it computes one leaf at a time.

* leaf maps R, H of sampled leaves: 1e-11 (as in the small parity cases);
* the mixed-form solution's FP64 residual b - (I + Pi R) f: below the tolerance globally, and on
  sampled face blocks the GPU's residual rows equal the oracle's, formed from the oracle's own
  maps of the neighbouring leaves: 1e-9 of the local terms before cancellation (both FP64; the
  map difference of ~1e-11 relative, times |R| |f|)."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


@pytest.fixture(scope="module")
def full():
    w = W.bump_16cubed()
    L, p = w.nx, w.p
    xi, xf = hps.nodes(L, L, L, p)
    b = w.sample_b(xi)
    s = w.sample_s(xi).reshape(-1)
    solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=b, lambda_bin=0.01)
    grid = O.Grid(L, L, L, p)
    b_or = w.sample_b(O.interior_nodes(grid))
    s_or = w.sample_s(O.interior_nodes(grid))[0]
    yield w, solver, grid, b_or, s_or, s
    solver.close()


def _maps(w, grid, b_or, leaf):
    return O.leaf_iti(grid.p, grid.h, w.eta, O.cdiag_from_b(w.kappa, b_or[leaf]))


def test_sampled_leaf_maps_at_full_size(full):
    w, solver, grid, b_or, s_or, s = full
    rng = np.random.default_rng(21)
    for leaf in rng.choice(grid.nleaves, 3, replace=False):
        R, H = _maps(w, grid, b_or, int(leaf))
        assert rel(solver.export("R", int(leaf)).reshape(grid.nb, grid.nb), R) < 1e-11
        assert rel(solver.export("H", int(leaf)).reshape(grid.nb, -1), H) < 1e-11


def test_full_size_solution_residual_against_oracle_rows(full):
    w, solver, grid, b_or, s_or, s = full
    sd = torch.from_numpy(s).cuda()
    f, info = solver.solve(s=sd, tol=w.tol, form="mixed")
    assert info["converged"] and info["iterations"] > 0, info
    bg = solver.rhs(sd)
    r = (bg - solver.apply(f)).cpu().numpy().reshape(grid.nleaves, 6, -1)
    bh = bg.cpu().numpy()
    assert np.linalg.norm(r) <= w.tol * np.linalg.norm(bh)
    fh = f.cpu().numpy().reshape(grid.nleaves, 6, -1)
    bh = bh.reshape(grid.nleaves, 6, -1)
    q2 = grid.q * grid.q
    rng = np.random.default_rng(22)
    checked = 0
    while checked < 8:
        leaf, face = int(rng.integers(grid.nleaves)), int(rng.integers(6))
        nbr = grid.neighbor(leaf, face)
        if nbr < 0:
            continue
        R, H = _maps(w, grid, b_or, nbr)
        rows = slice((face ^ 1) * q2, ((face ^ 1) + 1) * q2)
        # incoming data of leaf's face = -(outgoing data of nbr on the opposite face)
        y = fh[leaf, face] + R[rows, :] @ fh[nbr].reshape(-1)
        b_slot = -(H[rows, :] @ s_or[nbr])
        r_or = b_slot - y
        # rounding is relative to the terms before cancellation (far from the source y is
        # a small difference of the two incoming contributions)
        absprod = np.abs(R[rows, :]) @ np.abs(fh[nbr].reshape(-1))
        scale = np.linalg.norm(b_slot) + np.linalg.norm(fh[leaf, face]) + np.linalg.norm(absprod)
        assert np.linalg.norm(r_or - r[leaf, face]) <= 1e-9 * scale, (leaf, face)
        babs = np.abs(H[rows, :]) @ np.abs(s_or[nbr])
        assert np.linalg.norm(b_slot - bh[leaf, face]) <= 1e-9 * np.linalg.norm(babs), (leaf, face)
        checked += 1
