"""The multi-RHS and large configurations at their full sizes, on sampled outputs the oracle
computes one leaf at a time (the benchmark workload has its own file, test_gpu_fullsize.py):

* multi-RHS: 16^3 leaves, p = 12, kappa = eta = 60, five bumps, 64 Gaussian sources, lean mixed
  form with 2x2x2 clusters at lambda_bin 0.01 (stage K of all 64 right-hand sides on the tensor
  cores), the apply of all 64 right-hand sides on the tensor cores, tol 1e-6;
* large: 32^3 leaves, p = 10, kappa = eta = 200, smooth random complex medium, lean mixed form with
  2x2x2 clusters at lambda_bin 0.01, tol 1e-5.

Checks per configuration: sampled leaf maps (FP32 storage: 1e-6); for the multi-RHS case the
tensor-core apply on sampled blocks (1e-5 of |R| |f|, the truncating accumulation of the tensor
cores); the solution: converged, and its global FP64 residual b - A f formed on the GPU (lean
mode: FP32 maps plus FP16 remainders, FP64-accurate) within the tolerance.  On sampled face
blocks the oracle forms b and the residual from its own maps, each block compared with the GPU's
at that block's own scale: 1e-9 of |H| |s| and of |R| |f| + |b| (FP64-accurate maps on both
sides), so one wrong block cannot hide behind the global norm.

Skipped unless HPS_FULLSIZE_CONFIGS=1: the two setups take about 3.5 and 6.5 minutes on one
GB300 and hold up to 155 GB."""

import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.discretization import _leaf_node_coords

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("HPS_FULLSIZE_CONFIGS") != "1",
                                 reason="full-size multi-RHS and large configurations: set HPS_FULLSIZE_CONFIGS=1")]

hps = pytest.importorskip("paper_2112_02211_gb300")


def _interior(grid):
    """The oracle's interior nodes of one leaf at a time (the whole grid's take minutes here)."""
    def xi(leaf):
        return _leaf_node_coords(grid.p, grid.h, grid.corner(leaf))[: grid.layout.ni]
    return xi


def _maps(w, grid, leaf, xi_or):
    return O.leaf_iti(grid.p, grid.h, w.eta, O.cdiag_from_b(w.kappa, w.sample_b(xi_or(leaf))))


def _source_leaf(grid, x):
    ix, iy, iz = (min(int(x[a] * n), n - 1) for a, n in enumerate((grid.nx, grid.ny, grid.nz)))
    return grid.leaf_id(ix, iy, iz)


def _samples(grid, rng, near, count):
    """(leaf, face) pairs with a neighbour: the faces of the leaves in `near`, then random ones."""
    out = [(leaf, f) for leaf in near for f in range(6) if grid.neighbor(leaf, f) >= 0]
    while len(out) < len(near) * 6 + count:
        leaf, f = int(rng.integers(grid.nleaves)), int(rng.integers(6))
        if grid.neighbor(leaf, f) >= 0:
            out.append((leaf, f))
    return out


def _check_rows(w, grid, xi_or, samples, bh, rh, f, s_or_leaf):
    """bh, rh, f: (nrhs, nleaves, 6, q^2) GPU right-hand side, GPU residual b - A f and solution;
    s_or_leaf(leaf) -> the oracle's body loads of one leaf, (nrhs, n_i).  Every sampled block of
    b and of the residual, formed by the oracle from its own maps, must match the GPU's block to
    1e-9 of the block's own scale."""
    q2 = grid.q * grid.q
    cache = {}
    for leaf, face in samples:
        nbr = grid.neighbor(leaf, face)
        if nbr not in cache:
            cache[nbr] = _maps(w, grid, nbr, xi_or)
        R, H = cache[nbr]
        rows = slice((face ^ 1) * q2, ((face ^ 1) + 1) * q2)
        s_n = s_or_leaf(nbr)
        for r in range(f.shape[0]):
            b_slot = -(H[rows, :] @ s_n[r])
            babs = np.abs(H[rows, :]) @ np.abs(s_n[r])
            assert np.linalg.norm(bh[r, leaf, face] - b_slot) <= 1e-9 * np.linalg.norm(babs) + 1e-300, (leaf, face, r)
            fn = f[r, nbr].reshape(-1)
            res = b_slot - (f[r, leaf, face] + R[rows, :] @ fn)
            scale = np.linalg.norm(np.abs(R[rows, :]) @ np.abs(fn)) + np.linalg.norm(b_slot)
            assert np.linalg.norm(res - rh[r, leaf, face]) <= 1e-9 * scale, (leaf, face, r)


def _gpu_residual(solver, bg, f):
    """b - (I + Pi R) f on the GPU (complex double; lean mode: the compensated FP32 maps)."""
    return bg - solver.apply(f)


def test_multi_rhs_configuration_at_full_size():
    w = W.multi_rhs_16cubed()
    L, p, nrhs = w.nx, w.p, w.nrhs
    xi, xf = hps.nodes(L, L, L, p)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    grid = O.Grid(L, L, L, p)
    xi_or = _interior(grid)
    solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi), forms=("mixed",), lean=True,
                        max_rhs=nrhs, lambda_bin=0.01)
    try:
        rng = np.random.default_rng(31)
        for leaf in rng.choice(grid.nleaves, 2, replace=False):
            R, _ = _maps(w, grid, int(leaf), xi_or)
            assert np.linalg.norm(solver.export("R", int(leaf)).reshape(grid.nb, grid.nb) - R) <= \
                1e-6 * np.linalg.norm(R)
        # the tensor-core apply of 64 right-hand sides on sampled face blocks
        F = (rng.standard_normal((nrhs, grid.nf)) + 1j * rng.standard_normal((nrhs, grid.nf))).astype(np.complex64)
        y = solver.apply(torch.from_numpy(F.reshape(-1)).cuda()).cpu().numpy().reshape(nrhs, grid.nleaves, 6, -1)
        Fl = F.reshape(nrhs, grid.nleaves, 6, -1).astype(np.complex128)
        q2 = grid.q * grid.q
        for leaf, face in _samples(grid, rng, [], 6):
            nbr = grid.neighbor(leaf, face)
            R, _ = _maps(w, grid, nbr, xi_or)
            rows = slice((face ^ 1) * q2, ((face ^ 1) + 1) * q2)
            ref = Fl[:, leaf, face] + Fl[:, nbr].reshape(nrhs, -1) @ R[rows, :].T
            absprod = np.abs(Fl[:, nbr].reshape(nrhs, -1)) @ np.abs(R[rows, :]).T
            assert np.linalg.norm(y[:, leaf, face] - ref) <= 1e-5 * np.linalg.norm(absprod), (leaf, face)
        # the solve: converged, global FP64 residual, sampled blocks against the oracle's maps
        f, info = solver.solve(s=s, tol=w.tol, form="mixed", nrhs=nrhs)
        assert info["converged"], info
        bg = solver.rhs(s, nrhs=nrhs)
        rg = _gpu_residual(solver, bg, f)
        rel_res = (rg.reshape(nrhs, -1).norm(dim=1) / bg.reshape(nrhs, -1).norm(dim=1)).cpu().numpy()
        assert np.all(rel_res <= w.tol * (1 + 1e-6)), rel_res.max()
        pick = [0, 31, 63]
        shape = (nrhs, grid.nleaves, 6, -1)
        fh = f.cpu().numpy().reshape(shape)[pick]
        bh = bg.cpu().numpy().reshape(shape)[pick]
        rh = rg.cpu().numpy().reshape(shape)[pick]
        src = np.array(w.meta["sources"])
        near = [_source_leaf(grid, src[k]) for k in pick]

        def s_or_leaf(leaf):
            return w.sample_s(xi_or(leaf))[pick]

        _check_rows(w, grid, xi_or, _samples(grid, rng, near, 6), bh, rh, fh, s_or_leaf)
    finally:
        solver.close()


def test_large_configuration_at_full_size():
    w = W.large_32cubed()
    L, p = w.nx, w.p
    xi, xf = hps.nodes(L, L, L, p)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    grid = O.Grid(L, L, L, p)
    xi_or = _interior(grid)
    solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi), forms=("mixed",), lean=True,
                        lambda_bin=0.01)
    try:
        rng = np.random.default_rng(32)
        for leaf in rng.choice(grid.nleaves, 2, replace=False):
            R, _ = _maps(w, grid, int(leaf), xi_or)
            assert np.linalg.norm(solver.export("R", int(leaf)).reshape(grid.nb, grid.nb) - R) <= \
                1e-6 * np.linalg.norm(R)
        f, info = solver.solve(s=s, tol=w.tol, form="mixed")
        assert info["converged"], info
        bg = solver.rhs(s)
        rg = _gpu_residual(solver, bg, f)
        assert float(rg.norm() / bg.norm()) <= w.tol * (1 + 1e-6)
        shape = (1, grid.nleaves, 6, -1)
        fh = f.cpu().numpy().reshape(shape)
        bh = bg.cpu().numpy().reshape(shape)
        rh = rg.cpu().numpy().reshape(shape)
        near = [_source_leaf(grid, [0.5, 0.5, 0.5])]

        def s_or_leaf(leaf):
            return w.sample_s(xi_or(leaf))

        _check_rows(w, grid, xi_or, _samples(grid, rng, near, 8), bh, rh, fh, s_or_leaf)
    finally:
        solver.close()
