"""Shared preconditioner blocks (binned homogenized constants, Sec. 4.1 remark) on
the GPU against the oracle's preconditioner built from the same binned constants.

Bars as for the unshared preconditioner: FP64 blocks 1e-9, FP16 blocks 5e-3; the
number of distinct blocks equals the number of distinct (binned constant,
internal-face mask) keys the oracle's values give; the solve still reaches the
oracle's solution."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")

DELTAS = (0.0, 0.02, 0.2)


def _workload():
    # 4^3 leaves (8 clusters) of the bump medium: leaves far from the bump have nearly
    # equal constants, leaves on it do not.
    return W.scaled(W.bump_16cubed(p=6, kappa=10.0), 4)


def _keys(grid, lam):
    """Distinct leaf keys (constant, internal-face mask) and cluster keys."""
    leaf_key = {}
    cl_keys = set()
    for leaves in O.clusters(grid):
        members = set(leaves)
        key = []
        for leaf in leaves:
            mask = sum(1 << f for f in range(6) if grid.neighbor(leaf, f) in members)
            k = (complex(lam[leaf]), mask)
            leaf_key[leaf] = k
            key.append(k)
        cl_keys.add(tuple(key))
    return len(set(leaf_key.values())), len(cl_keys)


@pytest.fixture(scope="module")
def case():
    w = _workload()
    grid = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi = O.interior_nodes(grid)
    b_or = w.sample_b(xi)
    prob = O.build_problem(grid, w.kappa, w.eta, b_or)
    xi_g, xf_g, b, s, t = gpu_inputs(w, hps)
    return w, grid, b_or, prob, b, s


@pytest.mark.parametrize("delta", DELTAS)
def test_binned_precond_matches_oracle(case, delta):
    w, grid, b_or, prob, b, s = case
    hom = O.build_problem(grid, w.kappa, w.eta, b_or, homogenized=True, lambda_bin=delta)
    M = O.Preconditioner(grid, hom.R)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, max_rhs=3, lambda_bin=delta)
    try:
        nb_leaf, nb_cl = _keys(grid, hom.lam)
        ncl, k_blocks, b_blocks = solver.precond_info()
        assert ncl == len(O.clusters(grid))
        assert (k_blocks, b_blocks) == (nb_cl, nb_leaf)
        rng = np.random.default_rng(7)
        r = rng.standard_normal((3, grid.nf)) + 1j * rng.standard_normal((3, grid.nf))
        ref = np.stack([M(r[i]) for i in range(3)])
        z = solver.precond(torch.from_numpy(r.reshape(-1)).cuda()).cpu().numpy().reshape(3, -1)
        assert rel(z, ref) < 1e-9
        for i in range(3):
            assert rel(z[i], ref[i]) < 1e-9
        r32 = r[0].astype(np.complex64)
        z16 = solver.precond(torch.from_numpy(r32).cuda(), fp16_blocks=True).cpu().numpy()
        assert rel(z16, M(r32.astype(np.complex128))) < 5e-3
    finally:
        solver.close()


def test_coarse_bins_share_blocks_and_keep_the_solution(case):
    w, grid, b_or, prob, b, s = case
    rhs = O.rhs_face(grid, prob.H, w.sample_s(O.interior_nodes(grid))[0], None)
    f_ref, _, _ = O.gmres(lambda v: O.apply_face(grid, prob.R, v), rhs, tol=1e-13, restart=50)
    its = {}
    for delta in (0.0, 0.2):
        solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",),
                            lambda_bin=delta)
        try:
            f, info = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), tol=1e-8, form="mixed")
            assert info["converged"]
            assert rel(f.cpu().numpy(), f_ref) < 1e-6
            its[delta] = (info["iterations"], solver.precond_info())
        finally:
            solver.close()
    ncl, k0, _ = its[0.0][1]
    _, k1, b1 = its[0.2][1]
    assert k1 < k0 and b1 < grid.nleaves
    assert its[0.2][0] <= its[0.0][0] + 5


def _tc_workload():
    # b = 0: every leaf has the same constant, so 11 x 8 x 8 leaves give one block of 80
    # 2x2x2 clusters (two member tiles of 64, the second ragged) and one of 16 edge
    # clusters 1x2x2 (smaller block), both on the tensor-core path
    w = W.plane_wave(L=8, p=6, kappa=8.0)
    w.nx = 11
    return w


@pytest.fixture(scope="module")
def tc_case():
    w = _tc_workload()
    grid = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi = O.interior_nodes(grid)
    b_or = w.sample_b(xi)
    hom = O.build_problem(grid, w.kappa, w.eta, b_or, homogenized=True)
    M = O.Preconditioner(grid, hom.R)
    xi_g, xf_g, b, s, t = gpu_inputs(w, hps)
    return w, grid, M, b, t


def test_shared_blocks_on_tensor_cores_match_oracle(tc_case):
    """Complex-FP32 blocks through one TF32 product per term (both operands rounded to
    10-bit mantissas): the FP16-block bar on the tensor-core path, the FP32 bar without it."""
    w, grid, M, b, t = tc_case
    rng = np.random.default_rng(17)
    r = (rng.standard_normal(grid.nf) + 1j * rng.standard_normal(grid.nf)).astype(np.complex64)
    ref = M(r.astype(np.complex128))
    out = {}
    for tc in (True, False):
        solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), tc_apply=tc)
        try:
            assert solver.precond_info() == (96, 2, len({(m,) for m in _masks(grid)}))
            z = solver.precond(torch.from_numpy(r).cuda()).cpu().numpy()
            assert rel(z, ref) < (5e-3 if tc else 2e-5), tc
            out[tc] = z
        finally:
            solver.close()
    assert 0 < rel(out[True], out[False]) < 5e-3


def test_solve_with_tensor_core_blocks(tc_case):
    w, grid, M, b, t = tc_case
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",))
    try:
        f, info = solver.solve(t=torch.from_numpy(t.reshape(-1)).cuda(), tol=1e-8, form="mixed")
        assert info["converged"]
        xi, xf = O.interior_nodes(grid), O.face_nodes(grid)
        nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
        prob = O.build_problem(grid, w.kappa, w.eta, w.sample_b(xi))
        rhs = O.rhs_face(grid, prob.H, None, w.sample_t(xf, nrm)[0])
        f_ref, _, _ = O.gmres(lambda v: O.apply_face(grid, prob.R, v), rhs, tol=1e-12, restart=50)
        assert rel(f.cpu().numpy(), f_ref) < 1e-6
    finally:
        solver.close()


def _masks(grid):
    out = []
    for leaves in O.clusters(grid):
        members = set(leaves)
        for leaf in leaves:
            out.append(sum(1 << f for f in range(6) if grid.neighbor(leaf, f) in members))
    return out


def test_lean_mode_keeps_shared_blocks_on_tensor_cores(tc_case):
    """Lean mode keeps FP16 blocks for the SIMT stage and complex-FP32 copies of the widely
    shared blocks for the tensor cores; both preconditioner forms and the lean solve meet
    the bars of the non-lean handle."""
    w, grid, M, b, t = tc_case
    rng = np.random.default_rng(19)
    r = (rng.standard_normal(grid.nf) + 1j * rng.standard_normal(grid.nf)).astype(np.complex64)
    ref = M(r.astype(np.complex128))
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), lean=True)
    try:
        assert solver.precond_info() == (96, 2, len({(m,) for m in _masks(grid)}))
        z = solver.precond(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel(z, ref) < 5e-3
        z16 = solver.precond(torch.from_numpy(r).cuda(), fp16_blocks=True).cpu().numpy()
        assert rel(z16, ref) < 5e-3
        # the restart residual uses the FP32 maps plus their FP16 remainders with double-float
        # accumulation (FP64-accurate), so lean solves meet the mixed form's bar
        f, info = solver.solve(t=torch.from_numpy(t.reshape(-1)).cuda(), tol=1e-8, form="mixed")
        assert info["converged"], info
        xi, xf = O.interior_nodes(grid), O.face_nodes(grid)
        nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
        prob = O.build_problem(grid, w.kappa, w.eta, w.sample_b(xi))
        rhs = O.rhs_face(grid, prob.H, None, w.sample_t(xf, nrm)[0])
        f_ref, _, _ = O.gmres(lambda v: O.apply_face(grid, prob.R, v), rhs, tol=1e-12, restart=50)
        assert rel(f.cpu().numpy(), f_ref) < 1e-6
    finally:
        solver.close()
