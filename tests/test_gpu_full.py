"""The paper's own iterative path on the global system (Sec. 3-4) on the GPU
against the oracle (oracle/full_iterative.py), element by element.

Bars: FP64 apply 1e-12 (the same collocation sums in a different order), FP32
apply 2e-6; FP64 preconditioner 1e-9 (Algorithm 3's eigenvector basis and S~^{-1}
from the elimination amplify rounding by their condition numbers), FP32
preconditioner 1e-4; FP64 solve 1e-10 and mixed solve 1e-6 against the dense
global solution, whose incoming data also equals the face-system solution."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


def _workload():
    # 3 x 2 x 2 leaves (an odd axis), p = 7, the manufactured solution in the bump medium
    w = W.manufactured(L=2, p=7, kappa=9.0)
    w.nx, w.ny, w.nz = 3, 2, 2
    return w


@pytest.fixture(scope="module")
def case():
    w = _workload()
    grid = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi, xf = O.interior_nodes(grid), O.face_nodes(grid)
    nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
    b_or = w.sample_b(xi)
    cd = [O.cdiag_from_b(w.kappa, b_or[i]) for i in range(grid.nleaves)]
    xi_g, xf_g, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, full_system=True, max_rhs=2)
    oc = {"grid": grid, "cd": cd, "b": b_or, "s": w.sample_s(xi)[0], "t": w.sample_t(xf, nrm)[0]}
    yield w, oc, solver, (s, t)
    solver.close()


def _rand(n, seed, k=1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))


def test_full_apply_matches_oracle(case):
    w, oc, solver, _ = case
    grid = oc["grid"]
    u = _rand(grid.nleaves * grid.layout.n, 1, 2)
    ref = np.stack([O.full_apply(grid, w.eta, oc["cd"], u[i]) for i in range(2)])
    y = solver.full_apply(torch.from_numpy(u.reshape(-1)).cuda()).cpu().numpy().reshape(2, -1)
    assert rel(y, ref) < 1e-12
    y32 = solver.full_apply(torch.from_numpy(u.reshape(-1).astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y32.reshape(2, -1), ref) < 2e-6


def test_full_precond_matches_oracle(case):
    w, oc, solver, _ = case
    grid = oc["grid"]
    M = O.FullBlockJacobi(grid, w.eta, O.full_lambdas(grid, w.kappa, oc["b"]))
    r = _rand(grid.nleaves * grid.layout.n, 2, 2)
    ref = np.stack([M(r[i]) for i in range(2)])
    z = solver.full_precond(torch.from_numpy(r.reshape(-1)).cuda()).cpu().numpy().reshape(2, -1)
    assert rel(z, ref) < 1e-9
    z32 = solver.full_precond(torch.from_numpy(r.reshape(-1).astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(z32.reshape(2, -1), ref) < 1e-4


def test_full_precond_with_binned_constants(case):
    w, oc, _, _ = case
    grid = oc["grid"]
    lams = O.binned_lambdas(O.full_lambdas(grid, w.kappa, oc["b"]), 0.05)
    M = O.FullBlockJacobi(grid, w.eta, lams)
    xi_g, xf_g, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, full_system=True, lambda_bin=0.05)
    try:
        r = _rand(grid.nleaves * grid.layout.n, 3)[0]
        z = solver.full_precond(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel(z, M(r)) < 1e-9
    finally:
        solver.close()


@pytest.mark.parametrize("form,tol,bar", [("fp64", 1e-12, 1e-10), ("mixed", 1e-8, 1e-6)])
def test_full_solve_matches_oracle(case, form, tol, bar):
    w, oc, solver, (s, t) = case
    grid = oc["grid"]
    u_ref, f_ref = O.full_system_solve(grid, w.eta, oc["cd"], oc["s"].reshape(grid.nleaves, -1),
                                       oc["t"].reshape(grid.nleaves, 6, -1))
    u, info = solver.full_solve(s=torch.from_numpy(s.reshape(-1)).cuda(), t=torch.from_numpy(t.reshape(-1)).cuda(),
                                tol=tol, form=form)
    assert info["converged"], info
    u = u.cpu().numpy()
    assert rel(u, u_ref.reshape(-1)) < bar, info
    # the global solution's incoming data is the face-system solution
    f_face, _ = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), t=torch.from_numpy(t.reshape(-1)).cuda(),
                             tol=1e-12, form="fp64")
    assert rel(O.full_to_face(grid, w.eta, u), f_face.cpu().numpy()) < 10 * bar


def test_full_solve_preconditioner_cuts_iterations(case):
    w, oc, solver, (s, t) = case
    sd, td = torch.from_numpy(s.reshape(-1)).cuda(), torch.from_numpy(t.reshape(-1)).cuda()
    _, with_pc = solver.full_solve(s=sd, t=td, tol=1e-8, form="mixed")
    _, without = solver.full_solve(s=sd, t=td, tol=1e-8, form="mixed", precond=False)
    assert with_pc["converged"]
    assert with_pc["iterations"] < without["iterations"]
