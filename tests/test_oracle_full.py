"""Pins of the oracle's iterative path on the paper's global system (Sec. 3-4):
the matrix-free apply against the assembled matrix and against the closed-form
solution, the Schur/Algorithm-3 block solve against a dense solve, and
preconditioned GMRES against the dense global solution and the face system (no GPU)."""

import numpy as np

import oracle as O
import workloads as W


def _case(w, nx, ny, nz):
    grid = O.Grid(nx, ny, nz, w.p)
    xi, xf = O.interior_nodes(grid), O.face_nodes(grid)
    nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
    b = w.sample_b(xi)
    cd = [O.cdiag_from_b(w.kappa, b[i]) for i in range(grid.nleaves)]
    s = w.sample_s(xi)[0]
    t = w.sample_t(xf, nrm)[0]
    return grid, xi, xf, nrm, b, cd, s, t


def test_matrix_free_apply_equals_assembled_matrix():
    w = W.manufactured(L=2, p=6, kappa=7.0)
    grid, xi, xf, nrm, b, cd, s, t = _case(w, 2, 1, 2)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(grid.nleaves * grid.layout.n) + 1j * rng.standard_normal(grid.nleaves * grid.layout.n)
    A = O.full_system_matrix(grid, w.eta, cd)
    assert np.allclose(O.full_apply(grid, w.eta, cd, u), A @ u, rtol=0, atol=1e-9 * np.abs(A @ u).max())


def test_exact_solution_satisfies_the_global_system_spectrally():
    """A u_exact - rhs (u_exact at interior and Chebyshev face nodes) falls spectrally in p."""
    res = []
    for p in (6, 8, 10):
        w = W.manufactured(L=2, p=p, kappa=6.0)
        grid, xi, xf, nrm, b, cd, s, t = _case(w, 2, 2, 2)
        xc = O.cheb_face_nodes(grid)
        ue = np.concatenate([np.concatenate([w.meta["u"](xi[i]), w.meta["u"](xc[i]).reshape(-1)])
                             for i in range(grid.nleaves)])
        rhs = O.full_rhs(grid, s, t)
        r = O.full_apply(grid, w.eta, cd, ue) - rhs
        res.append(np.linalg.norm(r) / np.linalg.norm(rhs))
    assert res[1] < res[0] / 10 and res[2] < res[1] / 10


def test_block_solve_by_schur_and_algorithm3_equals_dense_solve():
    w = W.manufactured(L=2, p=6, kappa=9.0)
    grid, xi, xf, nrm, b, cd, s, t = _case(w, 2, 1, 1)
    lams = O.full_lambdas(grid, w.kappa, b)
    M = O.FullBlockJacobi(grid, w.eta, lams)
    rng = np.random.default_rng(5)
    n = grid.layout.n
    r = rng.standard_normal(grid.nleaves * n) + 1j * rng.standard_normal(grid.nleaves * n)
    z = M(r).reshape(grid.nleaves, n)
    for leaf in range(grid.nleaves):
        At = O.leaf_matrix(grid.p, grid.h, w.eta, np.full(grid.layout.ni, lams[leaf]))
        ref = np.linalg.solve(At, r.reshape(grid.nleaves, n)[leaf])
        assert np.linalg.norm(z[leaf] - ref) < 1e-10 * np.linalg.norm(ref)


def test_preconditioned_gmres_on_the_global_system():
    """Block-Jacobi GMRES reaches the dense global solution, whose incoming data is the
    face-system solution; the preconditioner cuts the iterations."""
    w = W.manufactured(L=2, p=6, kappa=8.0)
    grid, xi, xf, nrm, b, cd, s, t = _case(w, 2, 2, 1)
    rhs = O.full_rhs(grid, s, t)
    mv = lambda v: O.full_apply(grid, w.eta, cd, v)
    M = O.FullBlockJacobi(grid, w.eta, O.full_lambdas(grid, w.kappa, b))
    u_pc, its_pc, _ = O.gmres(mv, rhs, tol=1e-12, restart=50, precond=M)
    u_dense, f_dense = O.full_system_solve(grid, w.eta, cd, s.reshape(grid.nleaves, -1), t.reshape(grid.nleaves, 6, -1))
    assert O.relative_error(u_pc, u_dense.reshape(-1)) < 1e-9
    prob = O.build_problem(grid, w.kappa, w.eta, b)
    f_face = np.linalg.solve(O.dense_face_matrix(grid, prob.R), O.rhs_face(grid, prob.H, s, t))
    assert O.relative_error(O.full_to_face(grid, w.eta, u_pc), f_face) < 1e-9
    _, its_plain, _ = O.gmres(mv, rhs, tol=1e-12, restart=50, maxit=3000)
    assert its_pc < its_plain
