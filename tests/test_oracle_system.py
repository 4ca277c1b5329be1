"""Pins of the oracle's face system, GMRES and preconditioner against exact
algebra, the paper's global system and closed-form solutions (no GPU)."""

import numpy as np
import pytest

import oracle as O
import workloads as W


def _setup(w, homogenized=False):
    grid = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi = O.interior_nodes(grid)
    xf = O.face_nodes(grid)
    nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
    b = w.sample_b(xi)
    prob = O.build_problem(grid, w.kappa, w.eta, b, homogenized=homogenized)
    s = w.sample_s(xi)
    t = w.sample_t(xf, nrm)
    rhs = O.rhs_face(grid, prob.H, None if s is None else s[0], None if t is None else t[0])
    return grid, prob, rhs, (xi, xf, nrm, b, s, t)


def test_swap_is_an_involution_on_interior_faces():
    grid = O.Grid(3, 2, 2, 5)
    rng = np.random.default_rng(0)
    g = rng.standard_normal(grid.nf) + 1j * rng.standard_normal(grid.nf)
    y = O.swap(grid, O.swap(grid, g)).reshape(grid.nleaves, 6, -1)
    g = g.reshape(grid.nleaves, 6, -1)
    for leaf in range(grid.nleaves):
        for face in range(6):
            if grid.neighbor(leaf, face) >= 0:
                assert np.array_equal(y[leaf, face], g[leaf, face])
            else:
                assert not np.any(y[leaf, face])


def test_single_leaf_face_system_is_identity():
    """One leaf with impedance data on all faces: Pi = 0 so f = t."""
    w = W.plane_wave(L=1, p=6, kappa=5.0)
    grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
    M = O.dense_face_matrix(grid, prob.R)
    assert np.array_equal(M, np.eye(grid.nf))
    f, its, _ = O.gmres(lambda v: O.apply_face(grid, prob.R, v), rhs)
    assert np.allclose(f, t[0].reshape(-1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("p,bound", [(6, 5e-2), (8, 3e-3), (10, 1e-4), (12, 2e-6)])
def test_plane_wave_solution_converges(p, bound):
    w = W.plane_wave(L=2, p=p, kappa=10.0, seed=1)
    grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
    f = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
    err = O.relative_error(f, w.exact_f[0](xf, nrm))
    assert err < bound


def test_manufactured_solution_converges():
    errs = []
    for p in (6, 8, 10, 12):
        w = W.manufactured(L=2, p=p, kappa=8.0)
        grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
        f = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
        errs.append(O.relative_error(f, w.exact_f[0](xf, nrm)))
    assert errs[-1] < 1e-6
    for a, b_ in zip(errs, errs[1:]):
        assert b_ < a / 10


def test_bumps_solution_converges_spectrally():
    """The bumps test solution of Sec. 6.3 (not separable) with the bump medium: the face
    solution converges spectrally in p to its exact impedance data."""
    errs = []
    for p in (6, 8, 10):
        w = W.manufactured_bumps(L=2, p=p, kappa=6.0)
        grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
        f = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
        errs.append(O.relative_error(f, w.exact_f[0](xf, nrm)))
    assert errs[-1] < 1e-5
    for a, b_ in zip(errs, errs[1:]):
        assert b_ < a / 10


def test_recovered_interior_solution_converges():
    """u = A^{-1}[s; P^{-1} f] from the face solution reproduces the manufactured u at
    the interior nodes, spectrally in p."""
    errs = []
    for p in (6, 8, 10):
        w = W.manufactured(L=2, p=p, kappa=8.0)
        grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
        f = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
        u = O.recover_interior(grid, w.kappa, w.eta, b, s[0], f)
        errs.append(O.relative_error(u, w.meta["u"](xi)))
    assert errs[-1] < 1e-4
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10


def test_recovered_face_values_match_the_solution_at_chebyshev_face_nodes():
    """The face part of u = A^{-1}[s; P^{-1} f] is u at the Chebyshev face nodes (the rest
    of the paper's unknowns): spectral convergence to the manufactured u there, and
    leaves sharing a face agree on it."""
    errs = []
    for p in (6, 8, 10):
        w = W.manufactured(L=2, p=p, kappa=8.0)
        grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
        f = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
        u, ub = O.recover_interior(grid, w.kappa, w.eta, b, s[0], f, with_faces=True)
        xc = O.cheb_face_nodes(grid)
        errs.append(O.relative_error(ub, w.meta["u"](xc)))
        ub = ub.reshape(grid.nleaves, 6, -1)
        for leaf in range(grid.nleaves):
            for face in range(6):
                nbr = grid.neighbor(leaf, face)
                if nbr >= 0:
                    assert np.allclose(xc[leaf, face], xc[nbr, face ^ 1], atol=1e-15)
                    assert O.relative_error(ub[leaf, face], ub[nbr, face ^ 1]) < 10 * errs[-1]
    assert errs[-1] < 1e-4
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10


def test_dense_solve_matches_gmres_and_preconditioned_gmres():
    w = W.manufactured(L=2, p=6, kappa=12.0)
    w.ny = 2
    grid, prob, rhs, _ = _setup(w)
    f_dense = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
    mv = lambda v: O.apply_face(grid, prob.R, v)
    f_plain, its_plain, _ = O.gmres(mv, rhs, tol=1e-13, restart=30)
    hom = O.build_problem(grid, w.kappa, w.eta, _setup(w)[3][3], homogenized=True)
    M = O.Preconditioner(grid, hom.R)
    f_pc, its_pc, _ = O.gmres(mv, rhs, tol=1e-13, restart=30, precond=M)
    assert O.relative_error(f_plain, f_dense) < 1e-12
    assert O.relative_error(f_pc, f_dense) < 1e-12
    # one 2x2x2 cluster with homogenized maps: far fewer iterations
    assert its_pc < its_plain


def test_exact_single_cluster_preconditioner_solves_in_one_step():
    w = W.manufactured(L=2, p=6, kappa=9.0)
    grid, prob, rhs, _ = _setup(w)
    M = O.Preconditioner(grid, prob.R, size=2)  # exact maps, one cluster = the grid
    mv = lambda v: O.apply_face(grid, prob.R, v)
    f, its, hist = O.gmres(mv, rhs, tol=1e-12, restart=10, precond=M)
    assert its == 1
    assert hist[-1] < 1e-12


def test_preconditioner_clusters_odd_grid():
    grid = O.Grid(3, 2, 1, 5)
    blocks = O.clusters(grid)
    assert sorted(sum(blocks, [])) == list(range(grid.nleaves))
    assert [len(b) for b in blocks] == [4, 2]


@pytest.mark.parametrize("shape", [(2, 1, 1), (1, 2, 2)])
def test_face_system_equals_paper_global_system(shape):
    """The face system is the exact reduction of the global system of Sec. 3.1."""
    w = W.manufactured(L=1, p=6, kappa=7.0)
    w.nx, w.ny, w.nz = shape
    grid, prob, rhs, (xi, xf, nrm, b, s, t) = _setup(w)
    f_face = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
    cdiag = O.cdiag_from_b(w.kappa, b)
    u, f_full = O.full_system_solve(grid, w.eta, cdiag, s[0], t[0])
    assert O.relative_error(f_face, f_full) < 1e-10


def test_global_system_rows_follow_eq_2x2():
    """Two leaves: the coupling block of alpha's face 2 is G^beta on beta's face 1."""
    grid = O.Grid(2, 1, 1, 5)
    cd = np.full((2, grid.layout.ni), 4.0 + 0j)
    A = O.full_system_matrix(grid, 2.0, cd)
    n, ni, q2 = grid.layout.n, grid.layout.ni, grid.q ** 2
    G = O.leaf_outgoing_op(5, grid.h, 2.0)
    F = O.leaf_incoming_op(5, grid.h, 2.0)
    rows_a2 = slice(ni + 1 * q2, ni + 2 * q2)  # alpha = leaf 0, face +x
    assert np.array_equal(A[rows_a2, n:], G[0:q2, :])  # beta's -x face
    assert np.array_equal(A[rows_a2, :n], F[q2:2 * q2, :])
    rows_b1 = slice(n + ni, n + ni + q2)  # beta = leaf 1, face -x
    assert np.array_equal(A[rows_b1, :n], G[q2:2 * q2, :])
