"""Pins of the binned homogenized constants (reuse of one local solver for
leaves with nearly the same medium, Sec. 4.1 remark) in the oracle (no GPU)."""

import numpy as np

import oracle as O
import workloads as W


def _lams(grid, w, b):
    return np.array([O.homogenized_lambda(O.cdiag_from_b(w.kappa, b[i])) for i in range(grid.nleaves)])


def test_zero_bin_keeps_every_lambda():
    w = W.manufactured(L=2, p=6, kappa=9.0)
    grid = O.Grid(2, 1, 2, w.p)
    b = w.sample_b(O.interior_nodes(grid))
    plain = O.build_problem(grid, w.kappa, w.eta, b, homogenized=True)
    binned = O.build_problem(grid, w.kappa, w.eta, b, homogenized=True, lambda_bin=0.0)
    assert np.array_equal(plain.lam, _lams(grid, w, b))
    for leaf in range(grid.nleaves):
        assert np.array_equal(plain.R[leaf], binned.R[leaf])


def test_bins_are_a_lattice_within_half_a_width():
    rng = np.random.default_rng(11)
    lams = rng.uniform(-2000, 3000, 200) + 1j * rng.uniform(0, 80, 200)
    for delta in (1e-4, 1e-3, 3e-2, 0.25):
        w = delta * np.abs(lams).max()
        q = O.binned_lambdas(lams, delta)
        for part_q, part in ((q.real, lams.real), (q.imag, lams.imag)):
            k = part_q / w
            assert np.allclose(k, np.round(k), rtol=0, atol=1e-9)
            assert np.all(np.abs(part_q - part) <= 0.5 * w * (1 + 1e-12))
        # binning never creates distinct values
        assert len(set(q.tolist())) <= len(set(lams.tolist()))


def test_a_bin_wider_than_every_lambda_gives_the_laplace_maps():
    """delta >> 1 rounds every lambda to 0: R~ is then the exact map of -Delta u = 0."""
    w = W.manufactured(L=2, p=6, kappa=9.0)
    grid = O.Grid(2, 2, 1, w.p)
    b = w.sample_b(O.interior_nodes(grid))
    hom = O.build_problem(grid, w.kappa, w.eta, b, homogenized=True, lambda_bin=10.0)
    laplace = O.build_problem(grid, 0.0, w.eta, np.zeros_like(b))
    assert not np.any(hom.lam)
    for leaf in range(grid.nleaves):
        assert np.allclose(hom.R[leaf], laplace.R[leaf], rtol=0, atol=1e-13)


def test_binning_merges_leaves_and_equal_bins_share_maps():
    w = W.scaled(W.bump_16cubed(p=6, kappa=10.0), 4)
    grid = O.Grid(4, 4, 4, w.p)
    b = w.sample_b(O.interior_nodes(grid))
    lams = _lams(grid, w, b)
    counts = [len(set(O.binned_lambdas(lams, d).tolist())) for d in (0.0, 1e-3, 1e-2, 1e-1)]
    assert counts[0] == len(set(lams.tolist()))
    assert counts == sorted(counts, reverse=True) and counts[-1] < counts[0]
    hom = O.build_problem(grid, w.kappa, w.eta, b, homogenized=True, lambda_bin=1e-1)
    first = {}
    for leaf in range(grid.nleaves):
        key = complex(hom.lam[leaf])
        if key in first:
            assert np.array_equal(hom.R[leaf], hom.R[first[key]])
        else:
            first[key] = leaf


def test_binned_preconditioner_reaches_the_same_solution():
    """The bins change the preconditioner only: GMRES still converges to the dense solution."""
    w = W.manufactured(L=2, p=6, kappa=12.0)
    grid = O.Grid(4, 2, 2, w.p)
    xi, xf = O.interior_nodes(grid), O.face_nodes(grid)
    nrm = np.broadcast_to(O.face_normals()[None, :, None, :], xf.shape)
    b = w.sample_b(xi)
    prob = O.build_problem(grid, w.kappa, w.eta, b)
    rhs = O.rhs_face(grid, prob.H, w.sample_s(xi)[0], w.sample_t(xf, nrm)[0])
    f_dense = np.linalg.solve(O.dense_face_matrix(grid, prob.R), rhs)
    mv = lambda v: O.apply_face(grid, prob.R, v)
    _, its_plain, _ = O.gmres(mv, rhs, tol=1e-12, restart=40)
    hom = O.build_problem(grid, w.kappa, w.eta, b, homogenized=True, lambda_bin=0.05)
    f_pc, its_pc, _ = O.gmres(mv, rhs, tol=1e-12, restart=40, precond=O.Preconditioner(grid, hom.R))
    assert O.relative_error(f_pc, f_dense) < 1e-10
    assert its_pc < its_plain
