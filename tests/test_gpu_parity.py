"""CUDA path vs the CPU oracle, element by element on the same seeded inputs.

Tolerances (relative l2 unless stated):
* leaf maps R, H (FP64 elimination on both sides, different pivot/rounding
  order): 1e-11;
* hps_apply / hps_rhs in FP64: 1e-11 (dominated by the R difference above);
  the apply alone on the oracle's own maps (hps_import_map): 1e-13;
  complex FP32 apply: 2e-6 (FP32 storage of R, ~6e-8 per entry, summed over
  6 q^2 terms with FP32 accumulation);
* hps_precond: FP64 1e-9 (the cluster inverse amplifies the map difference by
  cond(I + D)); FP32 2e-5;
* solves: FP64 form 1e-10, mixed form 1e-6 (the stated targets).
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import OracleCase, gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


def _ragged_workload():
    # 3 x 2 x 2 leaves: an odd axis (clusters of width 1 and 2), p = 7 (q = 5,
    # 6 q^2 = 150 columns: ragged tails for the 2-complex-per-lane FP32 loads).
    w = W.manufactured(L=2, p=7, kappa=9.0)
    w.nx, w.ny, w.nz = 3, 2, 2
    return w


@pytest.fixture(scope="module")
def ragged():
    w = _ragged_workload()
    oc = OracleCase(w)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, max_rhs=4)
    yield w, oc, solver, (xi, xf, b, s, t)
    solver.close()


def test_nodes_match_oracle(ragged):
    w, oc, solver, (xi, xf, b, s, t) = ragged
    assert np.max(np.abs(xi - oc.xi)) < 1e-15
    assert np.max(np.abs(xf - oc.xf)) < 1e-15


def test_leaf_maps_match_oracle(ragged):
    w, oc, solver, _ = ragged
    for leaf in range(oc.grid.nleaves):
        R = solver.export("R", leaf).reshape(oc.grid.nb, oc.grid.nb)
        H = solver.export("H", leaf).reshape(oc.grid.nb, -1)
        assert rel(R, oc.prob.R[leaf]) < 1e-11, leaf
        assert rel(H, oc.prob.H[leaf]) < 1e-11, leaf


def test_homogenized_lambda_matches_oracle(ragged):
    w, oc, solver, _ = ragged
    for leaf in range(oc.grid.nleaves):
        lam = solver.export("lambda", leaf)[0]
        c = O.cdiag_from_b(w.kappa, oc.b[leaf])
        assert abs(lam - O.homogenized_lambda(c)) <= 1e-12 * abs(lam)


def _rand(n, seed, nrhs=1):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n)))


@pytest.mark.parametrize("nrhs", [1, 3])
def test_apply_matches_oracle(ragged, nrhs):
    w, oc, solver, _ = ragged
    f = _rand(oc.grid.nf, 10 + nrhs, nrhs)
    ref = np.stack([oc.apply(f[r]) for r in range(nrhs)])
    y64 = solver.apply(torch.from_numpy(f.reshape(-1)).cuda()).cpu().numpy().reshape(nrhs, -1)
    assert rel(y64, ref) < 1e-11
    f32 = torch.from_numpy(f.reshape(-1).astype(np.complex64)).cuda()
    y32 = solver.apply(f32).cpu().numpy().reshape(nrhs, -1)
    ref32 = np.stack([oc.apply(f[r].astype(np.complex64).astype(np.complex128)) for r in range(nrhs)])
    assert rel(y32, ref32) < 2e-6


@pytest.mark.parametrize("nrhs", [1, 3])
def test_apply_on_the_oracles_maps_fp64(nrhs):
    """The apply kernel alone: the oracle's own leaf maps are loaded into a handle
    (hps_import_map), so both sides apply the same R and only the summation order
    differs.  Bar 1e-13 (6q^2 = 150 FP64 terms per row, ~1e-16 each)."""
    w = _ragged_workload()
    oc = OracleCase(w, with_precond=False)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, max_rhs=4, cluster=0)
    try:
        for leaf in range(oc.grid.nleaves):
            solver.import_map(leaf, oc.prob.R[leaf])
        for leaf in (0, oc.grid.nleaves - 1):
            back = solver.export("R", leaf).reshape(oc.grid.nb, oc.grid.nb)
            assert np.array_equal(back, oc.prob.R[leaf])
        f = _rand(oc.grid.nf, 30 + nrhs, nrhs)
        ref = np.stack([oc.apply(f[r]) for r in range(nrhs)])
        y64 = solver.apply(torch.from_numpy(f.reshape(-1)).cuda()).cpu().numpy().reshape(nrhs, -1)
        assert rel(y64, ref) < 1e-13
        for r in range(nrhs):
            assert rel(y64[r], ref[r]) < 1e-13, r
    finally:
        solver.close()


@pytest.mark.parametrize("nrhs", [1, 2])
def test_precond_matches_oracle(ragged, nrhs):
    w, oc, solver, _ = ragged
    r = _rand(oc.grid.nf, 20 + nrhs, nrhs)
    ref = np.stack([oc.M(r[i]) for i in range(nrhs)])
    z64 = solver.precond(torch.from_numpy(r.reshape(-1)).cuda()).cpu().numpy().reshape(nrhs, -1)
    assert rel(z64, ref) < 1e-9
    r32 = r.astype(np.complex64)
    ref32 = np.stack([oc.M(r32[i].astype(np.complex128)) for i in range(nrhs)])
    z32 = solver.precond(torch.from_numpy(r32.reshape(-1)).cuda()).cpu().numpy().reshape(nrhs, -1)
    assert rel(z32, ref32) < 2e-5


def test_precond_fp16_blocks_close_to_oracle(ragged):
    """FP16 copies of the cluster blocks (one FP32 scale per row, as used by the mixed
    solve): half precision (2^-11) per entry, amplified by the sum over a row."""
    w, oc, solver, _ = ragged
    r = _rand(oc.grid.nf, 31, 1)[0].astype(np.complex64)
    ref = oc.M(r.astype(np.complex128))
    z = solver.precond(torch.from_numpy(r).cuda(), fp16_blocks=True).cpu().numpy()
    assert rel(z, ref) < 5e-3


def test_mixed_only_handle_builds_fp32_preconditioner(ragged):
    """Without the FP64 form the cluster blocks come from FP32 elimination; they stay
    within FP32 accuracy of the oracle's, and the mixed solve still meets its bar."""
    w, oc, _, (xi, xf, b, s, t) = ragged
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",))
    try:
        r = _rand(oc.grid.nf, 41, 1)[0].astype(np.complex64)
        z = solver.precond(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel(z, oc.M(r.astype(np.complex128))) < 1e-4
        f, info = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), t=torch.from_numpy(t.reshape(-1)).cuda(),
                               tol=1e-8, form="mixed")
        assert info["converged"] and rel(f.cpu().numpy(), oc.solve()) < 1e-6
    finally:
        solver.close()


def test_lean_mode_solve(ragged):
    """Lean mode keeps the maps in FP32 plus their FP16 rounding remainders (row-scaled), which
    reproduce the FP64 maps to ~3e-11; the restart residual, the right-hand side and
    complex-double applies use them with double-float accumulation.  So lean solves reach the
    FP64 form's accuracy: a tolerance of 1e-10 gives the oracle's solution to 1e-8 (the map
    remainder times the conditioning), a tolerance of 1e-8 the mixed form's bar of 1e-6."""
    w, oc, _, (xi, xf, b, s, t) = ragged
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), lean=True,
                        max_rhs=3)
    try:
        sd, td = torch.from_numpy(s.reshape(-1)).cuda(), torch.from_numpy(t.reshape(-1)).cuda()
        for tol, bar in ((1e-8, 1e-6), (1e-10, 1e-8)):
            f, info = solver.solve(s=sd, t=td, tol=tol, form="mixed")
            assert info["converged"], info
            assert rel(f.cpu().numpy(), oc.solve()) < bar, tol
        # the FP32 maps as stored
        R = solver.export("R", 3).reshape(oc.grid.nb, oc.grid.nb)
        assert 1e-9 < rel(R, oc.prob.R[3]) < 1e-6
        # complex-double apply and right-hand side through the compensated maps
        f3 = _rand(oc.grid.nf, 51, 3)
        y = solver.apply(torch.from_numpy(f3.reshape(-1)).cuda()).cpu().numpy().reshape(3, -1)
        for k in range(3):
            assert rel(y[k], oc.apply(f3[k])) < 1e-9, k
        assert rel(solver.rhs(sd, td).cpu().numpy(), oc.rhs()) < 1e-9
        assert rel(solver.rhs(None, td).cpu().numpy(), O.rhs_face(oc.grid, oc.prob.H, None, oc.t[0])) < 1e-12
    finally:
        solver.close()


@pytest.mark.parametrize("p", [7, 10, 12])
def test_compensated_maps_match_the_fp64_maps(p):
    """The compensated FP32 maps (FP32 rounding + FP16 remainder per row) against the FP64 maps
    of a handle built from the same medium: right-hand sides with 1 and 3 sources and
    complex-double applies with 1, 2 and 5 right-hand sides, at 1e-9.  p = 7, 10, 12 make the
    body-load map H narrower than, wider than and much wider than the ItI map (n1^3 vs 6q^2)."""
    w = W.manufactured(L=1, p=p, kappa=9.0)
    w.nx, w.ny, w.nz = 2, 2, 1
    xi, xf, b, s, t = gpu_inputs(w, hps)
    full = hps.Solver(2, 2, 1, p, kappa=9.0, eta=w.eta, b=b, cluster=0, max_rhs=5)
    lean = hps.Solver(2, 2, 1, p, kappa=9.0, eta=w.eta, b=b, forms=("mixed",), lean=True, cluster=0, max_rhs=5)
    try:
        rng = np.random.default_rng(p)
        for nrhs in (1, 3):
            sv = torch.from_numpy(rng.standard_normal(nrhs * full.nl * full.ni) + 0.5j).cuda()
            tv = torch.from_numpy(rng.standard_normal(nrhs * full.nf) + 1j).cuda()
            assert rel(lean.rhs(sv, tv, nrhs=nrhs).cpu().numpy(), full.rhs(sv, tv, nrhs=nrhs).cpu().numpy()) < 1e-9
        for nrhs in (1, 2, 5):
            f = torch.from_numpy(_rand(full.nf, 60 + nrhs, nrhs).reshape(-1)).cuda()
            assert rel(lean.apply(f).cpu().numpy(), full.apply(f).cpu().numpy()) < 1e-9, nrhs
    finally:
        full.close()
        lean.close()


def test_rhs_matches_oracle(ragged):
    w, oc, solver, (xi, xf, b, s, t) = ragged
    bg = solver.rhs(torch.from_numpy(s.reshape(-1)).cuda(), torch.from_numpy(t.reshape(-1)).cuda())
    assert rel(bg.cpu().numpy(), oc.rhs()) < 1e-11


@pytest.mark.parametrize("form,tol,bar", [("fp64", 1e-12, 1e-10), ("mixed", 1e-8, 1e-6), ("mixed", 1e-12, 1e-10)])
def test_solve_matches_oracle(ragged, form, tol, bar):
    """The mixed form restarts from the FP64 true residual, so at a tight tolerance it
    reaches the FP64 bar as well."""
    w, oc, solver, (xi, xf, b, s, t) = ragged
    f_ref = oc.solve()
    f, info = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), t=torch.from_numpy(t.reshape(-1)).cuda(),
                           tol=tol, form=form)
    assert info["converged"], info
    assert rel(f.cpu().numpy(), f_ref) < bar, info


def test_recover_interior_matches_oracle(ragged):
    """u = A^{-1}[s; P^{-1} f] per leaf from the GPU face solution, against the oracle's
    recovery from its own solution and against the manufactured u."""
    w, oc, solver, (xi, xf, b, s, t) = ragged
    sd = torch.from_numpy(s.reshape(-1)).cuda()
    f, info = solver.solve(s=sd, t=torch.from_numpy(t.reshape(-1)).cuda(), tol=1e-12, form="fp64")
    u, uf = solver.recover(f, s=sd, faces=True)
    u = u.cpu().numpy().reshape(oc.grid.nleaves, -1)
    uf = uf.cpu().numpy().reshape(oc.grid.nleaves, -1)
    ref, ref_f = O.recover_interior(oc.grid, w.kappa, w.eta, oc.b, oc.s[0], oc.solve(), with_faces=True)
    assert rel(u, ref) < 1e-10
    assert rel(uf, ref_f) < 1e-10
    assert rel(u, w.meta["u"](oc.xi)) < 1e-2
    _, _, xc = hps.nodes(w.nx, w.ny, w.nz, w.p, cheb_faces=True)
    assert np.abs(xc - O.cheb_face_nodes(oc.grid)).max() < 1e-15
    # face nodes sit where the p = 7 interpolant is least accurate: a looser sanity bar
    assert rel(uf, w.meta["u"](xc).reshape(oc.grid.nleaves, -1)) < 3e-2


def test_solve_host_buffers_match_device_buffers(ragged):
    w, oc, solver, (xi, xf, b, s, t) = ragged
    f_dev, _ = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), t=torch.from_numpy(t.reshape(-1)).cuda(),
                            tol=1e-12, form="fp64")
    out = np.zeros(oc.grid.nf, dtype=np.complex128)
    solver.solve(s=s.reshape(-1), t=t.reshape(-1), tol=1e-12, form="fp64", out=out)
    assert np.array_equal(out, f_dev.cpu().numpy())


def test_solve_several_rhs(ragged):
    w, oc, solver, (xi, xf, b, s, t) = ragged
    # three right-hand sides: the manufactured one, twice its body load, and boundary data only
    S = np.stack([s[0], 2.0 * s[0], np.zeros_like(s[0])])
    T = np.stack([t[0], np.zeros_like(t[0]), t[0]])
    f, info = solver.solve(s=torch.from_numpy(S.reshape(-1)).cuda(), t=torch.from_numpy(T.reshape(-1)).cuda(),
                           tol=1e-12, form="fp64", nrhs=3)
    assert info["converged"]
    f = f.cpu().numpy().reshape(3, -1)
    M = O.dense_face_matrix(oc.grid, oc.prob.R)
    for r in range(3):
        ref = np.linalg.solve(M, O.rhs_face(oc.grid, oc.prob.H, S[r], T[r]))
        assert rel(f[r], ref) < 1e-10, r


def test_zero_rhs_gives_zero():
    solver = hps.Solver(2, 2, 2, 6, kappa=5.0)
    f, info = solver.solve(tol=1e-10, form="fp64")
    assert info["converged"] and info["iterations"] == 0
    assert not torch.any(f != 0)
    solver.close()


def test_single_leaf_solution_is_boundary_data():
    w = W.plane_wave(L=1, p=6, kappa=5.0)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(1, 1, 1, 6, kappa=w.kappa, eta=w.eta, b=b)
    f, info = solver.solve(t=torch.from_numpy(t.reshape(-1)).cuda(), tol=1e-12, form="fp64")
    assert rel(f.cpu().numpy(), t.reshape(-1)) < 1e-14
    solver.close()


@pytest.fixture(scope="module")
def plane_wave_4cubed():
    w = W.plane_wave_4cubed()
    oc = OracleCase(w, with_precond=False)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b)
    yield w, oc, solver, t
    solver.close()


@pytest.mark.parametrize("form,bar", [("fp64", 1e-10), ("mixed", 1e-6)])
@pytest.mark.parametrize("precond", [True, False])
def test_plane_wave_4cubed_solve(plane_wave_4cubed, form, bar, precond):
    """4^3 leaves, p = 8, kappa = eta = 10, plane wave, GMRES(50) with 2x2x2 clusters."""
    w, oc, solver, t = plane_wave_4cubed
    f_ref = oc.solve()
    f, info = solver.solve(t=torch.from_numpy(t.reshape(-1)).cuda(), tol=w.tol if form == "fp64" else 1e-8,
                           form=form, precond=precond)
    assert info["converged"], info
    f = f.cpu().numpy()
    assert rel(f, f_ref) < bar, info
    # and both are close to the exact impedance data of the plane wave
    exact = w.exact_f[0](oc.xf, oc.nrm).reshape(-1)
    assert rel(f, exact) < 1e-3


@pytest.fixture(scope="module")
def bump_4cubed():
    w = W.scaled(W.bump_16cubed(), 4)
    oc = OracleCase(w, with_precond=False)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=b)
    yield w, oc, solver, s
    solver.close()


@pytest.mark.parametrize("form,tol,bar", [("fp64", 1e-11, 1e-10), ("mixed", 1e-7, 1e-6), ("mixed", 1e-11, 1e-10)])
def test_bump_scaled_solve(bump_4cubed, form, tol, bar):
    """The variable-coefficient workload (p = 10, kappa = 40, Gaussian bump and source) on 4^3 leaves."""
    w, oc, solver, s = bump_4cubed
    f_ref = oc.solve()
    f, info = solver.solve(s=torch.from_numpy(s.reshape(-1)).cuda(), tol=tol, form=form)
    assert info["converged"], info
    assert rel(f.cpu().numpy(), f_ref) < bar, info
