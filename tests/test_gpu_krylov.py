"""The GMRES driver on the GPU: the restart cycle replayed from a CUDA graph against the same
cycle launched step by step, the conditional second Gram-Schmidt pass against CGS2 at every step,
and resuming from a stored iterate (initial guess).

* Graph vs step-by-step: the same kernels on the same data in the same order; the graph only
  lets the steps after convergence return at once instead of stopping on the host.  Results
  must agree bit for bit, iteration counts exactly.
* One Gram-Schmidt pass plus a second where the first cancelled most of the vector
  (Rutishauser's test, ||w'|| < ||w||/10) vs two passes at every step: both keep the basis
  orthogonal to ~10 eps, so both reach the oracle's solution within the solve tolerance's bar,
  with iteration counts within a few of each other.
* Resume: a solve started from its own converged answer does no iteration; one stopped early
  (maxit) and resumed reaches the same solution as an uninterrupted solve.
"""

import numpy as np
import pytest

import workloads as W
from gpu_cases import OracleCase, gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


@pytest.fixture(scope="module")
def case():
    # 4^3 leaves, p = 8, bump medium and Gaussian source (the benchmark recipe on a small grid)
    w = W.scaled(W.bump_16cubed(), 4)
    w.p = 8
    oc = OracleCase(w, with_precond=False)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(4, 4, 4, 8, kappa=w.kappa, eta=w.eta, b=b, lambda_bin=0.01)
    yield w, oc, solver, torch.from_numpy(s.reshape(-1)).cuda()
    solver.close()


@pytest.mark.parametrize("form,tol,precond", [("mixed", 1e-8, True), ("fp64", 1e-10, True), ("mixed", 1e-8, False)])
def test_graph_replay_equals_step_by_step(case, form, tol, precond):
    w, oc, solver, s = case
    f_g, i_g = solver.solve(s=s, tol=tol, form=form, precond=precond)
    f_g2, i_g2 = solver.solve(s=s, tol=tol, form=form, precond=precond)  # replay of the cached graph
    f_s, i_s = solver.solve(s=s, tol=tol, form=form, precond=precond, graph=False)
    assert i_g["converged"] and i_s["converged"]
    assert i_g["iterations"] == i_s["iterations"] == i_g2["iterations"]
    assert i_g["reorth_steps"] == i_s["reorth_steps"]
    assert torch.equal(f_g, f_s) and torch.equal(f_g, f_g2)
    assert rel(f_g.cpu().numpy(), oc.solve()) < (1e-10 if form == "fp64" else 1e-6)


@pytest.mark.parametrize("form", ["mixed", "fp64"])
def test_conditional_second_pass_matches_cgs2(case, form):
    w, oc, solver, s = case
    tol = 1e-10 if form == "fp64" else 1e-8
    f1, i1 = solver.solve(s=s, tol=tol, form=form)
    f2, i2 = solver.solve(s=s, tol=tol, form=form, cgs2=True)
    assert i1["converged"] and i2["converged"]
    assert abs(i1["iterations"] - i2["iterations"]) <= 2, (i1, i2)
    assert i1["reorth_steps"] < i1["iterations"]  # the second pass is not taken at every step
    ref = oc.solve()
    bar = 1e-10 if form == "fp64" else 1e-6
    assert rel(f1.cpu().numpy(), ref) < bar and rel(f2.cpu().numpy(), ref) < bar


def test_resume_from_a_stored_iterate(case):
    w, oc, solver, s = case
    f, info = solver.solve(s=s, tol=1e-8, form="mixed")
    # from the converged answer: nothing to do, the answer comes back unchanged
    f_again, info2 = solver.solve(s=s, tol=1e-8, form="mixed", x0=f.clone())
    assert info2["converged"] and info2["iterations"] == 0 and info2["cycles"] == 0
    assert torch.equal(f_again, f)
    # stopped after 12 iterations (maxit), then resumed to the tolerance
    xi, xf = hps.nodes(4, 4, 4, 8)
    short = hps.Solver(4, 4, 4, 8, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi).reshape(-1), lambda_bin=0.01,
                       maxit=12, restart=10)
    try:
        f_part, ip = short.solve(s=s, tol=1e-8, form="mixed")
        assert not ip["converged"] and ip["iterations"] == 12 and ip["status"] == hps._native.HPS_ENOCONV
    finally:
        short.close()
    f_res, ir = solver.solve(s=s, tol=1e-8, form="mixed", x0=f_part)
    assert ir["converged"]
    assert rel(f_res.cpu().numpy(), oc.solve()) < 1e-6
    assert rel(f_res.cpu().numpy(), f.cpu().numpy()) < 1e-6


def test_profile_counts_under_graph_replay(case):
    """Per-phase intervals recorded inside the captured cycle are read after every replay and
    counted only for the steps that ran."""
    w, oc, solver, s = case
    solver.profile(enable=True, reset=True)
    f, info = solver.solve(s=s, tol=1e-8, form="mixed")
    p = solver.profile(enable=False, reset=True)
    assert p["count"]["apply"] == info["iterations"]
    assert p["count"]["arnoldi"] == info["iterations"]
    assert p["count"]["residual"] == info["cycles"]
    assert p["ms"]["apply"] > 0 and p["launches"] > 10 * info["iterations"]


def test_non_finite_residual_is_an_error(case):
    """A NaN in the data makes every residual norm NaN, which compares false against any
    tolerance: the solve must end with HPS_EBREAKDOWN, not report convergence."""
    w, oc, solver, s = case
    bad = s.clone()
    bad[7] = complex(float("nan"), 0.0)
    for form in ("mixed", "fp64"):
        with pytest.raises(hps.HPSError) as ei:
            solver.solve(s=bad, tol=1e-8, form=form)
        assert ei.value.code == -5 and "non-finite" in str(ei.value), ei.value
    # the handle still solves
    f, info = solver.solve(s=s, tol=1e-8, form="mixed")
    assert info["converged"] and rel(f.cpu().numpy(), oc.solve()) < 1e-6
