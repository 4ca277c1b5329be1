"""The preconditioner with many right-hand sides (Sec. 4, the block-Jacobi solves of Algorithm 4
in face form): stage B applies each leaf's block to 8 right-hand sides per pass, and stage K runs
every cluster block on the tensor cores in one launch, as the GEMM of K_c against the columns
(member cluster, right-hand side) -- 64 of them per tile.

Bars: stage K takes one TF32 product (both operands rounded to 10 mantissa bits, ~2^-11
relative each; tests/test_tf32_bounds.py) with the truncating FP32 accumulation of the tensor
cores (~1e-5), i.e. ~3e-4 relative on z; compared at 2e-3 with the oracle's preconditioner and
with the single-RHS call (FP32 blocks on the SIMT path).  The stage-B batching changes no
arithmetic: its right-hand sides agree with single-RHS calls to FP32 rounding.  Solves reach the
oracle's solution at the mixed form's bar (1e-6), the preconditioner changing only the
iteration count."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import OracleCase, gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


@pytest.fixture(scope="module")
def case():
    # 4^3 leaves (8 clusters of 2x2x2), p = 8 (q = 6, 864 internal values per cluster)
    w = W.scaled(W.bump_16cubed(), 4)
    w.p = 8
    oc = OracleCase(w)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(4, 4, 4, 8, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), max_rhs=64)
    yield w, oc, solver, (b, s)
    solver.close()


def test_batched_precond_matches_oracle_and_single_rhs(case):
    w, oc, solver, _ = case
    rng = np.random.default_rng(41)
    nrhs = 64
    r = (rng.standard_normal((nrhs, oc.grid.nf)) + 1j * rng.standard_normal((nrhs, oc.grid.nf))).astype(np.complex64)
    rd = torch.from_numpy(r.reshape(-1)).cuda()
    z = solver.precond(rd).cpu().numpy().reshape(nrhs, -1)
    single = np.stack([solver.precond(rd[k * oc.grid.nf:(k + 1) * oc.grid.nf].clone()).cpu().numpy()
                       for k in range(nrhs)])
    d = rel(z, single)
    assert 1e-6 < d < 2e-3  # a different (tensor-core) path, within its error model
    for k in (0, 31, 63):
        ref = oc.M(r[k].astype(np.complex128))
        assert rel(z[k], ref) < 2e-3, k
        assert rel(single[k], ref) < 2e-5, k
    # external faces are copied (z_ext = r_ext) by stage B for every right-hand side
    grid = oc.grid
    q2 = grid.q * grid.q
    for leaf in range(grid.nleaves):
        for face in range(6):
            if grid.neighbor(leaf, face) < 0:
                sl = slice(leaf * grid.nb + face * q2, leaf * grid.nb + (face + 1) * q2)
                assert np.array_equal(z[:, sl], r[:, sl])


def test_fp16_tensor_core_stage_k(case):
    """The preconditioner with FP16 blocks (the mixed solve's) runs stage K for every cluster on
    the tensor cores with FP16 operands: K_c's FP16 copy against t scaled per cluster by its
    largest component (stage B records it) and split into two FP16 terms.  K_c carries 2^-11
    relative rounding, the FP16 blocks' own precision: against the oracle's preconditioner at
    5e-3.  With 64
    right-hand sides the same products are tiled by (member, right-hand side) instead of by
    members: each right-hand side equals its single-RHS result to 1e-6."""
    w, oc, solver, _ = case
    rng = np.random.default_rng(43)
    n = oc.grid.nf
    r = (rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))).astype(np.complex64)
    rd = torch.from_numpy(r.reshape(-1)).cuda()
    z64 = solver.precond(rd, fp16_blocks=True).cpu().numpy().reshape(64, -1)
    for k in (0, 9, 63):
        zk = solver.precond(rd[k * n:(k + 1) * n].clone(), fp16_blocks=True).cpu().numpy()
        assert rel(zk, oc.M(r[k].astype(np.complex128))) < 5e-3, k
        assert rel(z64[k], zk) < 1e-6, k
    # linear in r to FP32 level: GMRES applies the preconditioner to V y in its update and
    # assumes M^{-1}(V y) = sum_j y_j M^{-1} v_j.  t enters the FP16 products as two FP16 terms
    # (~2^-22); one FP16 rounding of t (2^-11, input-dependent) gave ~2e-4 here
    zx = solver.precond(rd[n:2 * n].clone(), fp16_blocks=True).cpu().numpy()
    zy = solver.precond(rd[2 * n:3 * n].clone(), fp16_blocks=True).cpu().numpy()
    zxy = solver.precond((rd[n:2 * n] + 0.5 * rd[2 * n:3 * n]).contiguous(), fp16_blocks=True).cpu().numpy()
    assert rel(zxy, zx + 0.5 * zy) < 3e-5
    # a right-hand side that vanishes on some clusters: their z_int is exactly 0
    r0 = np.zeros(n, dtype=np.complex64)
    r0[: oc.grid.nb] = r[0, : oc.grid.nb]
    z0 = solver.precond(torch.from_numpy(r0).cuda(), fp16_blocks=True).cpu().numpy()
    assert np.all(np.isfinite(z0))
    assert rel(z0, oc.M(r0.astype(np.complex128))) < 5e-3
    # ... or holds only subnormal floats there (a source far away): the per-cluster scale of t
    # must not overflow; those clusters count as 0, a change far below the bar
    rs = np.full(n, 3e-40 + 2e-40j, dtype=np.complex64)
    rs[: oc.grid.nb] = r[0, : oc.grid.nb]
    zs = solver.precond(torch.from_numpy(rs).cuda(), fp16_blocks=True).cpu().numpy()
    assert np.all(np.isfinite(zs))
    assert rel(zs, oc.M(rs.astype(np.complex128))) < 5e-3
    zs64 = solver.precond(torch.from_numpy(np.tile(rs, 64)).cuda(), fp16_blocks=True).cpu().numpy()
    assert np.all(np.isfinite(zs64)) and rel(zs64.reshape(64, -1)[17], zs) < 1e-6


def test_batched_stage_b_equals_single_rhs_stage_b(case):
    """3 right-hand sides: stage B in one pass of NR = 4, stage K per right-hand side on the
    single-RHS path -- the same arithmetic as three single-RHS calls, rhs by rhs."""
    w, oc, solver, _ = case
    rng = np.random.default_rng(42)
    n = oc.grid.nf
    r = (rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))).astype(np.complex64)
    rd = torch.from_numpy(r.reshape(-1)).cuda()
    z = solver.precond(rd).cpu().numpy().reshape(3, -1)
    for k in range(3):
        zk = solver.precond(rd[k * n:(k + 1) * n].clone()).cpu().numpy()
        assert rel(z[k], zk) < 1e-6, k


def test_preconditioned_64_rhs_solve_matches_oracle(case):
    """64 right-hand sides through the preconditioned mixed solve: tensor-core apply (three TF32
    products), batched stage B, tensor-core stage K over member x RHS columns, captured cycle."""
    w, oc, solver, (b, s) = case
    S = np.stack([s[0] * (1.0 + 0.05 * k) * np.exp(0.1j * k) for k in range(64)])
    f, info = solver.solve(s=torch.from_numpy(S.reshape(-1)).cuda(), tol=1e-9, form="mixed", nrhs=64)
    assert info["converged"], info
    f = f.cpu().numpy().reshape(64, -1)
    M = O.dense_face_matrix(oc.grid, oc.prob.R)
    for k in (0, 40, 63):
        ref = np.linalg.solve(M, O.rhs_face(oc.grid, oc.prob.H, S[k], None))
        assert rel(f[k], ref) < 1e-6, k
    # the same right-hand sides without the preconditioner: the same solution (the preconditioner
    # changes the iteration count only; on this small grid it barely changes it)
    f2, info2 = solver.solve(s=torch.from_numpy(S.reshape(-1)).cuda(), tol=1e-9, form="mixed", nrhs=64,
                             precond=False)
    assert info2["converged"], info2
    assert rel(f, f2.cpu().numpy().reshape(64, -1)) < 1e-6
