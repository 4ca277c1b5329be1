"""The tensor-core apply (64 right-hand sides per launch, three TF32 products
with FP32 accumulation) against the oracle and against the SIMT apply.

Tolerance: the three-product TF32 split keeps about 22 bits per product
term (the dropped A_lo B_lo term and the rounding of the lo parts are each
~2^-22 relative); over the 2 x 6q^2 = 1200 real terms of a row at p = 12
with FP32 accumulation the measured relative error is ~5e-6 (first GPU run,
truncated hi parts), so the bar is 1e-5 overall and 3e-5 per right-hand side.
The SIMT FP32 apply (~1e-7) is compared at the same bar."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")

import workloads as W  # noqa: E402
from gpu_cases import OracleCase, gpu_inputs, rel  # noqa: E402


def _case(nx, ny, nz, p, kappa):
    w = W.manufactured(L=1, p=p, kappa=kappa)
    w.nx, w.ny, w.nz = nx, ny, nz
    oc = OracleCase(w, with_precond=False)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    tc = hps.Solver(nx, ny, nz, p, kappa=kappa, eta=w.eta, b=b, forms=("mixed",), max_rhs=64, cluster=0)
    simt = hps.Solver(nx, ny, nz, p, kappa=kappa, eta=w.eta, b=b, forms=("mixed",), max_rhs=64, cluster=0,
                      tc_apply=False)
    return w, oc, tc, simt, (s, t)


# p = 12: n_b = 600 -> five 128-row tiles (the last one partial), 38 K blocks;
# p = 7: n_b = 150 -> two tiles, a ragged last K block.
@pytest.mark.parametrize("shape,p", [((2, 2, 1), 12), ((3, 1, 1), 7)])
def test_tc_apply_matches_oracle_and_simt(shape, p):
    w, oc, tc, simt, _ = _case(*shape, p, 9.0)
    try:
        rng = np.random.default_rng(p)
        f = (rng.standard_normal((64, oc.grid.nf)) + 1j * rng.standard_normal((64, oc.grid.nf))).astype(np.complex64)
        fd = torch.from_numpy(f.reshape(-1)).cuda()
        y_tc = tc.apply(fd).cpu().numpy().reshape(64, -1)
        y_simt = simt.apply(fd).cpu().numpy().reshape(64, -1)
        ref = np.stack([oc.apply(f[r].astype(np.complex128)) for r in range(64)])
        assert rel(y_tc, ref) < 1e-5
        assert rel(y_tc, y_simt) < 1e-5
        # every right-hand side, not only the aggregate
        for r in range(64):
            assert rel(y_tc[r], ref[r]) < 3e-5, r
    finally:
        tc.close()
        simt.close()


def test_tc_multi_rhs_solve():
    """64 right-hand sides through the unpreconditioned mixed solve: each basis vector is also kept
    rounded to complex FP32, which the tensor-core apply takes as its operand.  The same solve with
    the SIMT apply (double-float operand) reaches the same solution by different arithmetic."""
    w, oc, tc, simt, (s, t) = _case(2, 2, 2, 7, 9.0)
    try:
        rng = np.random.default_rng(5)
        S = np.stack([s[0] * (1.0 + 0.1 * k) for k in range(64)])
        T = np.stack([t[0] * rng.uniform(0.5, 1.5) for _ in range(64)])
        f, info = tc.solve(s=torch.from_numpy(S.reshape(-1)).cuda(), t=torch.from_numpy(T.reshape(-1)).cuda(),
                           tol=1e-9, form="mixed", nrhs=64)
        assert info["converged"], info
        f = f.cpu().numpy().reshape(64, -1)
        import oracle as O
        M = O.dense_face_matrix(oc.grid, oc.prob.R)
        for r in (0, 17, 63):
            ref = np.linalg.solve(M, O.rhs_face(oc.grid, oc.prob.H, S[r], T[r]))
            assert rel(f[r], ref) < 1e-7, r
        f2, info2 = simt.solve(s=torch.from_numpy(S.reshape(-1)).cuda(), t=torch.from_numpy(T.reshape(-1)).cuda(),
                               tol=1e-9, form="mixed", nrhs=64)
        assert info2["converged"], info2
        f2 = f2.cpu().numpy().reshape(64, -1)
        assert 0 < rel(f, f2) < 1e-7
    finally:
        tc.close()
        simt.close()
