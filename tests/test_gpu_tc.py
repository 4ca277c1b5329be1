"""The tensor-core apply (64 right-hand sides per launch, three TF32 products
with FP32 accumulation) against the oracle, the SIMT apply and an emulation of
its arithmetic.

Bars from the error model of tests/tc_model.py (pinned on the CPU in
tests/test_tf32_bounds.py): the operand split keeps ~2^-22 per product term,
and the tensor cores' accumulator truncates (8 exact products and the FP32
accumulator aligned to the largest exponent, 2 guard bits, normalized toward
zero).  Those truncations drift toward zero by ~1e-5 relative over a 1200-term
row at p = 12 (~3e-6 at p = 7).  The test emulates that arithmetic for the
same FP32 maps and vectors and checks (1) the kernel against the emulation
element by element, to the FP32 rounding of the stored result (a wrong tile,
index, sign or split would be off by far more), and (2) the kernel against the
oracle within the emulation's own distance from the oracle (plus the FP32
storage of the maps and of the result)."""

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


def _model_apply(oc, R32, f):
    """y = f + Pi G with G = R F computed as the tensor-core kernel does (tc_model, GB300
    accumulation), the result rounded to complex FP32 like the kernel's store."""
    import tc_model as T
    g = oc.grid
    nb, q2 = g.nb, g.q * g.q
    y = f.copy()
    for leaf in range(g.nleaves):
        rows, dst = [], []
        for face in range(6):
            nbr = g.neighbor(leaf, face)
            if nbr >= 0:
                rows += [face * q2 + j for j in range(q2)]
                dst += [nbr * nb + (face ^ 1) * q2 + j for j in range(q2)]
        if not rows:
            continue
        F = f[:, leaf * nb:(leaf + 1) * nb].T
        A = T.complex_as_real(R32[leaf][rows].astype(np.complex128)).astype(np.float32)
        B = T.operands(F.astype(np.complex128)).astype(np.float32)
        D = T.tc_product(A, B, *T.GB300).astype(np.float32)
        k = F.shape[1]
        fd = f[:, dst]
        y[:, dst] = (fd.real + D[:, :k].T) + 1j * (fd.imag + D[:, k:].T)
    return y.astype(np.complex64)


# p = 12: n_b = 600 -> five 128-row tiles (the last one partial), 38 K blocks;
# p = 7: n_b = 150 -> two tiles, a ragged last K block.
@pytest.mark.parametrize("shape,p", [((2, 2, 1), 12), ((3, 1, 1), 7)])
def test_tc_apply_matches_model_oracle_and_simt(shape, p):
    w, oc, tc, simt, _ = _case(*shape, p, 9.0)
    try:
        rng = np.random.default_rng(p)
        f = (rng.standard_normal((64, oc.grid.nf)) + 1j * rng.standard_normal((64, oc.grid.nf))).astype(np.complex64)
        fd = torch.from_numpy(f.reshape(-1)).cuda()
        y_tc = tc.apply(fd).cpu().numpy().reshape(64, -1)
        y_simt = simt.apply(fd).cpu().numpy().reshape(64, -1)
        ref = np.stack([oc.apply(f[r].astype(np.complex128)) for r in range(64)])
        R32 = [tc.export("R", i).reshape(oc.grid.nb, oc.grid.nb).astype(np.complex64) for i in range(oc.grid.nleaves)]
        y_model = _model_apply(oc, R32, f)
        # (1) the kernel is the modelled arithmetic, to the FP32 rounding of the result
        assert rel(y_tc, y_model) < 1e-7
        for r in range(64):
            assert rel(y_tc[r], y_model[r]) < 2e-7, r
        # (2) against the oracle: the model's own error, plus FP32 storage of maps and result
        e_model = rel(y_model, ref)
        assert 1e-7 < e_model < (3e-5 if p == 12 else 1e-5)
        assert rel(y_tc, ref) < 1.05 * e_model + 1e-7
        assert rel(y_simt, ref) < 3e-7
        assert rel(y_tc, y_simt) < 1.05 * e_model + 3e-7
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
