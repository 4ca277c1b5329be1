"""The multi-RHS and large configurations on scaled grids, element by element against the oracle.

The scaled instances keep each configuration's medium, sources, p, q and kappa*h and run in the
configuration's form -- the memory-lean mixed form with 2x2x2 cluster blocks binned at 0.01:
* multi-RHS: 6^3 leaves, p = 12, kappa = 22.5, 64 right-hand sides in one solve: tensor-core
  apply (three TF32 products), batched stage B, every cluster block on the tensor cores against
  (member, right-hand side) columns, double-float Krylov basis, GMRES(50);
* large: 8^3 leaves, p = 10, kappa = 50, complex medium (Im b in [0, 0.05]), one source.
The oracle's solutions were written by tests/golden/make_scaled_configs.py (oracle only).  The
solves run at the configurations' tolerances (1e-6, 1e-5) and at 1e-9; at 1e-9 the solution
must match the oracle to the mixed form's bar of 1e-6 (lean mode restarts from an FP64-accurate
residual: FP32 maps plus their FP16 remainders)."""

import os

import numpy as np
import pytest

import workloads as W
from gpu_cases import gpu_inputs, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.load(os.path.join(GOLDEN, f"scaled_{name}.npz"))


def test_multi_rhs_scaled_matches_oracle():
    g = _golden("multi_rhs")
    L, p, kappa = int(g["L"]), int(g["p"]), float(g["kappa"])
    w = W.multi_rhs_16cubed(L=L, p=p, kappa=kappa)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(L, L, L, p, kappa=kappa, eta=kappa, b=b, forms=("mixed",), lean=True, max_rhs=64,
                        lambda_bin=0.01)
    try:
        sd = torch.from_numpy(s.reshape(-1)).cuda()
        f, info = solver.solve(s=sd, tol=1e-6, form="mixed", nrhs=64)
        assert info["converged"] and info["rel_residual"] <= 1e-6, info
        f, info = solver.solve(s=sd, tol=1e-9, form="mixed", nrhs=64)
        assert info["converged"], info
        f = f.cpu().numpy().reshape(64, -1)
        for k, r in enumerate(g["rhs"]):
            assert rel(f[r], g["f"][k].astype(np.complex128)) < 1e-6, r
    finally:
        solver.close()


def test_large_scaled_matches_oracle():
    g = _golden("large")
    L, p, kappa = int(g["L"]), int(g["p"]), float(g["kappa"])
    w = W.large_32cubed(L=L, p=p, kappa=kappa)
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(L, L, L, p, kappa=kappa, eta=kappa, b=b, forms=("mixed",), lean=True, lambda_bin=0.01)
    try:
        sd = torch.from_numpy(s.reshape(-1)).cuda()
        f, info = solver.solve(s=sd, tol=1e-5, form="mixed")
        assert info["converged"] and info["rel_residual"] <= 1e-5, info
        f, info = solver.solve(s=sd, tol=1e-9, form="mixed")
        assert info["converged"], info
        assert rel(f.cpu().numpy(), g["f"][0].astype(np.complex128)) < 1e-6
    finally:
        solver.close()
