"""Bounded device waits (failure detection without a GPU fault): every mbarrier wait of the
tensor-core kernels gives up after a limit; the CTA then sets the handle's error word, stops
issuing work, waits (bounded) for its own copies and tensor-core operations, frees its tensor
memory and returns, and the solve reports HPS_ETIMEOUT.

The test makes one wait run out on purpose through the library's test hook: one warp of CTA 0
of the multi-RHS tensor-core apply leaves out one mbarrier arrival (an arrival that nothing
else makes), with a short wait limit.  Expected: HPS_ETIMEOUT from the solve within seconds, a
usable GPU context afterwards, and -- with the hook cleared -- the same handle solving again to
the same result as before, bit for bit."""

import time

import numpy as np
import pytest

import workloads as W
from gpu_cases import gpu_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")
from paper_2112_02211_gb300 import _native as N  # noqa: E402


def test_bounded_wait_times_out_and_the_handle_recovers():
    w = W.manufactured(L=1, p=7, kappa=9.0)
    w.nx, w.ny, w.nz = 2, 2, 2
    xi, xf, b, s, t = gpu_inputs(w, hps)
    solver = hps.Solver(2, 2, 2, 7, kappa=9.0, eta=w.eta, b=b, forms=("mixed",), max_rhs=64, cluster=0)
    lib = N.load()
    try:
        S = torch.from_numpy(np.stack([s[0] * (1.0 + 0.1 * k) for k in range(64)]).reshape(-1)).cuda()
        f_ref, info = solver.solve(s=S, tol=1e-9, form="mixed", nrhs=64)
        assert info["converged"], info
        f_ref = f_ref.clone()
        assert lib.hps_test_inject(solver.handle, N.HPS_INJECT_SKIP_ARRIVAL, 4096) == N.HPS_OK
        t0 = time.time()
        with pytest.raises(hps.HPSError) as err:
            solver.solve(s=S, tol=1e-9, form="mixed", nrhs=64)
        assert err.value.code == N.HPS_ETIMEOUT
        assert time.time() - t0 < 60
        # the context still works
        assert float(torch.ones(1000, device="cuda").sum()) == 1000.0
        torch.cuda.synchronize()
        assert lib.hps_test_inject(solver.handle, N.HPS_INJECT_NONE, 0) == N.HPS_OK
        f2, info2 = solver.solve(s=S, tol=1e-9, form="mixed", nrhs=64)
        assert info2["converged"] and info2["iterations"] == info["iterations"]
        assert torch.equal(f2, f_ref)
    finally:
        lib.hps_test_inject(solver.handle, N.HPS_INJECT_NONE, 0)
        solver.close()


def test_inject_rejects_bad_arguments():
    lib = N.load()
    assert lib.hps_test_inject(None, N.HPS_INJECT_NONE, 0) == N.HPS_EINVAL
