"""The launch-shape autotuner: at setup it times the candidate shapes (matrix rows per warp,
resident CTAs per SM) of the ItI apply and of the preconditioner's SIMT stage K and keeps the
fastest.  A shape changes how rows are distributed, never how a row is summed (one warp, lanes
in a fixed order), so a tuned handle and an untuned one on the same medium must give the same
applies, preconditioner applies and solutions bit for bit."""

import numpy as np
import pytest

import workloads as W
from gpu_cases import gpu_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")


def test_tuned_shapes_give_the_default_results():
    w = W.scaled(W.bump_16cubed(), 4)
    w.p = 8
    xi, xf, b, s, t = gpu_inputs(w, hps)
    kw = dict(kappa=w.kappa, eta=w.eta, b=b, max_rhs=4, lambda_bin=0.01)
    tuned = hps.Solver(4, 4, 4, 8, autotune=True, **kw)
    plain = hps.Solver(4, 4, 4, 8, autotune=False, **kw)
    try:
        st, sp = tuned.launch_shapes(), plain.launch_shapes()
        assert st["tuned"] and not sp["tuned"]
        assert sp["apply_rows_per_warp"][0][0] == 4 and sp["stage_k_rows_per_warp"][0] == 4
        for rows in st["apply_rows_per_warp"] + [st["stage_k_rows_per_warp"]]:
            assert all(r in (1, 2, 4, 8) for r in rows)
        for c in st["apply_ctas_per_sm"] + [st["stage_k_ctas_per_sm"]]:
            assert all(0 <= v <= 3 for v in c)
        rng = np.random.default_rng(77)
        for nrhs in (1, 3):
            f = rng.standard_normal(nrhs * tuned.nf) + 1j * rng.standard_normal(nrhs * tuned.nf)
            for dt in (torch.complex128, torch.complex64):
                fd = torch.from_numpy(f).to(dt).cuda()
                assert torch.equal(tuned.apply(fd), plain.apply(fd)), (nrhs, dt)
                assert torch.equal(tuned.precond(fd), plain.precond(fd)), (nrhs, dt)
        sd = torch.from_numpy(s.reshape(-1)).cuda()
        for form in ("mixed", "fp64"):
            ft, it = tuned.solve(s=sd, tol=1e-8, form=form)
            fp, ip = plain.solve(s=sd, tol=1e-8, form=form)
            assert it["iterations"] == ip["iterations"] and torch.equal(ft, fp), form
    finally:
        tuned.close()
        plain.close()
