"""Writes the oracle's solutions of the scaled multi-RHS and large configurations to
tests/golden/scaled_*.npz.  Calls only oracle/ (and the input generators in workloads/).

Scaled instances keep the configuration's medium, sources, p, q and kappa*h (so the points per
wavelength), on fewer leaves:
* multi-RHS: 6^3 leaves, p = 12, kappa = eta = 60 * 6/16 = 22.5, five seeded bumps, 64 Gaussian
  sources of width 0.02 (solutions stored for sources 0, 31 and 63);
* large: 8^3 leaves, p = 10, kappa = eta = 200 * 8/32 = 50, the smooth random complex medium,
  one Gaussian source of width 0.01 at the centre.
Each solution is the oracle's restarted GMRES on (I + Pi R) f = -Pi H s to a relative residual of
1e-13, stored as complex64 (6e-8 relative, far below the 1e-6 bar it is compared at).

    python tests/golden/make_scaled_configs.py        # a few minutes on 8 cores
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

CASES = {
    "multi_rhs": dict(make=lambda: W.multi_rhs_16cubed(L=6, p=12, kappa=60.0 * 6 / 16), rhs=(0, 31, 63)),
    "large": dict(make=lambda: W.large_32cubed(L=8, p=10, kappa=200.0 * 8 / 32), rhs=(0,)),
}


def solve_case(name):
    spec = CASES[name]
    w = spec["make"]()
    g = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi = O.interior_nodes(g)
    t0 = time.time()
    prob = O.build_problem(g, w.kappa, w.eta, w.sample_b(xi))
    s_all = w.sample_s(xi)
    sols, res = [], []
    for r in spec["rhs"]:
        rhs = O.rhs_face(g, prob.H, s_all[r], None)
        f, its, hist = O.gmres(lambda v: O.apply_face(g, prob.R, v), rhs, tol=1e-13, restart=50)
        rr = np.linalg.norm(rhs - O.apply_face(g, prob.R, f)) / np.linalg.norm(rhs)
        assert rr < 1e-12, rr
        sols.append(f.astype(np.complex64))
        res.append(rr)
    out = os.path.join(HERE, f"scaled_{name}.npz")
    np.savez_compressed(out, f=np.stack(sols), rhs=np.array(spec["rhs"]), L=w.nx, p=w.p, kappa=w.kappa,
                        rel_residual=np.array(res))
    print(f"{name}: {g.nleaves} leaves, p = {w.p}, kappa = {w.kappa}, {len(sols)} solutions, "
          f"residuals {res}, {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        solve_case(n)
