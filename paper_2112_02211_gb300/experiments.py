"""Accuracy experiment of Sec. 6.2 (Table PlaneMinErr) on one GPU.

The test solution u = e^{i kappa (x+y+z)} e^x cosh(y) (z+1)^2 with the Gaussian
bump medium b = -1.5 exp(-160|x - 0.5|^2) is solved with n_c = 16 Chebyshev
points per leaf axis (q = 14 Gauss points per face edge) at a fixed number of
points per wavelength.  The wave number follows the tables of Sec. 6.1: a grid
of L leaves per axis at `ppw` points per wavelength spans 12 L / ppw
wavelengths (16 ppw on 4^3 leaves = 3 wavelengths), kappa = 2 pi 12 L / ppw.
The solve runs in FP64 to stagnation and E_h is the relative l2 error of the
recovered leaf solutions at the interior nodes.

    python -m paper_2112_02211_gb300.experiments [--L 4] [--ppw 24 16 9.6]
    python -m paper_2112_02211_gb300.experiments --large
    python -m paper_2112_02211_gb300.experiments --multi-rhs [--L 16]
"""

import argparse
import json
import math

import numpy as np


# Residual reduction that reaches the discretization's accuracy (Table PlaneResRed, Sec. 6.2),
# by points per wavelength.
RPRR = {24.0: 1e-13, 19.2: 1e-12, 16.0: 1e-10, 12.0: 1e-9, 9.6: 1e-8}


def accuracy_case(kind="plane", L=4, p=16, ppw=24.0, tol=1e-13):
    """One entry of the accuracy tables of Sec. 6.2-6.3: the modulated plane wave of eq. (plane)
    (kind "plane": Tables PlaneMinErr, PlaneResRed) or the bumps solution of eq. (bumps) (kind
    "bumps": Tables BumpsMinErr2, BumpsMinErr), both in the bump medium of eq. (source), n_c = p.
    Solved in the FP64 form twice: to `tol` (E_h, the discretization's accuracy) and to the
    table's residual reduction RPRR (E_h^it); E_h over all N = N_l (n_i + n_b) leaf unknowns
    (interior and Chebyshev face nodes).  kappa = 2 pi (12 L) / ppw: 12 points per leaf and
    axis, the count the paper's tables imply for n_c = 16 (48 points per axis on 4^3 leaves at
    3 wavelengths and 16 ppw)."""
    import torch

    import workloads as W

    from . import Solver, face_normals, nodes
    kappa = 2.0 * math.pi * 12.0 * L / ppw
    make = W.manufactured if kind == "plane" else W.manufactured_bumps
    w = make(L=L, p=p, kappa=kappa)
    xi, xf, xc = nodes(L, L, L, p, cheb_faces=True)
    nrm = np.broadcast_to(face_normals()[None, :, None, :], xf.shape)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    t = torch.from_numpy(w.sample_t(xf, nrm).reshape(-1)).cuda()
    rprr = RPRR.get(ppw, 1e-10)
    solver = Solver(L, L, L, p, kappa=kappa, eta=kappa, b=w.sample_b(xi), forms=("fp64",), cluster=0, max_rhs=2)
    try:
        f1, info1 = solver.solve(s=s, t=t, tol=tol, form="fp64")
        f2, info2 = solver.solve(s=s, t=t, tol=rprr, form="fp64")
        u, uf = solver.recover(torch.cat([f1, f2]), s=torch.cat([s, s]), nrhs=2, faces=True)
        u, uf = u.cpu().numpy().reshape(2, -1), uf.cpu().numpy().reshape(2, -1)
    finally:
        solver.close()
    ue, ufe = w.meta["u"](xi).reshape(-1), w.meta["u"](xc).reshape(-1)
    den = np.linalg.norm(ue) ** 2 + np.linalg.norm(ufe) ** 2

    def e_h(r):
        return float(np.sqrt((np.linalg.norm(u[r] - ue) ** 2 + np.linalg.norm(uf[r] - ufe) ** 2) / den))

    return {"kind": kind, "leaves": L, "p": p, "ppw": ppw, "kappa": kappa, "E_h": e_h(0), "E_h_it": e_h(1),
            "E_h_interior": float(np.linalg.norm(u[0] - ue) / np.linalg.norm(ue)), "rprr": rprr,
            "iterations": info1["iterations"], "iterations_rprr": info2["iterations"],
            "rel_residual": info1["rel_residual"], "rel_residual_rprr": info2["rel_residual"]}


def accuracy_table(L=4, p=16, ppws=(24.0, 16.0, 9.6), tol=1e-13):
    """Tables PlaneMinErr / PlaneResRed and BumpsMinErr2 (Sec. 6.2-6.3) on L^3 leaves: per points
    per wavelength one setup (both exact solutions live in the same bump medium at the same
    kappa, so they share the leaf maps), then for each solution the FP64 solve to `tol` (E_h)
    and to the table's residual reduction (E_h^it), as in accuracy_case."""
    import time

    import torch

    import workloads as W

    from . import Solver, face_normals, nodes
    xi, xf, xc = nodes(L, L, L, p, cheb_faces=True)
    nrm = np.broadcast_to(face_normals()[None, :, None, :], xf.shape)
    rows = []
    for ppw in ppws:
        kappa = 2.0 * math.pi * 12.0 * L / ppw
        rprr = RPRR.get(ppw, 1e-10)
        wp = W.manufactured(L=L, p=p, kappa=kappa)
        t0 = time.time()
        solver = Solver(L, L, L, p, kappa=kappa, eta=kappa, b=wp.sample_b(xi), forms=("fp64",), cluster=0,
                        max_rhs=4)
        setup_s = time.time() - t0
        try:
            # both solutions, each solved to tol (E_h) and to the table's residual reduction (E_h^it),
            # then one recovery of the four (the recovery repeats the leaf elimination)
            fs, ss, info = [], [], []
            kinds = (("plane", W.manufactured), ("bumps", W.manufactured_bumps))
            ws = [make(L=L, p=p, kappa=kappa) for _, make in kinds]
            for w in ws:
                s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
                t = torch.from_numpy(w.sample_t(xf, nrm).reshape(-1)).cuda()
                for tol_k in (tol, rprr):
                    f, inf = solver.solve(s=s, t=t, tol=tol_k, form="fp64")
                    fs.append(f)
                    ss.append(s)
                    info.append(inf)
            u, uf = solver.recover(torch.cat(fs), s=torch.cat(ss), nrhs=4, faces=True)
            u, uf = u.cpu().numpy().reshape(4, -1), uf.cpu().numpy().reshape(4, -1)
            for c, ((kind, _), w) in enumerate(zip(kinds, ws)):
                ue, ufe = w.meta["u"](xi).reshape(-1), w.meta["u"](xc).reshape(-1)
                den = np.linalg.norm(ue) ** 2 + np.linalg.norm(ufe) ** 2

                def e_h(r):
                    return float(np.sqrt((np.linalg.norm(u[r] - ue) ** 2 + np.linalg.norm(uf[r] - ufe) ** 2) / den))

                i1, i2 = info[2 * c], info[2 * c + 1]
                rows.append({"kind": kind, "leaves": L, "p": p, "ppw": ppw, "kappa": kappa, "E_h": e_h(2 * c),
                             "E_h_it": e_h(2 * c + 1), "rprr": rprr, "iterations": i1["iterations"],
                             "iterations_rprr": i2["iterations"], "rel_residual": i1["rel_residual"],
                             "setup_s": setup_s})
                print(json.dumps(rows[-1]), flush=True)
        finally:
            solver.close()
    return rows


def plane_min_err(L=4, p=16, ppw=24.0, tol=1e-13):
    """Table PlaneMinErr entry (see accuracy_case)."""
    return accuracy_case("plane", L=L, p=p, ppw=ppw, tol=tol)


def large_solve(L=32, steps=3, warmup=1):
    """The large single solve: 32^3 leaves, p = 10, kappa = eta = 200, smooth random complex
    medium, Gaussian source of width 0.01 at the centre, tol 1e-5, lean mixed form (FP32 maps,
    FP16 cluster inverses shared at lambda_bin 0.01 with complex-FP32 copies of the widely shared
    ones for the tensor cores, double-float Krylov basis).  Returns setup time, memory, the
    distinct blocks and the per-solve time, iterations and throughput (face unknowns/s), inputs
    resident on the GPU."""
    import time

    import torch

    import workloads as W

    from . import Solver, nodes
    w = W.large_32cubed(L=L)
    xi, xf = nodes(L, L, L, w.p)
    b = w.sample_b(xi)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    t0 = time.time()
    solver = Solver(L, L, L, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), lean=True, lambda_bin=0.01)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    try:
        out = torch.empty(solver.nf, dtype=torch.complex128, device="cuda")
        for _ in range(warmup):
            solver.solve(s=s, tol=w.tol, form="mixed", out=out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        solver.profile(enable=True, reset=True)
        e0.record()
        for _ in range(steps):
            _, info = solver.solve(s=s, tol=w.tol, form="mixed", out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile(enable=False, reset=True)
        mem = solver.memory_bytes
        blocks = solver.precond_info()
    finally:
        solver.close()
    return {"workload": f"large_{L}cubed", "leaves": L ** 3, "face_unknowns": solver.nf, "setup_s": setup_s,
            "device_bytes": mem, "clusters_k_blocks_b_blocks": blocks, "ms_per_solve": ms,
            "unknowns_per_s": solver.nf / (ms / 1e3),
            "iterations": info["iterations"], "rel_residual": info["rel_residual"],
            "phase_ms_per_solve": {k: v / steps for k, v in prof["ms"].items()}}


def multi_rhs(L=16, nrhs=64, restart=30, steps=2, warmup=1, precond=False):
    """The multi-RHS workload: L^3 leaves, p = 12 (q = 10, leaf ItI 600 x 600), kappa = eta = 60,
    five seeded bumps, 64 Gaussian sources of width 0.02, tol 1e-6; lean mixed form with the
    apply of all 64 right-hand sides on the tensor cores (tcgen05, three TF32 products).
    Restart 30 keeps the 64-RHS Krylov basis at 31 x 64 x N_f complex double-floats."""
    import time

    import torch

    import workloads as W

    from . import Solver, nodes
    w = W.multi_rhs_16cubed(L=L, nrhs=nrhs)
    xi, xf = nodes(L, L, L, w.p)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    t0 = time.time()
    solver = Solver(L, L, L, w.p, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi), forms=("mixed",), lean=True,
                    restart=restart, max_rhs=nrhs, cluster=2 if precond else 0)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    try:
        out = torch.empty(nrhs * solver.nf, dtype=torch.complex128, device="cuda")
        for _ in range(warmup):
            solver.solve(s=s, tol=w.tol, form="mixed", out=out, nrhs=nrhs)
        solver.profile(enable=True, reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            _, info = solver.solve(s=s, tol=w.tol, form="mixed", out=out, nrhs=nrhs)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile(enable=False, reset=True)
        nb, q2 = solver.nb, solver.q * solver.q
    finally:
        solver.close()
    napply = prof["count"]["apply"]
    apply_ms = prof["ms"]["apply"] / max(1, napply)
    r_bytes = L ** 3 * nb * nb * 8
    flops = 8.0 * L ** 3 * nb * nb * nrhs
    return {"workload": f"multi_rhs_{L}cubed", "nrhs": nrhs, "face_unknowns_per_rhs": solver.nf,
            "setup_s": setup_s, "ms_per_solve": ms, "unknowns_per_s": nrhs * solver.nf / (ms / 1e3),
            "iterations": info["iterations"], "rel_residual": info["rel_residual"],
            "apply_ms": apply_ms, "apply_R_GBps": r_bytes / (apply_ms / 1e3) / 1e9,
            "apply_complex_TFLOPs": flops / (apply_ms / 1e3) / 1e12,
            "phase_ms_per_solve": {k: v / steps for k, v in prof["ms"].items()}}


def precond_sharing(L=16, bins=(0.0, 0.001, 0.01, 0.05), steps=2, warmup=1):
    """Shared preconditioner blocks on the bump workload (16^3 leaves, p = 10, kappa = 40):
    for each bin width of the homogenized constants (relative to max |lambda|), the distinct
    K_c / B blocks, setup time, iterations and time per mixed-form solve (FP16 blocks).  The
    solutions agree to the tolerance whatever the bins."""
    import time

    import torch

    import workloads as W

    from . import Solver, nodes
    w = W.bump_16cubed(L=L)
    xi, xf = nodes(L, L, L, w.p)
    b = w.sample_b(xi)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    rows = []
    ref = None
    for delta in bins:
        t0 = time.time()
        solver = Solver(L, L, L, w.p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), lambda_bin=delta)
        torch.cuda.synchronize()
        setup_s = time.time() - t0
        try:
            out = torch.empty(solver.nf, dtype=torch.complex128, device="cuda")
            for _ in range(warmup):
                solver.solve(s=s, tol=w.tol, form="mixed", out=out)
            solver.profile(enable=True, reset=True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                _, info = solver.solve(s=s, tol=w.tol, form="mixed", out=out)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            prof = solver.profile(enable=False, reset=True)
            ncl, kb, bb = solver.precond_info()
            mem = solver.memory_bytes
        finally:
            solver.close()
        if ref is None:
            ref = out.clone()
        diff = float(torch.linalg.norm(out - ref).item() / torch.linalg.norm(ref).item())
        rows.append({"lambda_bin": delta, "clusters": ncl, "distinct_K": kb, "distinct_B": bb, "setup_s": setup_s,
                     "device_bytes": mem, "iterations": info["iterations"], "ms_per_solve": ms,
                     "unknowns_per_s": solver.nf / (ms / 1e3), "rel_diff_vs_first": diff,
                     "phase_ms_per_solve": {k: v / steps for k, v in prof["ms"].items()}})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=4)
    ap.add_argument("--ppw", type=float, nargs="*", default=[24.0, 19.2, 16.0, 12.0, 9.6])
    ap.add_argument("--kind", nargs="*", default=["plane"], choices=["plane", "bumps"],
                    help="exact solution of the accuracy runs: eq. (plane) and/or eq. (bumps)")
    ap.add_argument("--large", action="store_true", help="run the 32^3-leaf large solve instead")
    ap.add_argument("--multi-rhs", action="store_true", help="run the 64-RHS tensor-core workload instead")
    ap.add_argument("--sharing", action="store_true", help="run the shared-preconditioner-block sweep instead")
    ap.add_argument("--table", action="store_true",
                    help="both accuracy tables, one setup per points-per-wavelength value")
    args = ap.parse_args()
    if args.table:
        accuracy_table(L=args.L, ppws=tuple(args.ppw))
        return
    if args.sharing:
        for row in precond_sharing(L=args.L if args.L != 4 else 16):
            print(json.dumps(row), flush=True)
        return
    if args.large:
        print(json.dumps(large_solve()), flush=True)
        return
    if args.multi_rhs:
        print(json.dumps(multi_rhs(L=args.L if args.L != 4 else 16)), flush=True)
        return
    for kind in args.kind:
        for ppw in args.ppw:
            print(json.dumps(accuracy_case(kind, L=args.L, ppw=ppw)), flush=True)


if __name__ == "__main__":
    main()
