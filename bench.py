#!/usr/bin/env python
"""Benchmark of the iterative HPS Helmholtz solver on one GB300 per rank.

Workload (synthetic, seeded): 16^3 = 4096 leaves on (0,1)^3, Chebyshev order
p = 10, q = 8 Gauss points per face edge (1,572,864 face unknowns),
kappa = eta = 40, medium b = 1.5 exp(-160 |x - c|^2), source
s = exp(-400 |x - x0|^2), t = 0, relative tolerance 1e-6.

A step is one solve to tolerance through the C ABI: RHS build, restarted
GMRES(50) with the leaf ItI apply + face swap, the cluster block-Jacobi
preconditioner, classical Gram-Schmidt Arnoldi (a second pass where
Rutishauser's test asks for it) and FP64-accurate restart residuals.  `value`
is face unknowns solved per second with the inputs already in HBM (mixed form:
complex-FP32 operators, double-float Krylov basis, restart residual from the
FP32 maps plus their FP16 remainders at tol >= 1e-8, else FP64); the FP64
form and the runs without preconditioner are reported beside it.  Setup
(leaf maps, preconditioner) is outside the timed region.

--impl reference times the CPU oracle instead (see oracle/), on a bounded
sample of the same workload.  Under torchrun each rank solves its own
replica (no data-path collective); rank 0 prints one JSON line.
"""

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
T_START = time.time()
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "GMRES unknowns solved/s (mixed vs FP64, rel err<=1e-6); apply GB/s; p50/p99"
UNIT = "unknowns/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--L", type=int, default=16, help="leaves per axis (16 = the benchmark workload)")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / no-preconditioner comparison runs")
    ap.add_argument("--cpu-sample-L", type=int, default=4)
    ap.add_argument("--serving-requests", type=int, default=10,
                    help="requests of the serving stream timed after the solves (0 = skip)")
    ap.add_argument("--lambda-bin", type=float, default=0.01,
                    help="bin width of the homogenized constants, relative to max |lambda| (0 = per-leaf)")
    ap.add_argument("--no-full-system", action="store_true",
                    help="skip the comparison solve of the paper's global-system path")
    ap.add_argument("--unbinned", action="store_true",
                    help="also time the solve with per-leaf (unbinned) preconditioner blocks")
    ap.add_argument("--configs", default="multi_rhs,large",
                    help="full-size configurations timed after the headline (comma list of multi_rhs, large; "
                         "'' = none)")
    ap.add_argument("--budget-s", type=float, default=1500.0,
                    help="wall-time budget of the whole run: a configuration leg that would end after it is "
                         "skipped (with a note)")
    return ap.parse_args()


# --------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# --------------------------------------------------------------------------------------------
class Dist:
    def __init__(self, backend=None, group=True):
        """Rank and world from the torchrun environment; a process group only when `group` (the
        reference arm runs on rank 0 alone and needs none)."""
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1 and group:
            import torch.distributed as dist
            dist.init_process_group(backend=backend or "nccl")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        return self._reduce(x, "max")

    def sum(self, x):
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(unknowns_per_rank, seconds_per_rank):
    """Whole-job throughput: all ranks' unknowns over the slowest rank's time."""
    return sum(unknowns_per_rank) / max(seconds_per_rank)


# --------------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for n, f in zip(names[1:], flags[1:]):
                if f.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------------------------------
# algorithmic bytes per launch: the bytes each kernel must move at least (matrix entries read
# once, vectors read and written once), the numerator of the roofline fraction
# --------------------------------------------------------------------------------------------
def interior_face_pairs(L):
    return 6 * L ** 3 - 6 * L * L


def apply_bytes(L, q, mat_bytes, in_bytes, out_bytes):
    """Rows of R actually read (faces with a neighbour) + f read + f read at the target + y write."""
    nb = 6 * q * q
    nf = L ** 3 * nb
    return interior_face_pairs(L) * q * q * nb * mat_bytes + nf * (2 * in_bytes + out_bytes)


def precond_bytes(L, q, mat_bytes, vec_bytes, in_bytes=None, scale_bytes=0, k_blocks=None, b_blocks=None):
    """Stage K: every distinct K_c block once (+ one row scale per row for FP16 blocks) + t read +
    z_int write per cluster.  Stage B: every distinct B block once (+ row scales) + r read once +
    t and z_ext written.  Without sharing k_blocks = clusters, b_blocks = leaves.  L even."""
    in_bytes = vec_bytes if in_bytes is None else in_bytes
    q2 = q * q
    ncl = (L // 2) ** 3
    k_blocks = ncl if k_blocks is None else k_blocks
    b_blocks = L ** 3 if b_blocks is None else b_blocks
    nint = 24 * q2
    kb = k_blocks * nint * (nint * mat_bytes + scale_bytes) + ncl * nint * 2 * vec_bytes
    nf = L ** 3 * 6 * q2
    bb = b_blocks * (3 * q2) * (3 * q2 * mat_bytes + scale_bytes) + nf * in_bytes + nf * vec_bytes
    return kb, bb


def precond_k_flops(L, q):
    """Stage K: one complex multiply-add (8 real flops) per K_c entry per cluster."""
    nint = 24 * q * q
    return 8.0 * (L // 2) ** 3 * nint * nint


def workload_name(w):
    L, p, q = w.nx, w.p, w.q
    return (f"bump_{L}cubed: {L}^3 leaves, p={p}, q={q}, kappa=eta={w.kappa:g}, "
            f"b=1.5exp(-160|x-c|^2), s=exp(-400|x-x0|^2), t=0, tol={w.tol:g}")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def committed_traffic(kernel):
    """ncu DRAM bytes per launch from profiles/, valid only for the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2112_02211_gb300", "csrc", "apply.cu")
    try:
        with open(path) as fh:
            d = json.load(fh)
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        e = d.get(kernel)
        if e and e.get("apply_cu_sha256_16") == digest:
            return e["bytes_per_launch"]
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------------
def run_gpu(args, dist):
    import torch

    import paper_2112_02211_gb300 as hps

    torch.cuda.set_device(dist.local)
    w = W.bump_16cubed(L=args.L)
    L, p, q = w.nx, w.p, w.q
    xi, xf = hps.nodes(L, L, L, p)
    b = w.sample_b(xi)
    s = w.sample_s(xi).reshape(-1)
    t0 = time.time()
    solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=b, device=dist.local, lambda_bin=args.lambda_bin)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    ncl, k_blocks, b_blocks = solver.precond_info()
    shapes = solver.launch_shapes()
    nf = solver.nf
    s_dev = torch.from_numpy(s).cuda()
    out = torch.empty(nf, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(form, precond, steps, warmup, profile=False, clocks=None):
        for _ in range(warmup):
            _, info = solver.solve(s=s_dev, tol=w.tol, form=form, out=out, precond=precond)
        solver.profile(enable=profile, reset=True)
        dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = []
        for _ in range(steps):
            _, info = solver.solve(s=s_dev, tol=w.tol, form=form, out=out, precond=precond)
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        ck = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile(enable=False, reset=True)
        return ms, infos, prof, ck

    # headline: mixed form with the preconditioner
    clocks = Clocks(dist.local)
    ms, infos, prof, ck = timed("mixed", True, args.steps, args.warmup, profile=True, clocks=clocks)
    f_mixed = out.clone()
    ms_max = dist.max(ms)
    value = aggregate([nf * args.steps] * dist.world, [ms_max * args.steps / 1e3] * dist.world) \
        if dist.world > 1 else nf / (ms / 1e3)
    if dist.world > 1:
        value = dist.world * nf / (ms_max / 1e3)

    # end to end through the same call with host buffers (H2D of s, D2H of f inside)
    s_host = s.copy()
    f_host = np.zeros(nf, dtype=np.complex128)
    solver.solve(s=s_host, tol=w.tol, form="mixed", out=f_host)
    dist.barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        solver.solve(s=s_host, tol=w.tol, form="mixed", out=f_host)
    e2e_s = (time.perf_counter() - te) / args.steps
    e2e_s = dist.max(e2e_s)
    e2e_value = dist.world * nf / e2e_s

    # comparison runs (fewer steps): FP64 form, and both forms without the preconditioner
    compare = {}
    if not args.no_compare:
        for form, pc in (("fp64", True), ("mixed", False), ("fp64", False)):
            c_ms, c_infos, c_prof, _ = timed(form, pc, 1, 1, profile=True)
            key = f"{form}{'' if pc else '_no_precond'}"
            compare[key] = {"unknowns_per_s": nf / (c_ms / 1e3), "ms_per_solve": c_ms,
                            "iterations": c_infos[-1]["iterations"], "rel_residual": c_infos[-1]["rel_residual"],
                            "phase_ms": {k: round(v, 3) for k, v in c_prof["ms"].items()}}
            if key == "fp64":
                compare[key]["mixed_vs_fp64_rel_diff"] = float(
                    torch.linalg.norm(f_mixed - out).item() / torch.linalg.norm(out).item())

    # per-leaf (unbinned) preconditioner blocks, mixed form, for comparison
    if not args.no_compare and args.unbinned and args.lambda_bin > 0:
        solver.close()
        solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=b, device=dist.local, forms=("mixed",))
        c_ms, c_infos, c_prof, _ = timed("mixed", True, 1, 1, profile=True)
        compare["mixed_unbinned"] = {
            "unknowns_per_s": nf / (c_ms / 1e3), "ms_per_solve": c_ms, "iterations": c_infos[-1]["iterations"],
            "rel_residual": c_infos[-1]["rel_residual"], "k_blocks": solver.precond_info()[1],
            "phase_ms": {k: round(v, 3) for k, v in c_prof["ms"].items()},
            "rel_diff_vs_headline": float(torch.linalg.norm(f_mixed - out).item() / torch.linalg.norm(out).item())}

    # the paper's own design: GMRES on the global system with the per-leaf homogenized
    # block-Jacobi preconditioner (Algorithms 1-4), mixed form, same binning
    if not args.no_compare and not args.no_full_system:
        solver.close()
        solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=b, device=dist.local, forms=("mixed",),
                            cluster=0, full_system=True, lambda_bin=args.lambda_bin)
        for _ in range(1):
            solver.full_solve(s=s_dev, tol=w.tol, form="mixed")
        solver.profile(enable=True, reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u_full, finfo = solver.full_solve(s=s_dev, tol=w.tol, form="mixed")
        e1.record(stream)
        torch.cuda.synchronize()
        f_ms = e0.elapsed_time(e1)
        fprof = solver.profile(enable=False, reset=True)
        compare["full_system_mixed"] = {
            "unknowns_per_s": nf / (f_ms / 1e3), "ms_per_solve": f_ms, "iterations": finfo["iterations"],
            "rel_residual": finfo["rel_residual"], "global_unknowns": int(u_full.numel()),
            "phase_ms": {k: round(v, 3) for k, v in fprof["ms"].items()},
            "note": "unknowns/s counted in face unknowns (N_f) for comparison; the global system has "
                    "N_l (n_i + n_b) unknowns"}

    # roofline of the dominant kernel and of the ItI apply, from the library's events
    pk, pk_src = peaks()
    q2 = q * q
    # c64 maps, c64 input, double-float (16-byte) output
    a_bytes = apply_bytes(L, q, 8, 8, 16)
    # FP16 blocks (4 bytes per complex entry + a 4-byte scale per row), c64 vectors,
    # double-float (16-byte) input to stage B
    kb, bb = precond_bytes(L, q, 4, 8, in_bytes=16, scale_bytes=4, k_blocks=k_blocks, b_blocks=b_blocks)
    phases = {"apply": a_bytes, "precond_k": kb, "precond_b": bb}
    rpw = shapes["apply_rows_per_warp"][0][0]
    kernels = {"apply": f"seg_gemv_kernel<ApplyP<float2,float2,float4>,1,{rpw}> (rows per warp chosen at setup)",
               "precond_k": "tc_precond16_kernel<false> (every cluster block on the tensor cores, kind::f16, "
                            "t scaled per cluster as two FP16 terms) when the clusters are uniform, else "
                            "seg_gemv_kernel<PrecKP<__half2,float2,float2>,1,R>",
               "precond_b": "prec_b_kernel<__half2,float4,float2,1> (one leaf per item, one thread per row, "
                            "B transposed)"}
    roof = {}
    for ph, by in phases.items():
        cnt = prof["count"][ph]
        if cnt:
            dur = prof["ms"][ph] / cnt / 1e3
            ach = by / dur / 1e9
            roof[ph] = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk, "unit": "GB/s",
                        "frac": round(ach / pk, 4), "traffic": committed_traffic(ph),
                        "algorithmic_bytes": by, "avg_launch_ms": round(dur * 1e3, 4), "launches": cnt,
                        "kernel": kernels[ph], "peak_source": pk_src}
            if ph == "precond_k":
                # shared blocks: a GEMM for the widely shared block on the tensor cores plus
                # grouped GEMVs; the flop count beside the byte count
                fl = precond_k_flops(L, q)
                roof[ph]["algorithmic_flops"] = fl
                roof[ph]["flops_achieved_tflops"] = round(fl / dur / 1e12, 2)
    dominant = max(roof, key=lambda k: prof["ms"][k]) if roof else None
    iters = infos[-1]["iterations"]
    rec = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 operators, double-float Krylov, f64 residual",
        "data": "synthetic",
        "config": {
            "workload": workload_name(w),
            "form": "mixed (complex-FP32 apply and preconditioner, classical Gram-Schmidt Arnoldi in "
                    "double-float with a second pass on Rutishauser's test, restart residual from the "
                    "FP32 maps plus FP16 remainders (FP64-level))",
            "launch_shapes": shapes,
            "preconditioner": "2x2x2 cluster block Jacobi, homogenized leaf maps, blocks in FP16 with FP32 row scales",
            "lambda_bin": args.lambda_bin,
            "precond_blocks": {"clusters": ncl, "distinct_K": k_blocks, "distinct_B": b_blocks},
            "restart": 50,
            "face_unknowns": nf,
            "paper_unknowns": L ** 3 * ((p - 2) ** 3 + 6 * (p - 2) ** 2),
            "parallelism": f"replicas x{dist.world}",
            "l2": "inputs larger than L2 (leaf maps 4.8 GB c64 per apply)",
            "setup_s": round(setup_s, 2),
        },
        "iterations": iters,
        "cycles": infos[-1]["cycles"],
        "rel_residual": infos[-1]["rel_residual"],
        "paper_unknowns_per_s": dist.world * L ** 3 * ((p - 2) ** 3 + 6 * (p - 2) ** 2) / (ms_max / 1e3),
        "phase_ms_per_solve": {k: round(v / args.steps, 3) for k, v in prof["ms"].items()},
        "roofline": roof.get(dominant),
        "roofline_apply": roof.get("apply"),
        "roofline_all": roof,
        "gpu_launches": prof["launches"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(s_host.nbytes),
                "d2h_bytes_per_step": int(f_host.nbytes)},
        "clocks": ck,
        "compare": compare,
    }
    solver.close()
    if args.serving_requests > 0:
        rec["serving"] = run_serving(args, dist)
    extra = [c for c in args.configs.split(",") if c]
    if extra:
        rec["configurations"] = {}
        # measured wall time of each leg (setup dominates: FP64 elimination of every leaf)
        expected_s = {"multi_rhs": 340.0, "large": 430.0}
        for name in extra:
            elapsed = time.time() - T_START
            if elapsed + expected_s.get(name, 300.0) > args.budget_s:
                rec["configurations"][name] = {"skipped": f"would end after the {args.budget_s:.0f} s budget "
                                                          f"({elapsed:.0f} s elapsed)"}
                continue
            rec["configurations"][name] = run_config(name, dist)
    return rec


def tf32_peak():
    """Dense TF32 tensor peak for the tensor-core kernels: the measured BF16 burst figure times
    the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s dense)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"]) * (1.1 / 2.25), "measured bf16 x nominal tf32/bf16"
    except Exception:
        return 1900.0 * (1.1 / 2.25), "fallback bf16 x nominal tf32/bf16"


def run_config(name, dist):
    """One full-size configuration in its own form (lean mixed, 2x2x2 cluster blocks binned at
    0.01), inputs resident in HBM, CUDA events around `steps` solves after one warm-up:
    * multi_rhs: 16^3 leaves, p = 12, kappa = 60, five bumps, 64 Gaussian sources, tol 1e-6,
      GMRES(50) (30 if the basis does not fit); apply and stage K of the 64 right-hand sides on
      the tensor cores;
    * large: 32^3 leaves, p = 10, kappa = 200, smooth random complex medium, tol 1e-5, GMRES(50).
    Unknowns/s counts face unknowns over all right-hand sides."""
    import torch

    import paper_2112_02211_gb300 as hps

    if name == "multi_rhs":
        w, nrhs, steps = W.multi_rhs_16cubed(), 64, 1
    elif name == "large":
        w, nrhs, steps = W.large_32cubed(), 1, 3
    else:
        return {"error": f"unknown configuration {name}"}
    L, p, q = w.nx, w.p, w.q
    xi, xf = hps.nodes(L, L, L, p)
    s = torch.from_numpy(w.sample_s(xi).reshape(-1)).cuda()
    b = w.sample_b(xi)
    solver, restart, setup_s = None, None, None
    for m in (50, 30):
        try:
            t0 = time.time()
            solver = hps.Solver(L, L, L, p, kappa=w.kappa, eta=w.eta, b=b, forms=("mixed",), lean=True,
                                lambda_bin=0.01, max_rhs=nrhs, restart=m, device=dist.local)
            torch.cuda.synchronize()
            setup_s = time.time() - t0
            out = torch.empty(nrhs * solver.nf, dtype=torch.complex128, device="cuda")
            solver.solve(s=s, tol=w.tol, form="mixed", nrhs=nrhs, out=out)  # warm-up; allocates the basis
            restart = m
            break
        except hps.HPSError as e:
            if solver is not None:
                solver.close()
                solver = None
            torch.cuda.empty_cache()
            if m == 30:
                return {"error": str(e)}
    try:
        stream = torch.cuda.current_stream()
        solver.profile(enable=True, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _, info = solver.solve(s=s, tol=w.tol, form="mixed", nrhs=nrhs, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile(enable=False, reset=True)
        ncl, k_blocks, b_blocks = solver.precond_info()
        shapes = solver.launch_shapes()
        mem = solver.memory_bytes
        nf = solver.nf
    finally:
        solver.close()
    pk, pk_src = peaks()
    tpk, tpk_src = tf32_peak()
    nb = 6 * q * q
    rows = interior_face_pairs(L) * q * q  # rows of R whose output is used
    nint = 24 * q * q
    roof = {}

    def entry(phase, by, flops=None, tensor=False):
        cnt = prof["count"][phase]
        if not cnt:
            return
        dur = prof["ms"][phase] / cnt / 1e3
        e = {"avg_launch_ms": round(dur * 1e3, 4), "launches": cnt, "algorithmic_bytes": by,
             "achieved_gbs": round(by / dur / 1e9, 1), "hbm_peak_gbs": pk, "hbm_frac": round(by / dur / 1e9 / pk, 4)}
        if flops:
            e["algorithmic_flops"] = flops
            e["achieved_tflops"] = round(flops / dur / 1e12, 1)
            if tensor:
                e["tf32_peak_tflops"] = round(tpk, 1)
                e["tensor_frac"] = round(flops / dur / 1e12 / tpk, 4)
            # the roofline is the larger of the two time bounds
            t_bound = max(by / (pk * 1e9), (flops / (tpk * 1e12)) if tensor else 0.0)
            e["bound"] = "tensor" if tensor and flops / (tpk * 1e12) > by / (pk * 1e9) else "hbm"
            e["frac_of_bound"] = round(t_bound / dur, 4)
        else:
            e["bound"] = "hbm"
        roof[phase] = e

    if nrhs >= 64:
        # three TF32 products of R (n_b x 2 n_b real) against 128 real columns per 64 RHS
        a_flops = 3 * 2.0 * rows * (2 * nb) * (2 * nrhs)
        a_bytes = rows * nb * 8 + nrhs * nf * (8 + 8 + 16)
        entry("apply", a_bytes, a_flops, tensor=True)
        # stage K: one TF32 product of every K_c (n_int x 2 n_int real) against 128 real columns per
        # 64 RHS for each member cluster
        k_flops = 2.0 * ncl * nint * (2 * nint) * (2 * nrhs)
        k_bytes = k_blocks * nint * nint * 8 + ncl * nint * 2 * 8 * nrhs
        entry("precond_k", k_bytes, k_flops, tensor=True)
    else:
        entry("apply", apply_bytes(L, q, 8, 8, 16))
        kb, bb = precond_bytes(L, q, 4, 8, in_bytes=16, scale_bytes=4, k_blocks=k_blocks, b_blocks=b_blocks)
        entry("precond_k", kb)
        entry("precond_b", bb)
    return {"workload": w.name, "leaves": L ** 3, "p": p, "q": q, "kappa": w.kappa, "tol": w.tol, "nrhs": nrhs,
            "restart": restart, "form": "lean mixed (FP32 maps + FP16 remainders, FP16/FP32 cluster blocks)",
            "setup_s": round(setup_s, 1), "device_bytes": mem, "precond_blocks": [ncl, k_blocks, b_blocks],
            "steps": steps, "ms_per_solve": ms, "unknowns_per_s": nrhs * nf / (ms / 1e3),
            "iterations": info["iterations"], "cycles": info["cycles"], "rel_residual": info["rel_residual"],
            "converged": info["converged"], "reorth_steps": info["reorth_steps"],
            "phase_ms_per_solve": {k: round(v / steps, 3) for k, v in prof["ms"].items()},
            "gpu_launches_per_solve": prof["launches"] // steps, "roofline": roof, "peak_sources": [pk_src, tpk_src],
            "launch_shapes": shapes}


def run_serving(args, dist):
    """A stated subset of the serving stream, unshrunk: the stream of 500 requests as generated
    (Poisson arrivals at 20/s, seed 7; per request L ~ U{8..24} leaves per axis, p in {8, 10, 12},
    kappa ~ U[20, 120], 3-8 bumps, 1-16 Gaussian sources), of which the first
    `--serving-requests` with p = 8 are served at their own sizes and arrival times (the p = 10
    and 12 requests need 10 s to 11 min of FP64 leaf elimination each, more than a benchmark run
    can hold).  Mixed form, tol 1e-6, 2x2x2 clusters binned at 0.01, admission by an HBM budget
    of 96 GiB, up to 4 requests in flight.  Latency = arrival to result on the host, including
    queueing and each request's setup (its own medium, so its own leaf maps)."""
    from paper_2112_02211_gb300.serving import HPSBackend, Request, Server, latency_stats, overlapping_pairs

    ws = W.serving_stream(n=500, rate=20.0, seed=7)
    picked = [(i, w) for i, w in enumerate(ws) if w.p == 8][:args.serving_requests]
    reqs = [Request(i, w, w.meta["arrival"]) for i, w in picked]
    srv = Server(HPSBackend(form="mixed", device=dist.local, lambda_bin=0.01), hbm_budget=96 << 30, max_active=4)
    res = srv.run(reqs)
    st = latency_stats(res)
    st.update({"requests": len(reqs), "stream_indices": [i for i, _ in picked],
               "grids": [f"{w.nx}^3 p={w.p} kappa={w.kappa:.1f} nrhs={w.nrhs}" for _, w in picked],
               "peak_active": srv.peak_active, "peak_budget_bytes": srv.peak_bytes,
               "overlapping_pairs": len(overlapping_pairs(res)),
               "errors": [r.error for r in res if r.error],
               "stream": "serving stream (500 requests, seed 7) as generated; its first p = 8 requests at their "
                         "own sizes and arrival times; latency includes queueing and per-request setup"})
    return st


# --------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# --------------------------------------------------------------------------------------------
def oracle_sample(L_sample, steps=1, warmup=0, min_seconds=0.0):
    """Oracle solve of the same workload on an L_sample^3 grid (same p, kappa, medium and
    source): RHS build + GMRES(50) to 1e-6 without preconditioner, setup excluded; at least
    `steps` solves and at least `min_seconds` of them.  Returns (unknowns/s, seconds per
    solve, cores, solves)."""
    import oracle as O

    w = W.scaled(W.bump_16cubed(), L_sample)
    g = O.Grid(L_sample, L_sample, L_sample, w.p)
    xi = O.interior_nodes(g)
    prob = O.build_problem(g, w.kappa, w.eta, w.sample_b(xi))
    s = w.sample_s(xi)[0]

    def one():
        rhs = O.rhs_face(g, prob.H, s, None)
        f, its, hist = O.gmres(lambda v: O.apply_face(g, prob.R, v), rhs, tol=w.tol, restart=50)
        return its

    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    n = 0
    while n < steps or time.perf_counter() - t0 < min_seconds:
        one()
        n += 1
    dt = (time.perf_counter() - t0) / n
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return g.nf / dt, dt, cores, n


def oracle_apply_rate(L_sample, reps=5):
    """The oracle's apply (I + Pi R) f on the sample grid (its own FP64 maps), in GB/s of the same
    algorithmic bytes the GPU apply is credited with (rows of R with a neighbour, f read twice,
    y written; complex double)."""
    import oracle as O

    w = W.scaled(W.bump_16cubed(), L_sample)
    g = O.Grid(L_sample, L_sample, L_sample, w.p)
    xi = O.interior_nodes(g)
    prob = O.build_problem(g, w.kappa, w.eta, w.sample_b(xi))
    f = np.random.default_rng(0).standard_normal(g.nf) + 0j
    O.apply_face(g, prob.R, f)
    t0 = time.perf_counter()
    for _ in range(reps):
        O.apply_face(g, prob.R, f)
    dt = (time.perf_counter() - t0) / reps
    return apply_bytes(L_sample, w.q, 16, 16, 16) / dt / 1e9, dt


def single_core_sample(L_sample):
    """The oracle sample in a child process with BLAS and OpenMP limited to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "v, dt, c, n = bench.oracle_sample(%d, steps=1, warmup=0); print(json.dumps([v, dt, n]))" % (ROOT, L_sample))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        v, dt, n = json.loads(r.stdout.strip().splitlines()[-1])
        return v, dt
    except Exception:
        return None, None


def cpu_baseline_record(L_sample):
    v, dt, cores, n = oracle_sample(L_sample, steps=3, warmup=1, min_seconds=10.0)
    v1, dt1 = single_core_sample(L_sample)
    gbs, adt = oracle_apply_rate(L_sample)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"bump workload scaled to {L_sample}^3 leaves (same p, kappa, medium, source): "
                      f"oracle RHS build + GMRES(50) to 1e-6, no preconditioner, setup excluded; "
                      f"{n} solves of {dt:.2f} s; numpy with its default BLAS threading",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": "the same sample, BLAS and OpenMP limited to one thread",
                            "seconds_per_solve": dt1},
            "apply": {"achieved_gbs": round(gbs, 2), "seconds_per_apply": adt, "cores": cores,
                      "sample": f"oracle (I + Pi R) f on the {L_sample}^3 sample's FP64 maps, algorithmic "
                                f"bytes as for the GPU apply (complex double)"}}


def run_reference(args, dist):
    if dist.rank != 0:
        return None
    v, dt, cores, n = oracle_sample(args.cpu_sample_L, steps=args.steps, warmup=args.warmup)
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"bump workload scaled to {args.cpu_sample_L}^3 leaves (same p, kappa, medium, source); "
                    f"oracle RHS build + GMRES(50) to 1e-6 per step, no preconditioner, setup excluded"}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": workload_name(W.bump_16cubed(L=args.L)),
                       "sample": f"each step one oracle solve of the workload scaled to {args.cpu_sample_L}^3 leaves",
                       "parallelism": "host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist(group=args.impl != "reference")
    try:
        if args.impl == "reference":
            rec = run_reference(args, dist)
        else:
            rec = run_gpu(args, dist)
            if rec is not None and dist.rank == 0 and dist.world == 1:
                rec["cpu_baseline"] = cpu_baseline_record(args.cpu_sample_L)
            elif rec is not None:
                rec["cpu_baseline"] = None
        if dist.rank == 0 and rec is not None:
            print(json.dumps(rec), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
