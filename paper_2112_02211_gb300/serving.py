"""Request loop for many HPS solves on one GPU (continuous admission).

Requests arrive over time, each with its own grid, wave number, medium and
right-hand sides.  A request is admitted as soon as an active slot is free and
the device bytes it needs (``hps_setup_bytes``: leaf maps, preconditioner,
Krylov workspace and the transient setup workspace) fit in what is left of the
HBM budget; admission is first-come first-served, so a large request at the
head of the queue is not overtaken.  Every admitted request runs on its own
host thread and CUDA stream: its setup and its solve go into the library while
other requests' kernels are on the device, and its Krylov state stays on the
device until its result is read back.  Latency is measured from arrival to
result (queueing + setup + solve).

The compute runs in the CUDA library; this module only schedules.  The
backend is pluggable so the scheduling logic can be exercised without a GPU.
"""

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Callable, List, Optional

import numpy as np

__all__ = ["Request", "Result", "Server", "HPSBackend", "latency_stats", "overlapping_pairs"]


@dataclass
class Request:
    rid: int
    workload: Any      # workloads.Workload
    arrival: float     # seconds after the start of the run


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    bytes: int = 0
    f: Optional[np.ndarray] = None
    info: dict = field(default_factory=dict)
    error: Optional[str] = None

    @property
    def latency(self):
        return self.done - self.arrival


class HPSBackend:
    """Runs one request through the CUDA library on the calling thread's own stream.  Per request
    it reports the setup and solve times (host clock) and the request's interval on the device
    timeline: CUDA events on its stream at the start and the end of its work, read against one
    epoch event of the backend, so that intervals of different requests can be compared."""

    def __init__(self, form="mixed", device=0, precond=True, lean=False, lambda_bin=0.0):
        self.form = form
        self.device = device
        self.precond = precond
        self.lean = lean
        self.lambda_bin = lambda_bin
        self._epoch = None
        self._lock = threading.Lock()

    def bytes_needed(self, w):
        import ctypes

        from . import _native as N
        lib = N.load()
        o = N.Options()
        lib.hps_default_options(ctypes.byref(o))
        o.forms = N.HPS_FORM_MIXED if self.form == "mixed" else N.HPS_FORM_FP64
        o.max_rhs = w.nrhs
        o.device = self.device
        o.lean = 1 if self.lean else 0
        o.lambda_bin = self.lambda_bin
        g = N.Grid(w.nx, w.ny, w.nz, w.p, w.p - 2)
        return int(lib.hps_setup_bytes(ctypes.byref(g), ctypes.byref(o), w.nrhs))

    def epoch(self):
        import torch
        with self._lock:
            if self._epoch is None:
                torch.cuda.set_device(self.device)
                self._epoch = torch.cuda.Event(enable_timing=True)
                self._epoch.record(torch.cuda.current_stream(self.device))
        return self._epoch

    def run(self, w):
        import torch

        from . import Solver, face_normals, nodes
        torch.cuda.set_device(self.device)
        epoch = self.epoch()
        stream = torch.cuda.Stream(device=self.device)
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        xi, xf = nodes(w.nx, w.ny, w.nz, w.p)
        with torch.cuda.stream(stream):
            e_start.record(stream)
            t0 = time.perf_counter()
            solver = Solver(w.nx, w.ny, w.nz, w.p, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi),
                            forms=(self.form,), max_rhs=w.nrhs, device=self.device, lean=self.lean,
                            lambda_bin=self.lambda_bin)
            t1 = time.perf_counter()
            try:
                s = w.sample_s(xi)
                t = None
                if w.t is not None:
                    nrm = np.broadcast_to(face_normals()[None, :, None, :], xf.shape)
                    t = w.sample_t(xf, nrm).reshape(-1)
                out = np.zeros(w.nrhs * solver.nf, dtype=np.complex128)
                _, info = solver.solve(s=None if s is None else s.reshape(-1), t=t, tol=w.tol, form=self.form,
                                       nrhs=w.nrhs, out=out, stream=stream, precond=self.precond)
            finally:
                solver.close()
            e_end.record(stream)
        e_end.synchronize()
        info = dict(info)
        info["setup_s"] = t1 - t0
        info["solve_s"] = time.perf_counter() - t1
        epoch.synchronize()
        info["device_interval_ms"] = (epoch.elapsed_time(e_start), epoch.elapsed_time(e_end))
        return out, info


def overlapping_pairs(results):
    """Pairs of requests whose device intervals intersect (their work was on the GPU at the
    same time)."""
    iv = [(r.rid, r.info.get("device_interval_ms")) for r in results if r.error is None and r.info]
    iv = [(rid, x) for rid, x in iv if x]
    out = []
    for i in range(len(iv)):
        for j in range(i + 1, len(iv)):
            (a, (a0, a1)), (b, (b0, b1)) = iv[i], iv[j]
            if max(a0, b0) < min(a1, b1):
                out.append((a, b))
    return out


class Server:
    """First-come first-served admission by free slots and HBM budget."""

    def __init__(self, backend, hbm_budget, max_active=4, clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.clock = clock
        self.peak_bytes = 0
        self.peak_active = 0

    def run(self, requests: List[Request]) -> List[Result]:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results = {r.rid: Result(rid=r.rid, arrival=r.arrival) for r in reqs}
        pending = collections.deque()
        cond = threading.Condition()
        state = {"used": 0, "active": 0, "finished": 0}
        t0 = self.clock()

        def now():
            return self.clock() - t0

        def worker(req, nbytes):
            res = results[req.rid]
            try:
                f, info = self.backend.run(req.workload)
                res.f, res.info = f, info
            except Exception as exc:  # the request fails, the loop goes on
                res.error = f"{type(exc).__name__}: {exc}"
            with cond:
                res.done = now()
                state["used"] -= nbytes
                state["active"] -= 1
                state["finished"] += 1
                cond.notify_all()

        idx = 0
        n = len(reqs)
        threads = []
        with cond:
            while state["finished"] < n:
                t = now()
                while idx < n and reqs[idx].arrival <= t:
                    pending.append(reqs[idx])
                    idx += 1
                while pending and state["active"] < self.max_active:
                    req = pending[0]
                    need = self.backend.bytes_needed(req.workload)
                    if need > self.hbm_budget:
                        pending.popleft()
                        res = results[req.rid]
                        res.admitted = res.done = now()
                        res.error = f"needs {need} bytes, more than the HBM budget {self.hbm_budget}"
                        state["finished"] += 1
                        continue
                    if state["used"] + need > self.hbm_budget:
                        break
                    pending.popleft()
                    state["used"] += need
                    state["active"] += 1
                    self.peak_bytes = max(self.peak_bytes, state["used"])
                    self.peak_active = max(self.peak_active, state["active"])
                    results[req.rid].admitted = now()
                    results[req.rid].bytes = need
                    th = threading.Thread(target=worker, args=(req, need), daemon=True)
                    threads.append(th)
                    th.start()
                if state["finished"] >= n:
                    break
                timeout = None
                if idx < n:
                    timeout = max(0.0, reqs[idx].arrival - now())
                cond.wait(timeout=timeout if timeout is not None else 1.0)
        for th in threads:
            th.join()
        return [results[r.rid] for r in sorted(reqs, key=lambda r: r.rid)]


def latency_stats(results: List[Result]):
    """p50/p99 latency (arrival to result), throughput, and the median queue, setup and solve
    time per request (setup and solve as the backend reports them)."""
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
    span = (max(r.done for r in ok) - min(r.arrival for r in ok)) if ok else 0.0
    unknowns = sum(r.f.size for r in ok if r.f is not None)

    def med(vals):
        vals = [v for v in vals if v is not None]
        return float(np.median(vals)) if vals else None

    return {
        "completed": len(ok),
        "failed": len(results) - len(ok),
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_s": float(lat.mean()) if lat.size else None,
        "solves_per_s": len(ok) / span if span > 0 else None,
        "unknowns_per_s": unknowns / span if span > 0 else None,
        "makespan_s": span,
        "queue_s_p50": med([r.admitted - r.arrival for r in ok]),
        "setup_s_p50": med([(r.info or {}).get("setup_s") for r in ok]),
        "solve_s_p50": med([(r.info or {}).get("solve_s") for r in ok]),
    }
