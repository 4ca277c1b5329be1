"""Scheduling logic of the request loop with a fake backend (no GPU): FIFO
admission by free slots and HBM budget, overlap of admitted requests, and the
latency statistics."""

import threading
import time

import numpy as np

from paper_2112_02211_gb300.serving import Request, Server, latency_stats


class FakeWorkload:
    def __init__(self, nbytes, seconds, size=10):
        self.nbytes = nbytes
        self.seconds = seconds
        self.size = size


class FakeBackend:
    def __init__(self):
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.used = 0
        self.max_used = 0
        self.order = []

    def bytes_needed(self, w):
        return w.nbytes

    def run(self, w):
        with self.lock:
            self.running += 1
            self.used += w.nbytes
            self.max_running = max(self.max_running, self.running)
            self.max_used = max(self.max_used, self.used)
            self.order.append(id(w))
        time.sleep(w.seconds)
        with self.lock:
            self.running -= 1
            self.used -= w.nbytes
        return np.zeros(w.size, dtype=np.complex128), {"iterations": 1}


def test_budget_and_slots_are_respected():
    be = FakeBackend()
    ws = [FakeWorkload(40, 0.05) for _ in range(6)]
    reqs = [Request(i, w, 0.0) for i, w in enumerate(ws)]
    srv = Server(be, hbm_budget=100, max_active=4)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    assert be.max_used <= 100 and srv.peak_bytes <= 100
    assert be.max_running == 2  # only two 40-byte requests fit in 100 bytes
    assert srv.peak_active == 2


def test_requests_overlap_and_are_admitted_in_arrival_order():
    be = FakeBackend()
    ws = [FakeWorkload(10, 0.1) for _ in range(4)]
    reqs = [Request(i, w, 0.01 * i) for i, w in enumerate(ws)]
    t0 = time.perf_counter()
    res = Server(be, hbm_budget=1000, max_active=4).run(reqs)
    wall = time.perf_counter() - t0
    assert be.max_running == 4
    assert wall < 0.35  # four 0.1 s requests overlapped, not run one after another
    assert be.order == [id(w) for w in ws]
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert all(r.admitted >= r.arrival for r in res)


def test_head_of_line_request_is_not_overtaken():
    be = FakeBackend()
    big = FakeWorkload(90, 0.05)
    small = [FakeWorkload(20, 0.05) for _ in range(3)]
    reqs = [Request(0, small[0], 0.0), Request(1, big, 0.001), Request(2, small[1], 0.002),
            Request(3, small[2], 0.003)]
    res = Server(be, hbm_budget=100, max_active=4).run(reqs)
    by = {r.rid: r for r in res}
    # the big request waits for request 0; requests 2 and 3 wait behind it
    assert by[1].admitted >= by[0].done - 1e-3
    assert by[2].admitted >= by[1].admitted and by[3].admitted >= by[1].admitted


def test_oversized_request_is_rejected_and_loop_continues():
    be = FakeBackend()
    reqs = [Request(0, FakeWorkload(500, 0.01), 0.0), Request(1, FakeWorkload(10, 0.01), 0.0)]
    res = Server(be, hbm_budget=100, max_active=2).run(reqs)
    assert res[0].error and "budget" in res[0].error
    assert res[1].error is None


def test_latency_stats():
    be = FakeBackend()
    reqs = [Request(i, FakeWorkload(1, 0.02 * (i + 1)), 0.0) for i in range(5)]
    res = Server(be, hbm_budget=100, max_active=5).run(reqs)
    st = latency_stats(res)
    assert st["completed"] == 5 and st["failed"] == 0
    assert 0.05 <= st["p50_s"] <= st["p99_s"] <= 0.2
    assert st["solves_per_s"] > 0
