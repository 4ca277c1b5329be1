"""The request loop on the GPU: each request's result is the same when it runs
alone and when it runs admitted together with others (overlapping on the
device), and the loop reports latencies."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from paper_2112_02211_gb300.serving import HPSBackend, Request, Server, latency_stats, overlapping_pairs  # noqa: E402


def _stream():
    ws = W.serving_stream(n=5, rate=200.0, seed=11, L_range=(2, 4), p_choices=(6, 8), kappa_range=(6.0, 14.0),
                          max_sources=3)
    return [Request(i, w, w.meta["arrival"]) for i, w in enumerate(ws)]


@pytest.mark.parametrize("form", ["mixed", "fp64"])
def test_alone_equals_in_the_mix(form):
    be = HPSBackend(form=form)
    reqs = _stream()
    alone = Server(be, hbm_budget=64 << 30, max_active=1).run(reqs)
    mixed_srv = Server(be, hbm_budget=64 << 30, max_active=4)
    mixed = mixed_srv.run(reqs)
    assert mixed_srv.peak_active > 1, "requests were not admitted together"
    # their device work overlapped in time: CUDA-event intervals of two requests intersect
    assert overlapping_pairs(mixed), [r.info.get("device_interval_ms") for r in mixed]
    assert not overlapping_pairs(alone)
    for a, m in zip(alone, mixed):
        assert a.error is None and m.error is None, (a.error, m.error)
        assert a.info["converged"] and m.info["converged"]
        err = np.linalg.norm(a.f - m.f) / np.linalg.norm(a.f)
        assert err <= 1e-12, (a.rid, err)
    st = latency_stats(mixed)
    assert st["completed"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_budget_limits_concurrency():
    be = HPSBackend(form="mixed")
    reqs = _stream()
    need = max(be.bytes_needed(r.workload) for r in reqs)
    srv = Server(be, hbm_budget=need, max_active=4)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    assert srv.peak_bytes <= need
    # copies of the largest request: one fits at a time
    big = max(reqs, key=lambda r: be.bytes_needed(r.workload))
    same = [Request(i, big.workload, 0.001 * i) for i in range(3)]
    srv1 = Server(be, hbm_budget=need, max_active=4)
    res1 = srv1.run(same)
    assert all(r.error is None for r in res1)
    assert srv1.peak_active == 1 and srv1.peak_bytes == need
