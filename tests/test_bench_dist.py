"""Host logic of bench.py's multi-rank path (replicas: barrier + max/sum of
scalars, whole-job throughput), run as two gloo ranks on the CPU, and the
reference arm's JSON line (the oracle on host cores), alone and under torchrun."""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(backend="gloo")
    d.barrier()
    mx = d.max(10.0 + rank)
    sm = d.sum(1.0 + rank)
    out[rank] = (d.rank, d.world, mx, sm)
    d.close()


def test_two_rank_reductions():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == (0, 2, 11.0, 3.0)
    assert out[1] == (1, 2, 11.0, 3.0)


def test_aggregate_uses_slowest_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate([100, 100], [1.0, 2.0]) == 100.0
    assert bench.aggregate([50], [0.5]) == 100.0


def test_algorithmic_bytes_formulas():
    sys.path.insert(0, ROOT)
    import bench
    # 1 leaf: no interior faces, only vector traffic
    assert bench.apply_bytes(1, 8, 8, 8, 16) == 6 * 64 * 32
    # 16^3, q = 8, c64 maps: rows of faces with a neighbour x 384 columns x 8 bytes
    rows = (6 * 16 ** 3 - 6 * 16 ** 2) * 64
    assert bench.apply_bytes(16, 8, 8, 8, 16) == rows * 384 * 8 + 16 ** 3 * 384 * 32
    kb, bb = bench.precond_bytes(16, 8, 8, 8)
    assert kb == 512 * 1536 * 1536 * 8 + 512 * 1536 * 16
    kb16, _ = bench.precond_bytes(16, 8, 4, 8, in_bytes=16, scale_bytes=4)
    assert kb16 == 512 * 1536 * (1536 * 4 + 4) + 512 * 1536 * 16


def _json_lines(out):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def test_reference_arm_line():
    """`bench.py --impl reference`: the oracle on host cores, one JSON line with the contract's
    keys; its cpu_baseline and e2e repeat the line's own value."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample-L", "2"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    (rec,) = _json_lines(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in rec, k
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["steps"] == 1 and rec["n_gpus"] == 1
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["cores"] >= 1 and rec["cpu_baseline"]["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert rec["config"]["workload"].startswith("bump_16cubed")


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks: rank 0 alone runs the oracle and prints; the other exits 0 without work."""
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                        "--cpu-sample-L", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    recs = _json_lines(r.stdout)
    assert len(recs) == 1 and recs[0]["impl"] == "reference" and recs[0]["n_gpus"] == 2
