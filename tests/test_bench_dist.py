"""Host logic of bench.py's multi-rank path (replicas: barrier + max/sum of
scalars, whole-job throughput), run as two gloo ranks on the CPU."""

import os
import socket
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
