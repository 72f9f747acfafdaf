"""bench.py's multi-rank host logic on CPU: two gloo ranks (the N-GPU
replica run's max-over-ranks timing and whole-job aggregation), no GPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = [1200.0, 1350.5][rank]
        mx = bench.max_over_ranks(local_ms, device="cpu")
        q.put((rank, mx, bench.whole_job_gflops(4.0e12 / 3, 5, ws, mx)))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, gf in res:
        assert mx == 1350.5  # every rank sees the slowest rank's time
        assert abs(gf - (4.0e12 / 3) * 5 * 2 / 1.3505 / 1e9) < 1e-6


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(12.5, device="cpu") == 12.5
    assert abs(bench.whole_job_gflops(2e9, 3, 1, 1000.0) - 6.0) < 1e-12
