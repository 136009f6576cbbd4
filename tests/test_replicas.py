"""Multi-GPU runs are independent replicas (the path needs no collective):
bench.py's whole-job throughput takes the slowest rank's time.  Checked here
with two gloo ranks on the host."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench

        local_ms = [120.0, 150.0][rank]  # rank 1 is the slower one
        value, t = bench.whole_job_rate(local_ms, 3.0e9, ws)
        out.put((rank, value, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 150.0
        assert value == pytest.approx(2 * 3.0e9 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    value, t = bench.whole_job_rate(200.0, 1.0e9, 1)
    assert t == 200.0 and value == pytest.approx(5.0e9)
