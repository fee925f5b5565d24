"""Multi-rank bench aggregation on CPU (gloo, world size 2): replicas, the
job's time is the slowest rank's, the value counts every rank's unknowns."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    ms_local = 10.0 * (rank + 1)  # rank 1 is the slow one
    ms, value = bench.job_throughput(ms_local, units_per_rank=1000, steps=5, ws=ws, device="cpu")
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_throughput_takes_max_time_and_counts_all_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 20.0  # the slowest rank's time on every rank
        assert abs(value - 1000 * 5 * 2 / 0.020) < 1e-6


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_throughput(4.0, units_per_rank=100, steps=2, ws=1)
    assert ms == 4.0 and abs(value - 100 * 2 / 0.004) < 1e-9
