"""CPU, world_size 2 over gloo: the multi-GPU bench path is replicas only; its host
logic (max-over-ranks timing, whole-job throughput) is checked with gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1000.0 + 250.0 * rank          # rank 1 is the slow replica
    m = bench.max_over_ranks(ms, world, "cpu")
    v = bench.job_throughput(4, m, world)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 1250.0                   # both ranks see the slowest rank
        assert abs(v - 4 * 2 / 1.25) < 1e-12  # 8 iterations in 1.25 s
