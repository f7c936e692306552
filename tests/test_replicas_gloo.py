"""Replicas across ranks (one scheduler, pool and trace per GPU, no data
exchange): the bench's whole-job throughput is the jobs of all ranks over
the slowest rank's time. Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, max_s = bench.aggregate(100 * (rank + 1), 1.0 + rank, world, bench._torch_ops("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, value, max_s))


def test_two_rank_aggregate():
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
    for _, value, max_s in res:
        assert max_s == 2.0                  # slowest rank
        assert value == (100 + 200) / 2.0    # all jobs over that time


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(256, 0.05, 1) == (256 / 0.05, 0.05)
