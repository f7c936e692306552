"""Client processes on one GPU with the shared segment (distributed control,
Sec. III-A): the test process publishes a device pool through CUDA IPC; each
client process decides its own admission on the segment, maps the pool, runs
a triad job on its grant and releases it. A client killed while it holds a
grant (none of its work in flight) is reclaimed by the client that waits."""
import os

import numpy as np
import pytest

from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg
from shm_clients import ShmClient

pytestmark = pytest.mark.gpu
MS = 1_000_000
MIB = 1 << 20


def _digest(a: np.ndarray) -> int:
    w = a.view(np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(tg.mix64((np.arange(len(w), dtype=np.uint64) << np.uint64(32)) | w), dtype=np.uint64))


@pytest.fixture
def segment():
    import torch
    from paper_1712_04495_b300 import abi
    name = f"/sg_gpu_shm_{os.getpid()}"
    abi.sg_shm_unlink(name)
    pool = torch.empty(256 * MIB, dtype=torch.uint8, device="cuda")
    h = abi.sg_shm_open(name, pool.numel(), "first_fit")
    abi.sg_shm_set_pool(h, pool.data_ptr(), pool.numel())
    yield abi, h, name
    abi.sg_shm_close(h)
    abi.sg_shm_unlink(name)
    del pool
    torch.cuda.synchronize()


@pytest.mark.timeout(300)
def test_two_client_processes_run_jobs_on_their_grants(segment):
    abi, h, name = segment
    n = 3 << 20                                    # 36 MiB per triad job
    clients = [ShmClient(name, gpu=True) for _ in range(2)]
    try:
        for c in clients:
            c.call("open", timeout=120)
        tickets = []
        for c in clients:
            rc, t = c.call("declare", 12 * n, 0)
            assert rc == abi.SG_OK
            tickets.append(t)
        offs = []
        for c, t in zip(clients, tickets):
            rc, off, _ = c.call("wait", t, 5000 * MS)
            assert rc == abi.SG_OK
            offs.append(off)
        assert abs(offs[0] - offs[1]) >= 12 * n          # disjoint grants
        for i, (c, t) in enumerate(zip(clients, tickets)):
            digest, off = c.call("triad", t, n, 100 + i, timeout=120)
            assert off == offs[i]
            assert digest == _digest(K.triad(100 + i, n))
            assert c.call("release", t, 0) == abi.SG_OK
        st = abi.sg_shm_stats(h)
        assert st["grants"] == 2 and st["used"] == 0
    finally:
        for c in clients:
            c.exit()


@pytest.mark.timeout(300)
def test_killed_client_memory_goes_to_the_waiting_client(segment):
    abi, h, name = segment
    n = 12 << 20                                   # 144 MiB: two do not fit in 256 MiB
    a, b = ShmClient(name, gpu=True), ShmClient(name, gpu=True)
    try:
        a.call("open", timeout=120)
        b.call("open", timeout=120)
        rc, ta = a.call("declare", 12 * n, 0)
        assert a.call("wait", ta, 5000 * MS)[0] == abi.SG_OK
        digest, _ = a.call("triad", ta, n, 7, timeout=120)   # synchronised: nothing in flight
        assert digest == _digest(K.triad(7, n))
        rc, tb = b.call("declare", 12 * n, 0)
        assert b.call("wait", tb, 0)[0] == abi.SG_ERR_TIMEOUT    # not granted: withdrawn
        rc, tb = b.call("declare", 12 * n, 0)
        a.kill()                                   # dies between steps, holding its grant
        rc, off, _ = b.call("wait", tb, 30000 * MS)             # b, blocked, reclaims it
        assert rc == abi.SG_OK
        digest, _ = b.call("triad", tb, n, 8, timeout=120)
        assert digest == _digest(K.triad(8, n))
        assert b.call("release", tb, 0) == abi.SG_OK
        st = abi.sg_shm_stats(h)
        assert st["reaped"] == 1 and st["used"] == 0
    finally:
        b.exit()
