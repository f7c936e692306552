"""Client processes on one GPU: a server process owns the pool and the
device engine; client processes map the pool through CUDA IPC, run triad
jobs on their grants and release them. A client that is killed while it
holds a grant (with none of its work in flight) is reaped, and its memory
goes to the client waiting for it."""
import os
import tempfile

import numpy as np
import pytest

from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg
from server_clients import Client, wait_until

pytestmark = pytest.mark.gpu
MS = 1_000_000
MIB = 1 << 20


def _digest(a: np.ndarray) -> int:
    w = a.view(np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(tg.mix64((np.arange(len(w), dtype=np.uint64) << np.uint64(32)) | w), dtype=np.uint64))


@pytest.fixture
def served():
    from paper_1712_04495_b300 import abi, runtime
    sched = runtime.Scheduler(256 * MIB, "first_fit")
    path = os.path.join(tempfile.mkdtemp(prefix="sg_gpu_srv_"), "sock")
    srv = abi.sg_server_start(sched.ctx, path)
    yield abi, sched, srv, path
    abi.sg_server_stop(srv)
    sched.shutdown()


@pytest.mark.timeout(300)
def test_two_client_processes_run_jobs_on_their_grants(served):
    abi, sched, srv, path = served
    n = 3 << 20                                    # 36 MiB per triad job
    clients = [Client(path, gpu=True) for _ in range(2)]
    try:
        for c in clients:
            assert c.call("connect", timeout=120)[0] == 256 * MIB
        tickets = [c.call("declare", 12 * n, 0, abi.NO_TIMEOUT) for c in clients]
        offs = []
        for c, t in zip(clients, tickets):
            rc, off = c.call("wait", t, 5000 * MS)
            assert rc == abi.SG_OK
            offs.append(off)
        assert abs(offs[0] - offs[1]) >= 12 * n          # disjoint grants
        for i, (c, t) in enumerate(zip(clients, tickets)):
            digest, off = c.call("triad", t, n, 100 + i, timeout=120)
            assert off == offs[i]
            assert digest == _digest(K.triad(100 + i, n))
            assert c.call("release", t, 0) == abi.SG_OK
        cnt = abi.sg_server_counters(srv)
        assert cnt["declares"] == 2 and cnt["grants"] == 2 and cnt["releases"] == 2
    finally:
        for c in clients:
            c.exit()


@pytest.mark.timeout(300)
def test_killed_client_memory_goes_to_the_waiting_client(served):
    abi, sched, srv, path = served
    n = 12 << 20                                   # 144 MiB: two do not fit in 256 MiB
    a, b = Client(path, gpu=True), Client(path, gpu=True)
    try:
        a.call("connect", timeout=120)
        b.call("connect", timeout=120)
        ta = a.call("declare", 12 * n, 0, abi.NO_TIMEOUT)
        assert a.call("wait", ta, 5000 * MS)[0] == abi.SG_OK
        digest, _ = a.call("triad", ta, n, 7, timeout=120)   # synchronised: nothing in flight
        assert digest == _digest(K.triad(7, n))
        tb = b.call("declare", 12 * n, 0, abi.NO_TIMEOUT)
        assert b.call("wait", tb, 200 * MS) == (abi.SG_NOT_READY, None)
        a.kill()                                   # dies between steps, holding its grant
        assert wait_until(lambda: abi.sg_server_counters(srv)["clients_reaped"] == 1, timeout=30)
        rc, off = b.call("wait", tb, 30_000 * MS)
        assert rc == abi.SG_OK
        digest, _ = b.call("triad", tb, n, 8, timeout=120)
        assert digest == _digest(K.triad(8, n))
        assert b.call("release", tb, 0) == abi.SG_OK
    finally:
        b.exit()
        if a.proc.is_alive():
            a.kill()
