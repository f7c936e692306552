"""The shared-memory scheduler (distributed control, Sec. III-A) on the CPU.

- Replay parity: a trace driven through the library's calls in event order
  (arrivals, completions, timeouts on a logical clock) grants the same jobs
  in the same order at the same times and offsets as the oracle's
  discrete-event simulator, for the four policies of Sec. V.
- Client processes: no two grants that are held at the same time overlap;
  a killed holder's memory and a killed waiter's request are reclaimed by the
  clients that are blocked (sanity check); a client that dies holding the
  file lock in the middle of an update does not block the others, and the
  state it left is checked and rebuilt (abandonment, integrity check);
  a damaged ticket table is restored from the backup that a closing client
  wrote, and a damaged backup leads to a fresh state.
No GPU is involved."""
import heapq
import multiprocessing as mp
import os
import threading

import numpy as np
import pytest

from oracle import des
from paper_1712_04495_b300 import abi
from paper_1712_04495_b300 import tracegen as tg
from shm_clients import (HDR_DIRTY, TK_BASE, TK_OFFSET, TK_SIZE, ShmClient, peek, poke, seg_path,
                         stress)

MS = 1_000_000
NO_TIMEOUT = abi.NO_TIMEOUT


@pytest.fixture
def name(request):
    n = f"/sg_test_{os.getpid()}_{request.node.name[:40]}".replace("[", "_").replace("]", "_")
    abi.sg_shm_unlink(n)
    yield n
    abi.sg_shm_unlink(n)


def _jobs(rng, n, budget, prio_classes=1, timeouts=False):
    j = np.zeros(n, dtype=tg.JOB_DTYPE)
    gaps = rng.integers(0, 4, n) * rng.integers(0, 50, n)           # many equal arrival times
    j["arrival_ns"] = np.cumsum(gaps)
    j["need"] = rng.integers(1, budget // 2, n)
    j["need"][rng.random(n) < 0.05] = budget + 1                       # a few too large
    j["duration_ns"] = rng.integers(1, 200, n)
    j["prio"] = rng.integers(0, prio_classes, n)
    j["timeout_ns"] = NO_TIMEOUT
    if timeouts:
        sel = rng.random(n) < 0.3
        j["timeout_ns"][sel] = rng.integers(0, 150, sel.sum())
    return j


def _drive(name, jobs, budget, policy, flags=0):
    """Feed the trace to the library in the simulator's event order: at equal
    times completions, then arrivals, then timeouts, each by job id; a job
    granted while an event is handled is granted at that event's time."""
    n = len(jobs)
    h = abi.sg_shm_open(name, budget, policy, max_tickets=n + 1, flags=flags)
    out = np.zeros(n, dtype=des.OUT_DTYPE)
    out["grant_seq"] = -1
    tk = [None] * n
    waiting = set()
    ev = [(int(jobs["arrival_ns"][j]), 1, j) for j in range(n)]
    heapq.heapify(ev)

    def collect(t):
        for j in sorted(waiting):
            rc, g = abi.sg_shm_try(h, tk[j])
            if rc == abi.SG_OK:
                rc, r = abi.sg_shm_record(h, tk[j])
                assert rc == abi.SG_OK
                waiting.discard(j)
                out[j]["status"] = des.ST_RUNNING
                out[j]["grant_seq"] = int(r["grant_seq"])
                out[j]["grant_t"] = t
                out[j]["offset"] = g.offset
                heapq.heappush(ev, (t + int(jobs["duration_ns"][j]), 0, j))
            else:
                assert rc == abi.SG_NOT_READY, rc

    try:
        while ev:
            t, kind, j = heapq.heappop(ev)
            if kind == 1:
                rc, tk[j] = abi.sg_shm_declare(h, int(jobs["need"][j]), int(jobs["prio"][j]))
                if rc == abi.SG_ERR_TOO_LARGE:
                    out[j]["status"] = des.ST_TOO_LARGE
                    continue
                assert rc == abi.SG_OK
                out[j]["status"] = des.ST_QUEUED
                waiting.add(j)
                tmo = int(jobs["timeout_ns"][j])
                if tmo != NO_TIMEOUT:
                    heapq.heappush(ev, (t + tmo, 2, j))
            elif kind == 0:
                assert abi.sg_shm_release(h, tk[j], 0) == abi.SG_OK
                out[j]["status"] = des.ST_DONE
                out[j]["done_t"] = t
            else:
                if j not in waiting:
                    continue
                rc, _ = abi.sg_shm_wait(h, tk[j], 0)
                assert rc == abi.SG_ERR_TIMEOUT, rc
                waiting.discard(j)
                out[j]["status"] = des.ST_TIMEOUT
                out[j]["done_t"] = t
            collect(t)
        st = abi.sg_shm_stats(h)
        assert abi.sg_shm_check(h) == 0
    finally:
        abi.sg_shm_close(h)
    return out, st


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_replay_matches_oracle(name, policy, seed):
    rng = np.random.default_rng(100 + seed)
    budget = 64 * 1024 + 100                       # not a granule multiple: rounded down
    jobs = _jobs(rng, 120, budget, prio_classes=3 if policy.startswith("prio") else 1, timeouts=seed == 2)
    ref, rst = des.simulate(jobs, budget, policy)
    got, st = _drive(name, jobs, budget, policy)
    for f in ("status", "grant_seq", "grant_t", "offset", "done_t"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    assert st["passes"] == rst["passes"]
    assert st["frag_waits"] == rst["frag_waits"]
    assert st["peak_used"] == rst["peak_used"]
    assert st["used"] == 0 and st["waiting"] == 0 and st["running"] == 0


def test_replay_fifo_bypass_matches_oracle(name):
    rng = np.random.default_rng(7)
    budget = 1 << 16
    jobs = _jobs(rng, 100, budget)
    ref, rst = des.simulate(jobs, budget, "fifo", flags=des.FLAG_FIFO_BYPASS)
    got, st = _drive(name, jobs, budget, "fifo", flags=abi.SG_FLAG_FIFO_BYPASS)
    for f in ("status", "grant_seq", "grant_t", "offset", "done_t"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    assert st["passes"] == rst["passes"]


def test_timeout_withdraws_and_unblocks_fifo(name):
    h = abi.sg_shm_open(name, 1 << 20, "fifo")
    try:
        _, big = abi.sg_shm_declare(h, 3 << 18)             # 3/4 of the pool, granted
        _, head = abi.sg_shm_declare(h, 1 << 19)            # waits
        _, small = abi.sg_shm_declare(h, 1 << 16)           # fits, but FIFO keeps it behind the head
        assert abi.sg_shm_try(h, big)[0] == abi.SG_OK
        assert abi.sg_shm_try(h, small)[0] == abi.SG_NOT_READY
        rc, _ = abi.sg_shm_wait(h, head, 5 * MS)
        assert rc == abi.SG_ERR_TIMEOUT
        assert abi.sg_shm_try(h, head)[0] == abi.SG_ERR_INVALID   # withdrawn, ticket ended
        rc, g = abi.sg_shm_try(h, small)
        assert rc == abi.SG_OK and g.offset == 3 << 18
        st = abi.sg_shm_stats(h)
        assert st["timeouts"] == 1 and st["used"] == (3 << 18) + (1 << 16)
    finally:
        abi.sg_shm_close(h)


def test_partial_release_and_errors(name):
    h = abi.sg_shm_open(name, 1 << 16, "first_fit", max_tickets=4)
    try:
        assert abi.sg_shm_declare(h, (1 << 16) + 1)[0] == abi.SG_ERR_TOO_LARGE
        assert abi.sg_shm_declare(h, 1, 1 << 20)[0] == abi.SG_ERR_INVALID     # priority beyond 16 bits
        _, a = abi.sg_shm_declare(h, 40000)                  # 40192 B granted at 0
        _, b = abi.sg_shm_declare(h, 30000)                  # waits: 25344 B free
        assert abi.sg_shm_try(h, b)[0] == abi.SG_NOT_READY
        assert abi.sg_shm_release(h, a, 20000) == abi.SG_OK  # keep 20000 -> 20224 B at the front
        st = abi.sg_shm_stats(h)
        assert st["used"] == 20224 + 30208
        rc, g = abi.sg_shm_try(h, b)
        assert rc == abi.SG_OK and g.offset == 20224
        assert abi.sg_shm_used_by(h, os.getpid()) == 20224 + 30208
        assert abi.sg_shm_release(h, a, 0) == abi.SG_OK
        assert abi.sg_shm_release(h, a, 0) == abi.SG_ERR_INVALID              # ended
        _, c = abi.sg_shm_declare(h, 1)
        _, d = abi.sg_shm_declare(h, 1)
        _, e = abi.sg_shm_declare(h, 1)
        assert abi.sg_shm_declare(h, 1)[0] == abi.SG_ERR_CAPACITY            # 4 tickets in use
        for t in (b, c, d, e):
            assert abi.sg_shm_release(h, t, 0) == abi.SG_OK
        assert abi.sg_shm_stats(h)["used"] == 0
        with pytest.raises(abi.SgError):
            abi.sg_shm_open(name, 1 << 20, "first_fit")       # same name, other budget
    finally:
        abi.sg_shm_close(h)
    with pytest.raises(abi.SgError):
        abi.sg_shm_open(name + "_missing")                   # attach needs an existing segment


def test_threads_share_a_handle(name):
    h = abi.sg_shm_open(name, 1 << 20, "first_fit")
    errors = []

    def run(seed):
        rnd = np.random.default_rng(seed)
        try:
            for _ in range(200):
                rc, t = abi.sg_shm_declare(h, int(rnd.integers(1, 1 << 19)))
                assert rc == abi.SG_OK
                rc, _ = abi.sg_shm_wait(h, t, 10 ** 10)
                assert rc == abi.SG_OK
                assert abi.sg_shm_release(h, t, 0) == abi.SG_OK
        except Exception as e:
            errors.append(e)

    th = [threading.Thread(target=run, args=(s,)) for s in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join(60)
    try:
        assert not errors, errors
        st = abi.sg_shm_stats(h)
        assert st["used"] == 0 and st["waiting"] == 0 and st["grants"] == 800
        assert abi.sg_shm_check(h) == 0
    finally:
        abi.sg_shm_close(h)


@pytest.mark.parametrize("policy", ["first_fit", "prio_first_fit"])
def test_processes_never_overlap(name, policy):
    budget = 1 << 20
    h = abi.sg_shm_open(name, budget, policy)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=stress, args=(name, s, 60, budget // 2, q)) for s in range(4)]
    for p in procs:
        p.start()
    logs = []
    try:
        for _ in procs:
            kind, res = q.get(timeout=120)
            assert kind == "done", res
            logs += res
    finally:
        for p in procs:
            p.join(30)
    try:
        assert len(logs) == 240
        logs.sort()
        for i, (g0, o0, n0, r0) in enumerate(logs):
            for g1, o1, n1, r1 in logs[i + 1:]:
                if g1 >= r0:
                    break                                    # later grants start after this release
                assert o0 + n0 <= o1 or o1 + n1 <= o0, "two held grants overlap"
        st = abi.sg_shm_stats(h)
        assert st["used"] == 0 and st["waiting"] == 0 and st["peak_used"] <= budget
        assert st["backups"] == 4                            # every client wrote one when it closed
        assert abi.sg_shm_check(h) == 0
    finally:
        abi.sg_shm_close(h)


def test_killed_holder_memory_reclaimed_by_blocked_waiter(name):
    h = abi.sg_shm_open(name, 1 << 20, "fifo")
    c = ShmClient(name)
    try:
        pid = c.call("open")
        rc, t = c.call("declare", 3 << 18, 0)
        assert rc == abi.SG_OK and c.call("try", t)[0] == abi.SG_OK
        assert abi.sg_shm_used_by(h, pid) == 3 << 18
        _, mine = abi.sg_shm_declare(h, 1 << 19)
        assert abi.sg_shm_try(h, mine)[0] == abi.SG_NOT_READY
        c.kill()
        rc, g = abi.sg_shm_wait(h, mine, 10 * 10 ** 9)       # blocked: checks the holders
        assert rc == abi.SG_OK and g.offset == 0
        st = abi.sg_shm_stats(h)
        assert st["reaped"] == 1 and st["used"] == 1 << 19
        assert abi.sg_shm_used_by(h, pid) == 0
    finally:
        abi.sg_shm_close(h)


def test_killed_waiter_request_withdrawn(name):
    h = abi.sg_shm_open(name, 1 << 20, "fifo")
    c = ShmClient(name)
    try:
        _, hold = abi.sg_shm_declare(h, 3 << 18)
        c.call("open")
        rc, dead = c.call("declare", 1 << 19, 0)           # the FIFO head, never served alive
        c.kill()
        _, mine = abi.sg_shm_declare(h, 1 << 18)            # behind the dead head
        assert abi.sg_shm_try(h, mine)[0] == abi.SG_NOT_READY
        rc, g = abi.sg_shm_wait(h, mine, 10 * 10 ** 9)      # the check withdraws the dead head
        assert rc == abi.SG_OK
        assert abi.sg_shm_stats(h)["reaped"] == 1
        abi.sg_shm_release(h, hold, 0)
        abi.sg_shm_release(h, mine, 0)
        assert abi.sg_shm_stats(h)["used"] == 0
    finally:
        abi.sg_shm_close(h)


def test_wake_up_across_processes(name):
    h = abi.sg_shm_open(name, 1 << 20, "first_fit")
    c = ShmClient(name)
    try:
        _, hold = abi.sg_shm_declare(h, 1 << 20)
        c.call("open")
        rc, t = c.call("declare", 1 << 19, 0)
        c.conn.send(("wait", t, 30 * 10 ** 9))              # blocks in the client
        import time
        time.sleep(0.2)
        assert abi.sg_shm_release(h, hold, 0) == abi.SG_OK
        assert c.conn.poll(10)
        status, (rc, off, waited_ns) = c.conn.recv()
        assert status == "ok" and rc == abi.SG_OK and off == 0
        assert waited_ns < 5 * 10 ** 9
        c.call("release", t, 0)
        c.call("close")
        c.exit()
    finally:
        abi.sg_shm_close(h)


def test_lock_holder_dies_mid_update_state_rebuilt(name):
    h = abi.sg_shm_open(name, 1 << 20, "first_fit")
    try:
        _, a = abi.sg_shm_declare(h, 1 << 18)
        _, b = abi.sg_shm_declare(h, 1 << 17)
        c = ShmClient(name)
        c.call("die_holding_lock", 12345)                   # used = 12345, dirty, lock held
        c.proc.join(10)
        assert peek(name, HDR_DIRTY, "<I") == 1
        st = abi.sg_shm_stats(h)                            # the next holder checks and rebuilds
        assert st["abandoned"] == 1 and st["rebuilt"] == 1
        assert st["used"] == (1 << 18) + (1 << 17)
        assert abi.sg_shm_check(h) == 0
        _, d = abi.sg_shm_declare(h, 1 << 18)
        assert abi.sg_shm_try(h, d)[1].offset == (1 << 18) + (1 << 17)
        for t in (a, b, d):
            assert abi.sg_shm_release(h, t, 0) == abi.SG_OK
    finally:
        abi.sg_shm_close(h)


def _slot(t):
    return t & 0xffff


def test_damaged_tickets_restored_from_backup(name):
    h = abi.sg_shm_open(name, 1 << 20, "first_fit")
    try:
        _, a = abi.sg_shm_declare(h, 1 << 18)
        _, b = abi.sg_shm_declare(h, 1 << 18)
        other = abi.sg_shm_open(name)
        abi.sg_shm_close(other)                              # a client ends: backup written
        assert os.path.exists(seg_path(name) + ".bak")
        # two held grants made to overlap: the ticket table itself is wrong
        poke(name, TK_BASE + _slot(b) * TK_SIZE + TK_OFFSET, "<Q", 0)
        found = abi.sg_shm_check(h)
        assert found & abi.SG_SHM_BAD_TICKETS
        st = abi.sg_shm_stats(h)
        assert st["restored"] == 1 and st["used"] == 1 << 19
        assert abi.sg_shm_try(h, a)[1].offset == 0
        assert abi.sg_shm_try(h, b)[1].offset == 1 << 18
        assert abi.sg_shm_check(h) == 0
    finally:
        abi.sg_shm_close(h)


def test_damaged_state_and_backup_start_afresh(name):
    h = abi.sg_shm_open(name, 1 << 20, "first_fit")
    try:
        _, a = abi.sg_shm_declare(h, 1 << 18)
        _, b = abi.sg_shm_declare(h, 1 << 18)
        other = abi.sg_shm_open(name)
        abi.sg_shm_close(other)
        with open(seg_path(name) + ".bak", "r+b") as f:     # the backup is damaged too
            f.seek(1000)
            byte = f.read(1)
            f.seek(1000)
            f.write(bytes([byte[0] ^ 0xff]))
        poke(name, TK_BASE + _slot(b) * TK_SIZE + TK_OFFSET, "<Q", 0)
        assert abi.sg_shm_check(h) & abi.SG_SHM_BAD_TICKETS
        st = abi.sg_shm_stats(h)
        assert st["reset"] == 1 and st["used"] == 0 and st["running"] == 0
        assert abi.sg_shm_try(h, a)[0] == abi.SG_ERR_INVALID
        _, c = abi.sg_shm_declare(h, 1 << 20)
        assert abi.sg_shm_try(h, c)[0] == abi.SG_OK
    finally:
        abi.sg_shm_close(h)


def test_new_client_repairs_damaged_header(name):
    h = abi.sg_shm_open(name, 1 << 20, "fifo")
    try:
        _, a = abi.sg_shm_declare(h, 1 << 18)
        poke(name, 0, "<Q", 0)                               # the magic number
        other = abi.sg_shm_open(name, 1 << 20, "fifo")      # a client that starts checks it
        abi.sg_shm_close(other)
        assert abi.sg_shm_check(h) == 0
        assert abi.sg_shm_try(h, a)[1].offset == 0
        assert abi.sg_shm_stats(h)["used"] == 1 << 18
    finally:
        abi.sg_shm_close(h)
