"""The device engine's own source (engine.cuh) run on the CPU by 32 host
threads standing in for its warp (tests/engine_harness). No GPU is needed.

- Replay: the engine's replay loop on seeded traces gives the oracle's log
  (grant order, times, offsets, statuses) and counters, bit for bit, for
  the four policies.
- Live steps: random sequences of declare, full and partial release and
  withdrawal keep every invariant of the state (free extents ordered,
  coalesced and tiling the pool with the grants; used bytes; largest extent;
  queue membership; the queue's min-tree) and grant exactly what the
  shared-memory scheduler, driven by the same sequence, grants."""
import ctypes
import os
import sys
import tempfile

import numpy as np
import pytest

from oracle import des
from paper_1712_04495_b300 import abi
from paper_1712_04495_b300 import tracegen as tg

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "engine_harness"))
import build as harness_build  # noqa: E402

NO_TIMEOUT = abi.NO_TIMEOUT


@pytest.fixture(scope="module")
def eh():
    so = harness_build.build(tempfile.mkdtemp(prefix="sg_engine_host_"))
    L = ctypes.CDLL(so)
    P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    L.eh_create.restype = P
    L.eh_create.argtypes = [U32, U64, U64, U32, U32]
    L.eh_destroy.argtypes = [P]
    L.eh_declare.argtypes = [P, U32, U64, ctypes.c_int32]
    L.eh_release.argtypes = [P, U32, U64]
    L.eh_cancel.argtypes = [P, U32]
    L.eh_status.restype = U32
    L.eh_status.argtypes = [P, U32, P]
    L.eh_header.argtypes = [P, P]
    L.eh_check.restype = U32
    L.eh_check.argtypes = [P]
    L.eh_replay.restype = ctypes.c_int
    L.eh_replay.argtypes = [P, U32, U64, U64, U32, U32, U32, P, P]
    return L


def _jobs(rng, n, budget, prio_classes=1, timeouts=False):
    j = np.zeros(n, dtype=tg.JOB_DTYPE)
    gaps = rng.integers(0, 4, n) * rng.integers(0, 50, n)
    j["arrival_ns"] = np.cumsum(gaps)
    j["need"] = rng.integers(1, budget // 2, n)
    j["need"][rng.random(n) < 0.05] = budget + 1
    j["duration_ns"] = rng.integers(1, 200, n)
    j["prio"] = rng.integers(0, prio_classes, n)
    j["timeout_ns"] = NO_TIMEOUT
    if timeouts:
        sel = rng.random(n) < 0.3
        j["timeout_ns"][sel] = rng.integers(0, 150, sel.sum())
    return j


def _replay(L, jobs, budget, policy, flags=0, exclusive=False):
    n = len(jobs)
    jobs = np.ascontiguousarray(jobs)
    rec = np.zeros(n, dtype=abi.RECORD_DTYPE)
    st = np.zeros(4, dtype=np.uint64)
    pol = abi.POLICIES[policy]
    rc = L.eh_replay(jobs.ctypes.data, n, budget, 256, pol, flags, int(exclusive), rec.ctypes.data, st.ctypes.data)
    return rc, rec, st


def _compare(rec, ref):
    np.testing.assert_array_equal(rec["status"], ref["status"])
    for f in ("grant_seq", "grant_t", "offset"):
        m = ref["status"] == des.ST_DONE
        np.testing.assert_array_equal(rec[f][m], ref[f][m], err_msg=f)
    m = (ref["status"] == des.ST_DONE) | (ref["status"] == des.ST_TIMEOUT)
    np.testing.assert_array_equal(rec["done_t"][m], ref["done_t"][m])


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_replay_matches_oracle(eh, policy, seed):
    rng = np.random.default_rng(300 + seed)
    budget = 64 * 1024
    jobs = _jobs(rng, 200, budget, prio_classes=3 if policy.startswith("prio") else 1, timeouts=seed == 2)
    rc, rec, st = _replay(eh, jobs, budget, policy)
    ref, rst = des.simulate(jobs, budget, policy)
    assert rc == 0
    _compare(rec, ref)
    assert (int(st[0]), int(st[1]), int(st[2]), int(st[3])) == (rst["peak_used"], rst["frag_waits"],
                                                                 rst["passes"], 0)


def test_replay_bypass_and_exclusive(eh):
    rng = np.random.default_rng(9)
    budget = 1 << 16
    jobs = _jobs(rng, 150, budget)
    rc, rec, st = _replay(eh, jobs, budget, "fifo", flags=abi.SG_FLAG_FIFO_BYPASS)
    ref, rst = des.simulate(jobs, budget, "fifo", flags=des.FLAG_FIFO_BYPASS)
    assert rc == 0
    _compare(rec, ref)
    rc, rec, st = _replay(eh, jobs, budget, "first_fit", exclusive=True)
    ref, rst = des.simulate(jobs, budget, "first_fit", exclusive=True)
    assert rc == 0
    _compare(rec, ref)


def test_replay_deep_queue_many_extents(eh):
    # 1200 small jobs at once in a pool that holds about a hundred: a queue
    # a thousand deep and a long, fragmented free list
    rng = np.random.default_rng(11)
    n, budget = 1200, 2 << 20
    jobs = np.zeros(n, dtype=tg.JOB_DTYPE)
    jobs["need"] = rng.integers(256, 40000, n)
    jobs["duration_ns"] = rng.integers(1, 1000, n)
    jobs["timeout_ns"] = NO_TIMEOUT
    for policy in ("first_fit", "fifo"):
        rc, rec, st = _replay(eh, jobs, budget, policy)
        ref, rst = des.simulate(jobs, budget, policy)
        assert rc == 0
        _compare(rec, ref)
        assert int(st[1]) == rst["frag_waits"] and int(st[2]) == rst["passes"]


@pytest.mark.parametrize("seed, policy", [(1, "fifo"), (2, "first_fit"), (3, "prio_fifo"), (4, "prio_first_fit")])
def test_live_steps_keep_invariants_and_match_the_host_scheduler(eh, seed, policy):
    rng = np.random.default_rng(seed)
    cap, budget = 400, 1 << 20
    h = eh.eh_create(cap, budget, 256, abi.POLICIES[policy], 0)
    name = f"/sg_eh_{os.getpid()}_{policy}"
    abi.sg_shm_unlink(name)
    sh = abi.sg_shm_open(name, budget, policy, max_tickets=cap)
    rec = np.zeros(1, dtype=abi.RECORD_DTYPE)
    shm_of = {}
    held = {}          # ticket -> declared bytes still held
    waiting = set()
    try:
        for step in range(600):
            r = rng.random()
            if (r < 0.45 or not (held or waiting)) and len(shm_of) < cap:
                t = len(shm_of)
                need = int(rng.integers(1, budget // 3))
                prio = int(rng.integers(0, 3))
                eh.eh_declare(h, t, need, prio)
                rc, st_t = abi.sg_shm_declare(sh, need, prio)
                assert rc == abi.SG_OK
                shm_of[t] = st_t
                waiting.add(t)
                held[t] = need
            elif r < 0.85 and held:
                run = [t for t in held if t not in waiting]
                if not run:
                    continue
                t = int(rng.choice(run))
                part = int(rng.integers(1, held[t])) if rng.random() < 0.3 and held[t] > 1 else 0
                eh.eh_release(h, t, part)
                assert abi.sg_shm_release(sh, shm_of[t], part) == abi.SG_OK
                if part:
                    held[t] -= part
                else:
                    del held[t]
            elif waiting:
                t = int(rng.choice(sorted(waiting)))
                eh.eh_cancel(h, t)
                rc, _ = abi.sg_shm_wait(sh, shm_of[t], 0)
                assert rc == abi.SG_ERR_TIMEOUT
                waiting.discard(t)
                del held[t]
            bad = eh.eh_check(h)
            assert bad == 0, (step, bad)
            for t in list(waiting):
                st_dev = eh.eh_status(h, t, rec.ctypes.data)
                rc, g = abi.sg_shm_try(sh, shm_of[t])
                assert (st_dev == abi.SG_ST_RUNNING) == (rc == abi.SG_OK), (step, t)
                if rc == abi.SG_OK:
                    assert int(rec["offset"][0]) == g.offset, (step, t)
                    waiting.discard(t)
        hdr = np.zeros(9, dtype=np.uint64)
        eh.eh_header(h, hdr.ctypes.data)
        assert int(hdr[0]) == abi.sg_shm_stats(sh)["used"]
    finally:
        eh.eh_destroy(h)
        abi.sg_shm_close(sh)
        abi.sg_shm_unlink(name)
