"""Pins of the oracle's op-sequence mode: the life-cycle calls of Sec. IV
(pre-allocation, post-free of all or part of a grant, the withdrawal of a
timed-out wait) issued one at a time.

Hand-worked cases fix the partial post-free (the ticket keeps the front of
its extent, granule-rounded), full release by 0 bytes or by at least what is
held, refusal of a second release, withdrawal that unblocks FIFO, and
fragmentation after a shrink. A property ties the op mode to the trace
mode: the declares and full releases of a trace, issued in the event order
of the trace simulator, give its log bit for bit (the trace mode is pinned
by brute force and closed forms in test_oracle_des.py).
"""
import numpy as np
import pytest

from oracle import des
from paper_1712_04495_b300 import tracegen as tg

KIB = 1 << 10
MIB = 1 << 20


def _st(o, k):
    return {f: int(o[f][k]) for f in ("used", "peak_used", "grants", "passes", "frag_waits",
                                       "max_free_extent", "free_extents", "waiting", "done")}


def test_partial_release_then_regrant_into_freed_tail():
    t, o = des.simulate_ops([("declare", 600 * KIB), ("declare", 500 * KIB),
                             ("release", 0, 200 * KIB),       # A keeps its first 400 KiB
                             ("release", 0, 400 * KIB),       # exactly what is held: all
                             ("release", 0),                  # A holds nothing: refused
                             ("release", 1, 0)], MIB, "fifo")
    assert list(o["rc"]) == [des.RC_OK] * 4 + [des.RC_INVALID, des.RC_OK]
    assert list(o["ticket"][:2]) == [0, 1]
    assert _st(o, 0)["used"] == 600 * KIB and _st(o, 0)["max_free_extent"] == 424 * KIB
    # B waits: 424 KiB are free
    assert _st(o, 1)["waiting"] == 1 and _st(o, 1)["grants"] == 1
    # the freed tail [400, 600) KiB joins [600, 1024) KiB and B is served there
    assert t["offset"][1] == 400 * KIB and t["grant_seq"][1] == 1 and t["grant_t"][1] == 2
    s2 = _st(o, 2)
    assert s2["used"] == 900 * KIB and s2["free_extents"] == 1 and s2["max_free_extent"] == 124 * KIB
    s3 = _st(o, 3)
    assert s3["used"] == 500 * KIB and s3["free_extents"] == 2 and s3["max_free_extent"] == 400 * KIB
    assert s3["done"] == 1 and t["status"][0] == des.ST_DONE and t["done_t"][0] == 3
    assert _st(o, 4) == s3                                              # refused: nothing ran
    s5 = _st(o, 5)
    assert s5["used"] == 0 and s5["free_extents"] == 1 and s5["max_free_extent"] == MIB
    assert s5["peak_used"] == 900 * KIB and s5["done"] == 2
    # passes: one per declare and one per accepted release
    assert s5["passes"] == 5


def test_partial_release_rounds_the_kept_part_up_to_the_granule():
    t, o = des.simulate_ops([("declare", 1000), ("release", 0, 100), ("release", 0, 200),
                             ("release", 0, 700), ("release", 0, 1)], 4096, "first_fit")
    assert list(o["rc"]) == [des.RC_OK] * 4 + [des.RC_INVALID]
    # 1000 B take 1024; keeping 900 B still takes 1024: nothing is freed, the pass still runs
    assert _st(o, 1)["used"] == 1024 and _st(o, 1)["passes"] == 2
    # keeping 700 B takes 768: [768, 1024) merges with [1024, 4096)
    s = _st(o, 2)
    assert s["used"] == 768 and s["free_extents"] == 1 and s["max_free_extent"] == 4096 - 768
    # 700 B are what is held now: the release frees everything
    assert _st(o, 3)["used"] == 0 and t["status"][0] == des.ST_DONE


def test_zero_bytes_frees_all_and_a_second_release_is_refused():
    t, o = des.simulate_ops([("declare", 5000), ("release", 0, 0), ("release", 0, 0),
                             ("release", 0, 100)], 1 << 16, "fifo")
    assert list(o["rc"]) == [des.RC_OK, des.RC_OK, des.RC_INVALID, des.RC_INVALID]
    assert t["status"][0] == des.ST_DONE and _st(o, 3)["used"] == 0


@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_withdrawing_the_blocked_head_serves_the_next(policy):
    t, o = des.simulate_ops([("declare", 700 * KIB), ("declare", 500 * KIB), ("declare", 100 * KIB),
                             ("cancel", 1), ("cancel", 2), ("cancel", 1), ("release", 1),
                             ("cancel", 0), ("release", 0), ("cancel", 0)], MIB, policy)
    if policy == "fifo":
        # strict FIFO: C waits behind B although 324 KiB are free
        assert _st(o, 2)["waiting"] == 2 and t["grant_t"][2] == 3
    else:
        # first fit serves C at once
        assert _st(o, 2)["waiting"] == 1 and t["grant_t"][2] == 2
    assert t["offset"][2] == 700 * KIB
    assert list(o["rc"][3:]) == [des.RC_TIMEOUT, des.RC_OK, des.RC_TIMEOUT, des.RC_INVALID,
                                 des.RC_OK, des.RC_OK, des.RC_INVALID]
    assert t["status"][1] == des.ST_TIMEOUT and t["grant_seq"][1] == -1
    # the withdrawal runs a pass; asking again, or about a granted ticket, does not
    assert _st(o, 3)["passes"] == 4 and _st(o, 4)["passes"] == 4 and _st(o, 5)["passes"] == 4
    assert _st(o, 9)["done"] == 2 and _st(o, 9)["used"] == 100 * KIB


def test_too_large_gets_no_ticket_and_runs_no_pass():
    t, o = des.simulate_ops([("declare", MIB + 1), ("declare", MIB), ("declare", 0)], MIB, "fifo")
    assert list(o["rc"]) == [des.RC_TOO_LARGE, des.RC_OK, des.RC_OK]
    assert list(o["ticket"]) == [-1, 0, 1]
    assert _st(o, 0)["passes"] == 0
    # the whole pool is served; a 0-byte request waits for one granule
    assert t["offset"][0] == 0 and t["status"][1] == des.ST_QUEUED and _st(o, 2)["waiting"] == 1


def test_fragmentation_after_a_shrink():
    calls = [("declare", 256 * KIB)] * 4 + [
        ("release", 1),                    # [256, 512) KiB free
        ("release", 3, 128 * KIB),         # D keeps [768, 896), frees [896, 1024)
        ("declare", 300 * KIB),            # 384 KiB free, no extent holds 300: waits
        ("release", 2)]                    # [256, 768) KiB: E fits there
    t, o = des.simulate_ops(calls, MIB, "first_fit")
    assert list(t["offset"][:4]) == [0, 256 * KIB, 512 * KIB, 768 * KIB]
    s = _st(o, 6)
    assert s["waiting"] == 1 and s["used"] == 640 * KIB and s["free_extents"] == 2
    assert s["frag_waits"] == 1 and s["max_free_extent"] == 256 * KIB
    assert t["offset"][4] == 256 * KIB and t["grant_t"][4] == 7 and _st(o, 7)["frag_waits"] == 1


def test_bypass_serves_an_arrival_that_fits_without_a_pass():
    calls = [("declare", 700 * KIB), ("declare", 500 * KIB), ("declare", 100 * KIB)]
    t, o = des.simulate_ops(calls, MIB, "fifo", flags=des.FLAG_FIFO_BYPASS)
    # the literal reading of Sec. IV: C is served on arrival, past the waiting B
    assert t["status"][2] == des.ST_RUNNING and t["grant_t"][2] == 2
    assert _st(o, 1)["passes"] == 1 and _st(o, 2)["passes"] == 1


def _ops_from_trace_events(jobs, out):
    """The trace's arrivals as declares and its completions as full releases,
    in the simulator's event order (time, completions before arrivals, id)."""
    ev = []
    for j in range(len(jobs)):
        ev.append((int(jobs["arrival_ns"][j]), 1, j))
        if out["status"][j] == des.ST_DONE:
            ev.append((int(out["done_t"][j]), 0, j))
    ev.sort()
    ops = np.zeros(len(ev), dtype=des.OP_DTYPE)
    for k, (t, typ, j) in enumerate(ev):
        ops["t"][k] = t
        if typ == 1:
            ops["type"][k] = des.OP_DECLARE
            ops["arg"][k] = jobs["need"][j]
            ops["prio"][k] = jobs["prio"][j]
            ops["ticket"][k] = -1
        else:
            ops["type"][k] = des.OP_RELEASE
            ops["ticket"][k] = j
    return ops


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
def test_op_mode_reproduces_trace_mode(policy):
    for seed in range(40):
        budget = 64 * 256
        jobs = tg.random_admission_trace(seed, 12, budget, prio_levels=3)
        out, st = des.simulate(jobs, budget, policy)
        t, o = des.simulate_ops(_ops_from_trace_events(jobs, out), budget, policy)
        assert len(t) == len(jobs)
        for f in ("status", "grant_seq", "grant_t", "offset", "done_t"):
            assert np.array_equal(t[f], out[f]), (seed, f)
        assert int(o["peak_used"][-1]) == st["peak_used"]
        assert int(o["passes"][-1]) == st["passes"]
        assert int(o["frag_waits"][-1]) == st["frag_waits"]


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
def test_random_call_sequences_keep_the_invariants(policy):
    """Capacity, disjoint extents inside the pool and the state counters,
    recomputed from the per-ticket results after every op of a seeded
    sequence of calls with partial releases and withdrawals."""
    budget = 1 << 20
    calls = tg.random_lifecycle_calls(5, 300, budget, prio_levels=3)
    for n in range(1, len(calls) + 1, 23):
        t, o = des.simulate_ops(calls[:n], budget, policy)
        held = {}
        for k, c in enumerate(calls[:n]):
            if c[0] == "declare":
                held[int(o["ticket"][k])] = c[1]
            elif c[0] == "release" and o["rc"][k] == des.RC_OK and t["status"][c[1]] == des.ST_RUNNING:
                held[c[1]] -= c[2]
        running = [j for j in range(len(t)) if t["status"][j] == des.ST_RUNNING]
        ext = sorted((int(t["offset"][j]), tg.r256(max(held[j], 1))) for j in running)
        for (a, la), (b, _) in zip(ext, ext[1:]):
            assert a + la <= b
        assert all(a + la <= budget for a, la in ext)
        assert int(o["used"][n - 1]) == sum(la for _, la in ext) <= budget
        assert int(o["grants"][n - 1]) == int(np.sum(t["grant_seq"] >= 0))
        assert int(o["waiting"][n - 1]) == int(np.sum(t["status"] == des.ST_QUEUED))
        free = budget - int(o["used"][n - 1])
        assert int(o["max_free_extent"][n - 1]) <= free
