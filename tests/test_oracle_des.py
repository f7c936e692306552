"""Pins of the admission / notification oracle (discrete-event simulator).

Closed forms, the paper's concurrency arithmetic (Sec. VI use-cases),
brute-force enumeration on 3-5 job traces, and log invariants.
"""
import math
import os

import numpy as np
import pytest

from oracle import brute, des, invariants, metrics
from paper_1712_04495_b300 import tracegen as tg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MIB = 1 << 20


def _jobs(arr, need, dur, prio=None, timeout=None):
    n = len(arr)
    j = np.zeros(n, dtype=tg.JOB_DTYPE)
    j["arrival_ns"] = arr
    j["need"] = need
    j["duration_ns"] = dur
    j["prio"] = 0 if prio is None else prio
    j["timeout_ns"] = tg.NO_TIMEOUT if timeout is None else timeout
    return j


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
def test_all_fit_granted_at_arrival(policy):
    jobs = _jobs([0, 5, 5, 9, 30], [1000, 2560, 256, 4096, 100], [50, 3, 7, 1, 2])
    out, st = des.simulate(jobs, 1 << 20, policy)
    assert np.all(out["status"] == des.ST_DONE)
    assert np.array_equal(out["grant_t"], jobs["arrival_ns"])
    # offsets are granule-rounded prefix sums; job 1's hole [1024, 3584) is
    # free again at t=8 but too small for job 3, which goes above job 2
    assert list(out["offset"][:4]) == [0, 1024, 3584, 3840]
    # peak at t=9: jobs 0, 2 and 3 (job 1 ended at t=8)
    assert st["peak_used"] == 1024 + 256 + 4096


def test_exclusive_serial_closed_form():
    # budget below any two needs: grant_j = max(arrival_j, done_{j-1})
    arr = [0, 2, 3, 50, 51]
    dur = [10, 5, 40, 1, 1]
    jobs = _jobs(arr, [600, 700, 800, 900, 1000], dur)
    out, _ = des.simulate(jobs, 1280, "fifo")
    prev = 0
    for j in range(5):
        g = max(arr[j], prev)
        assert out["grant_t"][j] == g and out["offset"][j] == 0
        prev = g + dur[j]
    # the exclusive flag (each job declares the whole pool) gives the same
    out2, _ = des.simulate(_jobs(arr, [1, 2, 3, 4, 5], dur), 1 << 20, "first_fit", exclusive=True)
    assert np.array_equal(out2["grant_t"], out["grant_t"])


def _golden_instances():
    rows = []
    with open(os.path.join(GOLDEN, "concurrent_instances.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, pct, inst = line.split()
                rows.append((name, int(pct), int(inst)))
    return rows


@pytest.mark.parametrize("name,pct,instances", _golden_instances())
@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_paper_maximum_concurrent_instances(name, pct, instances, policy):
    # 12 instances (the paper runs up to 12, one per CPU core) of an
    # application using pct% of a 4,799 MiB GPU, all submitted at once.
    budget = 4799 * MIB
    need = math.ceil(budget * pct / 100)
    dur = 1000
    jobs = _jobs([0] * 12, [need] * 12, [dur] * 12)
    out, st = des.simulate(jobs, budget, policy)
    conc = max(int(np.sum((out["grant_t"] <= t) & (out["done_t"] > t)))
               for t in out["grant_t"])
    assert conc == instances
    # waves: instance i starts at floor(i / c) * duration
    assert [int(x) for x in out["grant_t"]] == [(i // instances) * dur for i in range(12)]


def test_equal_needs_first_fit_equals_fifo():
    for seed in range(20):
        jobs = tg.random_admission_trace(seed, 40, 1 << 16)
        jobs["need"] = 5000
        a, _ = des.simulate(jobs, 1 << 16, "fifo")
        b, _ = des.simulate(jobs, 1 << 16, "first_fit")
        assert np.array_equal(a, b)


def test_equal_priorities_reduce_to_plain_policies():
    for seed in range(20):
        jobs = tg.random_admission_trace(seed, 40, 1 << 16)
        for p, q in (("prio_fifo", "fifo"), ("prio_first_fit", "first_fit")):
            a, _ = des.simulate(jobs, 1 << 16, p)
            b, _ = des.simulate(jobs, 1 << 16, q)
            assert np.array_equal(a, b)


def test_too_large_rejected_and_others_unaffected():
    jobs = _jobs([0, 1, 2], [2048, 1 << 30, 512], [10, 10, 10])
    out, _ = des.simulate(jobs, 4096, "fifo")
    assert list(out["status"]) == [des.ST_DONE, des.ST_TOO_LARGE, des.ST_DONE]
    assert out["grant_t"][2] == 2


def test_timeout_removes_waiter_and_unblocks_fifo():
    # head 1 cannot fit until t=100, but times out at t=20; job 2 then fits
    jobs = _jobs([0, 1, 2], [3000, 3000, 1000], [100, 5, 5], timeout=[tg.NO_TIMEOUT, 19, tg.NO_TIMEOUT])
    out, _ = des.simulate(jobs, 4096, "fifo")
    assert out["status"][1] == des.ST_TIMEOUT and out["done_t"][1] == 20
    assert out["grant_t"][2] == 20
    # zero timeout = non-blocking request: refused at once if it does not fit
    jobs = _jobs([0, 1], [3000, 3000], [100, 5], timeout=[tg.NO_TIMEOUT, 0])
    out, _ = des.simulate(jobs, 4096, "first_fit")
    assert out["status"][1] == des.ST_TIMEOUT and out["done_t"][1] == 1


def test_fifo_blocks_first_fit_overtakes():
    # Sec. V: under FIFO a later small request waits behind a large head;
    # under MMU it is served as soon as it fits.
    jobs = _jobs([0, 1, 2], [3072, 2048, 512], [100, 10, 10])
    f, _ = des.simulate(jobs, 4096, "fifo")
    m, _ = des.simulate(jobs, 4096, "first_fit")
    assert f["grant_t"][2] == 100 and m["grant_t"][2] == 2
    assert f["grant_t"][1] == 100 and m["grant_t"][1] == 100


def test_fifo_bypass_literal_reading():
    jobs = _jobs([0, 1, 2], [3072, 2048, 512], [100, 10, 10])
    out, _ = des.simulate(jobs, 4096, "fifo", flags=des.FLAG_FIFO_BYPASS)
    assert out["grant_t"][2] == 2 and out["grant_t"][1] == 100


def test_fragmentation_wait():
    # 4 KiB pool; A[0,1K) B[1K,2K) C[2K,3K) D[3K,4K); B and D finish: 2 KiB free
    # in two holes, a 2 KiB request count-fits but cannot be placed until C ends.
    jobs = _jobs([0, 0, 0, 0, 1], [1024] * 4 + [2048], [50, 5, 30, 5, 1])
    out, st = des.simulate(jobs, 4096, "first_fit")
    assert out["grant_t"][4] == 30 and out["offset"][4] == 1024
    # exactly one pass ends blocked by fragmentation: the one after D ends
    # (after B's, 1 KiB free does not even fit the count)
    assert st["frag_waits"] == 1


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
def test_brute_force_agrees(policy):
    checked = 0
    for seed in range(160):
        n = 3 + seed % 3
        jobs = tg.random_admission_trace(seed, n, 4096, max_arrival=12, max_dur=12,
                                         prio_levels=2 if policy.startswith("prio") else 1)
        out, _ = des.simulate(jobs, 4096, policy)
        needg = invariants.need_g(jobs["need"])
        sols = brute.enumerate_schedules(jobs["arrival_ns"], needg, jobs["duration_ns"], 4096,
                                         policy, jobs["prio"])
        assert len(sols) == 1, f"seed {seed}: {len(sols)} schedules satisfy {policy}"
        got = [(int(o["grant_t"]), int(o["offset"]), int(o["done_t"]), int(o["grant_seq"]))
               for o in out]
        assert got == sols[0], f"seed {seed}"
        checked += 1
    assert checked == 160


@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_invariants_random(policy):
    for seed in range(30):
        jobs = tg.random_admission_trace(seed, 200, 1 << 16, max_arrival=2000, max_dur=300)
        out, st = des.simulate(jobs, 1 << 16, policy)
        peak = invariants.check_log(jobs, out, 1 << 16, policy)
        assert peak == st["peak_used"]


def test_invariant_checker_catches_planted_mistakes():
    jobs = tg.random_admission_trace(3, 60, 1 << 14, max_arrival=400, max_dur=100)
    out, _ = des.simulate(jobs, 1 << 14, "first_fit")
    invariants.check_log(jobs, out, 1 << 14, "first_fit")
    bad = out.copy()
    j = int(np.argmax(out["grant_t"] > out["grant_t"].min()))
    bad["offset"][j] += 256
    with pytest.raises(AssertionError):
        invariants.check_log(jobs, bad, 1 << 14, "first_fit")
    bad = out.copy()
    waited = np.nonzero(out["grant_t"] > jobs["arrival_ns"])[0]
    k = int(waited[0])
    bad["grant_t"][k] += 1
    bad["done_t"][k] += 1
    with pytest.raises(AssertionError):
        invariants.check_log(jobs, bad, 1 << 14, "first_fit")


def test_c1_trace_log():
    tr = tg.trace_c1()
    out, st = des.simulate(tr.jobs, tr.budget, "fifo")
    invariants.check_log(tr.jobs, out, tr.budget, "fifo")
    assert np.all(out["status"] == des.ST_DONE)


@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_mixed_trace_logs(policy):
    tr = tg.trace_mixed(0, 256, None, 16 << 30, spmv_rng=(1e5, 1e6))
    out, st = des.simulate(tr.jobs, tr.budget, policy)
    invariants.check_log(tr.jobs, out, tr.budget, policy)
    ser, _ = des.simulate(tr.jobs, tr.budget, "fifo", exclusive=True)
    invariants.check_log(tr.jobs, ser, tr.budget, "fifo", exclusive=True)
    ms = metrics.summarize(tr.jobs, out)
    mser = metrics.summarize(tr.jobs, ser)
    # serial makespan is the sum of declared durations (all arrive at t=0)
    assert mser["makespan_ns"] == int(tr.jobs["duration_ns"].sum())
    assert ms["makespan_ns"] < mser["makespan_ns"]


def test_nearest_rank_percentiles():
    assert metrics.nearest_rank([5, 1, 3, 2, 4], 0.5) == 3
    assert metrics.nearest_rank(list(range(1, 101)), 0.99) == 99
    assert metrics.nearest_rank(list(range(1, 101)), 1.0) == 100
    assert metrics.nearest_rank([7], 0.01) == 7
