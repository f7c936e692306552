"""Checks that every admission log must satisfy (test infrastructure only).

A log is, per job: status, grant sequence number, grant time, offset and
completion (release) time. The checks rebuild the pool's occupancy from the
log itself, independently of how the log was produced:

* no overcommit (Sec. III-B "total used" never exceeds "total memory"):
  at every instant the granule-rounded bytes of running jobs fit the pool;
* memory safety: extents of jobs that run at the same time are disjoint and
  inside the pool;
* a job starts no earlier than it arrives;
* FIFO order (Sec. V, Policy 1): grants follow arrival order;
* no lost waiter: with no timeouts, every request that fits the pool is
  eventually served;
* work conservation after every event time (Sec. V): under FIFO the oldest
  waiter cannot be placed; under first fit (MMU) no waiter can be placed;
* lowest-address placement: each offset is the lowest free address that
  holds the request, given the jobs running when it was granted.
"""
from __future__ import annotations

import bisect

import numpy as np

ST_DONE = 3
ST_TIMEOUT = 4
ST_TOO_LARGE = 5


def need_g(need, granule=256):
    need = np.asarray(need, dtype=np.uint64).astype(object)
    return [max(granule, (int(x) + granule - 1) // granule * granule) for x in need]


def check_no_overcommit(grant_t, done_t, needg, budget, mask):
    ev = []
    for j in np.nonzero(mask)[0]:
        if done_t[j] > grant_t[j]:
            ev.append((int(grant_t[j]), 1, int(needg[j])))
            ev.append((int(done_t[j]), 0, -int(needg[j])))
    ev.sort()
    used = 0
    peak = 0
    for _, _, dv in ev:
        used += dv
        assert used <= budget, f"overcommit: used {used} > budget {budget}"
        peak = max(peak, used)
    return peak


def check_disjoint(grant_t, done_t, offset, needg, budget, mask):
    idx = [int(j) for j in np.nonzero(mask)[0] if done_t[j] > grant_t[j]]
    for j in idx:
        assert offset[j] + needg[j] <= budget, f"job {j} extent leaves the pool"
    ev = []
    for j in idx:
        ev.append((int(grant_t[j]), 1, j))
        ev.append((int(done_t[j]), 0, j))
    ev.sort()
    active = []   # sorted (offset, end, j)
    for _, typ, j in ev:
        item = (int(offset[j]), int(offset[j]) + int(needg[j]), j)
        if typ == 0:
            active.remove(item)
            continue
        pos = bisect.bisect_left(active, item)
        if pos > 0:
            assert active[pos - 1][1] <= item[0], f"jobs {active[pos-1][2]} and {j} overlap"
        if pos < len(active):
            assert item[1] <= active[pos][0], f"jobs {j} and {active[pos][2]} overlap"
        active.insert(pos, item)


def check_fifo_order(arrival, grant_seq, grant_t, mask):
    idx = [int(j) for j in np.nonzero(mask)[0]]
    idx.sort(key=lambda j: (int(arrival[j]), j))
    seqs = [int(grant_seq[j]) for j in idx]
    times = [int(grant_t[j]) for j in idx]
    assert seqs == sorted(seqs), "FIFO: grants out of arrival order"
    assert times == sorted(times), "FIFO: grant times not monotone in arrival order"


def _lowest_fit(running, size, budget):
    """Lowest offset with [o, o+size) free, given running [(off, end)]."""
    cand = 0
    for off, end in sorted(running):
        if off - cand >= size:
            return cand
        cand = max(cand, end)
    return cand if budget - cand >= size else None


def check_placement(grant_seq, grant_t, done_t, offset, needg, budget, mask):
    """Each offset is the lowest fit given the jobs holding memory at its grant.

    Completions at the grant's own time t are processed one at a time (job id
    order), each followed by its notification pass, so a job granted at t may
    have been placed while some of them still held memory: the holders are
    the jobs running past t plus the ones completing at t whose completion
    comes after the grant. The checker accepts the smallest number p of
    completions at t already processed (a prefix in id order) that explains
    the offset, and requires p to never decrease along the grants at t.
    """
    idx = sorted((int(grant_seq[j]), int(j)) for j in np.nonzero(mask)[0])
    granted = []
    last_t, last_p = None, 0
    for _, j in idx:
        t = int(grant_t[j])
        if t != last_t:
            last_t, last_p = t, 0
        later = [(int(offset[k]), int(offset[k]) + int(needg[k])) for k in granted
                 if int(done_t[k]) > t]
        at_t = sorted(k for k in granted if int(done_t[k]) == t and int(grant_t[k]) < t)
        found = None
        for p in range(last_p, len(at_t) + 1):
            running = later + [(int(offset[k]), int(offset[k]) + int(needg[k])) for k in at_t[p:]]
            if _lowest_fit(running, int(needg[j]), budget) == int(offset[j]):
                found = p
                break
        assert found is not None, f"job {j}: offset {int(offset[j])} is not the lowest fit"
        last_p = found
        granted.append(j)


def check_work_conserving(arrival, grant_t, done_t, offset, needg, budget, status, policy):
    """After all events at each event time, the policy could serve no one else."""
    n = len(arrival)
    times = sorted(set(int(x) for x in arrival) | set(int(done_t[j]) for j in range(n)
                                                         if status[j] == ST_DONE))
    for t in times:
        running = [(int(offset[k]), int(offset[k]) + int(needg[k])) for k in range(n)
                   if status[k] == ST_DONE and int(grant_t[k]) <= t < int(done_t[k])]
        waiting = [j for j in range(n) if status[j] == ST_DONE and int(arrival[j]) <= t < int(grant_t[j])]
        if not waiting:
            continue
        waiting.sort(key=lambda j: (int(arrival[j]), j))
        if policy == "fifo":
            waiting = waiting[:1]
        for j in waiting:
            assert _lowest_fit(running, int(needg[j]), budget) is None, \
                f"t={t}: job {j} waits but could be placed ({policy})"


def check_log(jobs, out, budget, policy, granule=256, exclusive=False, replay=True):
    """Run every check that applies; returns the peak used bytes."""
    arrival = jobs["arrival_ns"]
    needg = need_g(jobs["need"], granule)
    if exclusive:
        needg = [budget // granule * granule] * len(jobs)
    budget = budget // granule * granule
    status = out["status"]
    done = status == ST_DONE
    gt, dt, off, seq = out["grant_t"], out["done_t"], out["offset"], out["grant_seq"]
    for j in np.nonzero(done)[0]:
        assert gt[j] >= arrival[j], f"job {j} granted before it arrived"
        if replay:
            assert dt[j] == gt[j] + jobs["duration_ns"][j], f"job {j}: done != grant + duration"
    for j in range(len(jobs)):
        if needg[j] > budget:
            assert status[j] == ST_TOO_LARGE, f"job {j} larger than the pool not rejected"
        elif int(jobs["timeout_ns"][j]) == (1 << 64) - 1:
            assert status[j] == ST_DONE, f"job {j} lost (status {status[j]})"
    peak = check_no_overcommit(gt, dt, needg, budget, done)
    check_disjoint(gt, dt, off, needg, budget, done)
    if replay:
        # needs exact event times; a real run's clock can tie distinct events
        check_placement(seq, gt, dt, off, needg, budget, done)
    if policy in ("fifo",):
        check_fifo_order(arrival, seq, gt, done)
    if policy in ("fifo", "first_fit") and np.all(status != ST_TIMEOUT) and replay:
        check_work_conserving(arrival, gt, dt, off, needg, budget, status, policy)
    return peak
