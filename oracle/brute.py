"""Brute-force schedule enumeration for traces of 3-5 jobs (test infrastructure).

Independent of the event-driven simulator in ``des.c``: instead of stepping
a queue and a free list forward, it enumerates every assignment of a
*cause* to each job -- granted in the pass of its own arrival, or in the
pass of some other job's completion -- derives start times from the causes,
and keeps the assignments that a notification policy of Sec. V would have
produced. The pool's free space is recomputed from scratch from the running
set at every step. A policy is deterministic, so exactly one assignment must
survive; the tests compare it with the simulator bit for bit.

The validity rules, per event in time order (completions before arrivals at
equal times, then job id), with the queue ordered by arrival (or by
priority, then arrival, for the priority policies):

* FIFO / Priority FIFO: the jobs granted in this event's pass are the
  longest prefix of the queue that can be placed one after another;
* MMU (first fit): scanning the queue in order, a job is granted in this
  pass if and only if it can be placed at its turn;
* Priority MMU: first fit restricted to the highest priority class present,
  moving to the next class only when a class is emptied;

and every grant takes the lowest free address that holds it.
"""
from __future__ import annotations

import itertools

ST_DONE = 3


def _lowest_fit(running, size, budget):
    cand = 0
    for off, end in sorted(running):
        if off - cand >= size:
            return cand
        cand = max(cand, end)
    return cand if budget - cand >= size else None


def _starts(causes, a, d):
    n = len(a)
    s = [None] * n
    visiting = set()

    def get(j):
        if s[j] is not None:
            return s[j]
        if j in visiting:
            return None
        visiting.add(j)
        c = causes[j]
        if c == n:
            v = a[j]
        else:
            sk = get(c)
            v = None if sk is None else sk + d[c]
        visiting.discard(j)
        s[j] = v
        return v

    for j in range(n):
        if get(j) is None:
            return None
    return s


def enumerate_schedules(arrival, needg, duration, budget, policy, prio=None):
    """All cause assignments that satisfy the policy's rules.

    Returns a list of schedules, each a list of (grant_t, offset, done_t,
    grant_seq) per job. Every job must fit the pool on its own.
    """
    n = len(arrival)
    a = [int(x) for x in arrival]
    g = [int(x) for x in needg]
    d = [int(x) for x in duration]
    pr = [0] * n if prio is None else [int(x) for x in prio]
    prio_pol = policy in ("prio_fifo", "prio_first_fit")
    survivors = []
    for causes in itertools.product(range(n + 1), repeat=n):
        if any(causes[j] == j for j in range(n)):
            continue
        s = _starts(causes, a, d)
        if s is None:
            continue
        ok = True
        for j in range(n):
            c = causes[j]
            # granted in a completion's pass only if already waiting then
            if c != n and not (a[j] < s[j]):
                ok = False
                break
        if not ok:
            continue
        events = [(a[j], 1, j) for j in range(n)] + [(s[k] + d[k], 0, k) for k in range(n)]
        events.sort()
        running = {}      # job -> (off, end)
        waiting = []
        off = [None] * n
        seq = [None] * n
        nseq = 0
        for t, typ, j in events:
            if typ == 0:
                if j not in running:
                    ok = False
                    break
                del running[j]
            else:
                waiting.append(j)
            trig = (j if typ == 1 else None, j if typ == 0 else None)
            grants = {x for x in waiting if (causes[x] == n and trig[0] == x) or
                      (causes[x] != n and trig[1] == causes[x])}
            if prio_pol:
                order = sorted(waiting, key=lambda x: (pr[x], a[x], x))
            else:
                order = sorted(waiting, key=lambda x: (a[x], x))
            stopped = False
            cls = None
            for x in order:
                if prio_pol and policy == "prio_first_fit":
                    if cls is None:
                        cls = pr[x]
                    if pr[x] != cls:
                        # next class only if the previous one was emptied
                        if any(pr[y] == cls and y not in grants for y in order):
                            stopped = True
                        cls = pr[x]
                fit = None if stopped else _lowest_fit(running.values(), g[x], budget)
                if x in grants:
                    if fit is None or s[x] != t:
                        ok = False
                        break
                    running[x] = (fit, fit + g[x])
                    off[x] = fit
                    seq[x] = nseq
                    nseq += 1
                else:
                    if fit is not None:
                        ok = False       # the pass would have served it
                        break
                    if policy in ("fifo", "prio_fifo"):
                        stopped = True
            if not ok:
                break
            waiting = [x for x in waiting if x not in grants]
            if any(x in grants for x in order if s[x] != t):
                ok = False
                break
        if ok and not waiting and all(o is not None for o in off):
            survivors.append([(s[j], off[j], s[j] + d[j], seq[j]) for j in range(n)])
    return survivors
