"""Schedule metrics (test infrastructure only): makespan, wait, turnaround.

Wait = grant - arrival; turnaround = completion - arrival; makespan = last
completion - first arrival. Percentiles are nearest-rank: the p-th
percentile of N values is the ceil(p*N)-th smallest (integer ns, no
interpolation).
"""
from __future__ import annotations

import math

import numpy as np

ST_DONE = 3


def nearest_rank(values, p: float) -> int:
    v = sorted(int(x) for x in values)
    if not v:
        return 0
    r = max(1, math.ceil(p * len(v)))
    return v[r - 1]


def summarize(jobs, out) -> dict:
    done = out["status"] == ST_DONE
    arr = jobs["arrival_ns"][done].astype(np.int64)
    g = out["grant_t"][done].astype(np.int64)
    d = out["done_t"][done].astype(np.int64)
    if len(arr) == 0:
        return {"jobs": 0}
    wait = g - arr
    turn = d - arr
    makespan = int(d.max() - arr.min())
    return {
        "jobs": int(done.sum()),
        "makespan_ns": makespan,
        "jobs_per_s": done.sum() / (makespan * 1e-9) if makespan > 0 else float("inf"),
        "wait_p50_ns": nearest_rank(wait, 0.50),
        "wait_p99_ns": nearest_rank(wait, 0.99),
        "turnaround_p50_ns": nearest_rank(turn, 0.50),
        "turnaround_p99_ns": nearest_rank(turn, 0.99),
    }
