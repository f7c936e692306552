"""Replay parity: the device engine's admission log equals the oracle's bit
for bit (status, grant order, grant time, offset, completion) on the
logical clock with declared durations."""
import numpy as np
import pytest

from oracle import des, invariants
from paper_1712_04495_b300 import tracegen as tg

pytestmark = pytest.mark.gpu


def _parity(jobs, budget, policy, flags=0, exclusive=False):
    from paper_1712_04495_b300 import runtime
    rec, st = runtime.replay(jobs, budget, policy, flags=flags, exclusive=exclusive)
    out, ost = des.simulate(jobs, budget, policy, flags=flags, exclusive=exclusive)
    assert st["err"] == 0, f"device engine error flags {st['err']}"
    for f in ("status", "grant_seq", "grant_t", "offset", "done_t"):
        a = rec[f].astype(np.int64)
        b = out[f].astype(np.int64)
        bad = np.nonzero(a != b)[0]
        assert len(bad) == 0, f"{f} differs at jobs {bad[:8]}: gpu {a[bad[:8]]} oracle {b[bad[:8]]}"
    assert st["peak_used"] == ost["peak_used"]
    assert st["frag_waits"] == ost["frag_waits"]
    assert st["passes"] == ost["passes"]
    return rec, out


@pytest.mark.parametrize("policy", ["fifo", "first_fit", "prio_fifo", "prio_first_fit"])
def test_random_small_traces(policy):
    for seed in range(40):
        jobs = tg.random_admission_trace(seed, 3 + seed % 60, 1 << 16, max_arrival=300, max_dur=80,
                                         prio_levels=3 if policy.startswith("prio") else 1,
                                         timeout_frac=0.2 if seed % 3 == 0 else 0.0)
        _parity(jobs, 1 << 16, policy)


def test_fifo_bypass_and_exclusive():
    for seed in range(10):
        jobs = tg.random_admission_trace(seed, 50, 1 << 15, max_arrival=200, max_dur=50)
        _parity(jobs, 1 << 15, "fifo", flags=des.FLAG_FIFO_BYPASS)
        _parity(jobs, 1 << 15, "first_fit", exclusive=True)


def test_edge_cases():
    one = tg.random_admission_trace(1, 1, 4096)
    _parity(one, 4096, "fifo")
    big = tg.random_admission_trace(2, 20, 4096)
    big["need"][::3] = 1 << 40                   # larger than the pool: rejected at once
    rec, _ = _parity(big, 4096, "first_fit")
    assert np.all(rec["status"][::3] == des.ST_TOO_LARGE)
    zero = tg.random_admission_trace(3, 10, 4096)
    zero["need"] = 0                             # still takes a granule
    _parity(zero, 4096, "fifo")
    nonblock = tg.random_admission_trace(4, 40, 4096)
    nonblock["timeout_ns"] = 0                   # non-blocking requests
    _parity(nonblock, 4096, "first_fit")


@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_workload_traces(policy):
    for tr in (tg.trace_c1(), tg.trace_c2(saturated=True), tg.trace_c2(), tg.trace_c3(),
               tg.trace_c4()):
        rec, out = _parity(tr.jobs, tr.budget, policy)
        _parity(tr.jobs, tr.budget, "fifo", exclusive=True)
        if len(tr) <= 1000:
            invariants.check_log(tr.jobs, out, tr.budget, policy)


@pytest.mark.parametrize("policy", ["prio_fifo", "prio_first_fit"])
def test_priority_workload_traces(policy):
    """The priority policies on the workload traces: one kind prioritised
    (mixed trace), three classes by kind (10,000 tiny jobs, memory pressure)."""
    c2 = tg.trace_c2(saturated=True)
    jobs = c2.jobs.copy()
    jobs["prio"] = np.where(jobs["kind"] == tg.KIND_SPMV, 0, 1)
    _parity(jobs, c2.budget, policy)
    for tr in (tg.trace_c4(), tg.trace_c3()):
        jobs = tr.jobs.copy()
        jobs["prio"] = (jobs["kind"].astype(np.int64) * 7) % 3 - 1
        _parity(jobs, tr.budget, policy)


@pytest.mark.parametrize("policy", ["prio_fifo", "prio_first_fit"])
def test_priority_extremes(policy):
    """The whole int16 range of priorities, including both ends."""
    for seed in range(6):
        jobs = tg.random_admission_trace(seed, 120, 1 << 16, max_arrival=200, max_dur=60, prio_levels=3)
        jobs["prio"] = np.array([-32768, 0, 32767])[jobs["prio"]]
        _parity(jobs, 1 << 16, policy)


@pytest.mark.timeout(600)
def test_serving_trace_100k():
    tr = tg.trace_c5(rate_per_s=20000.0)
    _parity(tr.jobs, tr.budget, "first_fit")
