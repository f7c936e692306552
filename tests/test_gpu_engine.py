"""The life cycle through the C ABI on a real pool (Sec. IV): declare, try,
wait (with timeout), release (full and partial), launch; and whole traces
run co-scheduled, checked for memory safety, FIFO order and the same job
results alone and in the mix."""
import numpy as np
import pytest
import torch

from job_outputs import check_job_output
from oracle import invariants
from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]

MIB = 1 << 20


def _rt():
    from paper_1712_04495_b300 import abi, runtime
    return abi, runtime


def _digest_f32(a: np.ndarray) -> int:
    w = a.view(np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(tg.mix64((np.arange(len(w), dtype=np.uint64) << np.uint64(32)) | w),
                          dtype=np.uint64))


def test_life_cycle_fifo():
    abi, rt = _rt()
    s = rt.Scheduler(MIB, "fifo")
    t1 = s.declare(600 * 1024)
    rc, g1 = s.wait(t1, 1_000_000_000)
    assert rc == abi.SG_OK and g1.offset == 0 and g1.ptr == s.pool.data_ptr()
    t2 = s.declare(600 * 1024)
    assert s.wait(t2, 2_000_000)[0] == abi.SG_ERR_TIMEOUT       # withdrawn after 2 ms
    t3 = s.declare(300 * 1024)
    rc, g3 = s.wait(t3, 1_000_000_000)                          # fits next to t1
    assert rc == abi.SG_OK and g3.offset == 600 * 1024
    t4 = s.declare(500 * 1024)                                  # 124 KiB free: waits
    assert s.try_grant(t4)[0] == abi.SG_NOT_READY               # non-blocking check
    with pytest.raises(abi.SgError) as e:
        s.declare(2 * MIB)
    assert e.value.code == abi.SG_ERR_TOO_LARGE
    assert s.release(t1) == abi.SG_OK                           # post-free wakes t4
    assert s.release(t1) == abi.SG_ERR_INVALID                  # double release refused
    rc, g4 = s.wait(t4, 1_000_000_000)
    assert rc == abi.SG_OK and g4.offset == 0
    # partial post-free: t3 keeps its first 100 KiB
    assert s.release(t3, 200 * 1024) == abi.SG_OK
    torch.cuda.synchronize()
    t5 = s.declare(200 * 1024)
    rc, g5 = s.wait(t5, 1_000_000_000)
    assert rc == abi.SG_OK and g5.offset == 700 * 1024
    assert abi.sg_device_error(s.ctx) == 0
    s.shutdown()


def test_first_fit_serves_later_small_request():
    abi, rt = _rt()
    s = rt.Scheduler(MIB, "first_fit")
    t1 = s.declare(768 * 1024)
    assert s.wait(t1, 10 ** 9)[0] == abi.SG_OK
    t2 = s.declare(512 * 1024)                                   # does not fit
    t3 = s.declare(128 * 1024)                                   # fits: MMU serves it
    assert s.wait(t3, 10 ** 9)[0] == abi.SG_OK
    assert s.try_grant(t2)[0] == abi.SG_NOT_READY
    s.release(t1)
    assert s.wait(t2, 10 ** 9)[0] == abi.SG_OK
    s.shutdown()


def test_launch_runs_job_in_grant_and_releases():
    abi, rt = _rt()
    tr = tg.trace_single_kind_t0(7, 2, 1 << 16, 1 << 18, 64 * MIB, "two")
    s = rt.Scheduler(64 * MIB, "fifo")
    job = tr.jobs[0]
    t = s.declare(int(job["need"]))
    rc, g = s.wait(t, 10 ** 9)
    assert rc == abi.SG_OK
    assert s.launch(t, job) == abi.SG_OK
    torch.cuda.synchronize()
    assert s.try_grant(t)[0] == abi.SG_ERR_INVALID               # released by the job itself
    n = int(job["p0"])
    a = s.pool[g.offset:g.offset + 4 * n].view(torch.float32).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), K.triad(int(job["key"]), n).view(np.uint32))
    s.shutdown()


def _small_mixed(seed, n_jobs, budget):
    return tg.trace_mixed(seed, n_jobs, None, budget, "small_mixed",
                          triad_rng=(1 << 16, 1 << 20), spmv_rng=(2e3, 5e4),
                          gemm_set=(128, 256, 512))


def _check_real_log(jobs, rec, budget, policy, exclusive=False):
    assert np.all(rec["status"] == 3), rec["status"]
    out = np.zeros(len(jobs), dtype=[("status", "<i4"), ("grant_seq", "<i8"), ("grant_t", "<u8"),
                                     ("offset", "<u8"), ("done_t", "<u8")])
    for f in out.dtype.names:
        out[f] = rec[f]
    j2 = jobs.copy()
    j2["arrival_ns"] = rec["arrival_t"]
    invariants.check_log(j2, out, budget, policy, exclusive=exclusive, replay=False)


@pytest.mark.parametrize("overlap", [False, True], ids=["kinds_apart", "overlap"])
@pytest.mark.parametrize("policy", ["fifo", "first_fit"])
def test_trace_alone_equals_mix(policy, overlap):
    abi, rt = _rt()
    budget = 48 * MIB
    tr = _small_mixed(3, 40, budget)
    s = rt.Scheduler(budget, policy, run_flags=abi.SG_RUNF_OVERLAP if overlap else 0)
    d_jobs = rt.to_device(tr.jobs)
    d_tab = rt.device_tables(tr)
    rc, log, keep, st = s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED, keep=True)
    assert rc == abi.SG_OK, st
    rec = rt.records(log)
    _check_real_log(tr.jobs, rec, budget, policy)
    assert st["peak_used"] <= budget and st["jobs_done"] == len(tr)
    rc, log2, keep2, st2 = s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE,
                                       keep=True)
    assert rc == abi.SG_OK
    rec2 = rt.records(log2)
    _check_real_log(tr.jobs, rec2, budget, "fifo", exclusive=True)
    # exclusive: one job at a time, in arrival order
    order = np.argsort(rec2["grant_seq"])
    assert np.all(rec2["grant_t"][order][1:] >= rec2["done_t"][order][:-1])
    # each job's result is the same alone and in the mix
    assert torch.equal(keep, keep2)
    # every grant came back: one free extent spanning the pool, nobody waiting
    eng = abi.sg_state(s.ctx)
    assert eng["used"] == 0 and eng["waiting"] == 0 and eng["error_flags"] == 0
    assert eng["free_extents"] == 1 and eng["max_free_extent"] == eng["budget"] == budget
    assert eng["done"] == len(tr) and eng["grants"] == len(tr)
    for j in np.nonzero(tr.jobs["kind"] == tg.KIND_TRIAD)[0]:
        ref = K.triad(int(tr.jobs["key"][j]), int(tr.jobs["p0"][j]))
        assert int(keep[j].item()) & ((1 << 64) - 1) == _digest_f32(ref)
    s.shutdown()


def test_trace_host_io_and_c1():
    abi, rt = _rt()
    tr = tg.trace_c1()
    s = rt.Scheduler(tr.budget, "fifo")
    rc, rec, keep, st = s.run_trace_host(tr.jobs, rt.device_tables(tr), abi.SG_RUN_SATURATED, keep=True)
    assert rc == abi.SG_OK
    _check_real_log(tr.jobs, rec, tr.budget, "fifo")
    for j in range(len(tr)):
        ref = K.triad(int(tr.jobs["key"][j]), int(tr.jobs["p0"][j]))
        assert int(keep[j]) == _digest_f32(ref)
    s.shutdown()


def test_timed_arrivals():
    abi, rt = _rt()
    budget = 32 * MIB
    tr = tg.trace_mixed(5, 30, 2000.0, budget, "timed", triad_rng=(1 << 16, 1 << 19),
                        spmv_rng=(2e3, 2e4), gemm_set=(128, 256))
    s = rt.Scheduler(budget, "first_fit")
    rc, log, keep, st = s.run_trace(rt.to_device(tr.jobs), rt.device_tables(tr), abi.SG_RUN_TIMED)
    assert rc == abi.SG_OK
    rec = rt.records(log)
    _check_real_log(tr.jobs, rec, budget, "first_fit")
    span = int(tr.jobs["arrival_ns"][-1])
    assert st["makespan_ns"] >= span * 0.9
    s.shutdown()


def test_priority_fifo_serves_higher_priority_first():
    abi, rt = _rt()
    s = rt.Scheduler(MIB, "prio_fifo")
    t1 = s.declare(900 * 1024)
    assert s.wait(t1, 10 ** 9)[0] == abi.SG_OK
    t2 = s.declare(600 * 1024, priority=1)
    t3 = s.declare(600 * 1024, priority=0)      # smaller value = higher priority
    torch.cuda.synchronize()
    assert s.try_grant(t2)[0] == abi.SG_NOT_READY and s.try_grant(t3)[0] == abi.SG_NOT_READY
    s.release(t1)
    rc, g3 = s.wait(t3, 10 ** 9)
    assert rc == abi.SG_OK and g3.offset == 0
    assert s.try_grant(t2)[0] == abi.SG_NOT_READY
    s.release(t3)
    assert s.wait(t2, 10 ** 9)[0] == abi.SG_OK
    for bad in (-32769, 32768):                 # priorities are 16-bit
        with pytest.raises(abi.SgError):
            s.declare(1024, priority=bad)
    s.shutdown()


@pytest.mark.parametrize("policy", ["first_fit", "prio_first_fit"])
def test_tickets_are_recycled_and_queue_positions_compacted(policy):
    """A long-running context: far more requests than tickets (64) and queue
    positions (128) while one large request keeps waiting; the waiters keep
    their order across the compactions."""
    abi, rt = _rt()
    s = rt.Scheduler(MIB, policy, max_tickets=64)
    hold = s.declare(600 * 1024)
    assert s.wait(hold, 10 ** 9)[0] == abi.SG_OK
    big = s.declare(800 * 1024)                     # waits: 424 KiB free
    seen = set()
    for i in range(500):
        t = s.declare(100 * 1024)                   # first fit serves it past the waiter
        seen.add(t)
        assert s.wait(t, 10 ** 9)[0] == abi.SG_OK
        assert s.release(t) == abi.SG_OK
        torch.cuda.synchronize()
    assert len(seen) < 64                           # ticket numbers were reused
    assert s.try_grant(big)[0] == abi.SG_NOT_READY
    second = s.declare(800 * 1024)                  # waits behind `big`
    torch.cuda.synchronize()
    assert s.try_grant(second)[0] == abi.SG_NOT_READY
    s.release(hold)
    rc, g = s.wait(big, 10 ** 9)
    assert rc == abi.SG_OK and g.offset == 0
    assert s.try_grant(second)[0] == abi.SG_NOT_READY
    s.release(big)
    assert s.wait(second, 10 ** 9)[0] == abi.SG_OK
    s.release(second)
    torch.cuda.synchronize()
    s.shutdown()


def test_cancel_and_grant_notifications():
    """sg_cancel withdraws a waiting request (and reports a grant that came
    first); sg_poll_grants lists grants in grant order, once each."""
    abi, rt = _rt()
    s = rt.Scheduler(MIB, "fifo")
    cur = 0
    a = s.declare(700 * 1024)
    assert s.wait(a, 10 ** 9)[0] == abi.SG_OK
    b = s.declare(700 * 1024)                      # waits
    c = s.declare(100 * 1024)                      # waits behind b (strict FIFO)
    torch.cuda.synchronize()
    rc, cur, got = abi.sg_poll_grants(s.ctx, cur)
    assert rc == abi.SG_OK and got == [a]
    assert abi.sg_cancel(s.ctx, b)[0] == abi.SG_ERR_TIMEOUT   # withdrawn: c is now the head
    rc, g = s.wait(c, 10 ** 9)
    assert rc == abi.SG_OK
    assert abi.sg_cancel(s.ctx, c)[0] == abi.SG_OK             # already granted
    assert abi.sg_cancel(s.ctx, 999)[0] == abi.SG_ERR_INVALID  # never declared
    rc, cur, got = abi.sg_poll_grants(s.ctx, cur)
    assert rc == abi.SG_OK and got == [c]
    rc, cur, got = abi.sg_poll_grants(s.ctx, cur)
    assert got == []
    s.release(a)
    s.release(c)
    torch.cuda.synchronize()
    s.shutdown()


@pytest.mark.parametrize("overlap", [False, True], ids=["kinds_apart", "overlap"])
def test_serving_results_equal_alone_and_in_the_mix(overlap):
    # open-loop arrivals admitted while earlier requests run; every request's
    # output equals its output when it runs alone on the GPU
    abi, rt = _rt()
    budget = 48 * MIB
    tr = tg.trace_mixed(21, 60, 3000.0, budget, "serve_small", triad_rng=(1 << 16, 1 << 20),
                        spmv_rng=(2e3, 4e4), gemm_set=(128, 256, 512))
    s = rt.Scheduler(budget, "first_fit", run_flags=abi.SG_RUNF_OVERLAP if overlap else 0)
    d_jobs, d_tab = rt.to_device(tr.jobs), rt.device_tables(tr)
    rc, log, keep_mix, st = s.run_trace(d_jobs, d_tab, abi.SG_RUN_TIMED, keep=True)
    assert rc == abi.SG_OK
    rec = rt.records(log)
    _check_real_log(tr.jobs, rec, budget, "first_fit")
    rc, _, keep_alone, _ = s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE, keep=True)
    assert rc == abi.SG_OK
    assert torch.equal(keep_mix, keep_alone)
    # and each request's output, run alone through the same runner, is the
    # oracle's: the served result equals it through the digests
    for j in range(len(tr)):
        one = tr.jobs[[j]].copy()
        one["arrival_ns"] = 0
        rc, log1, keep1, _ = s.run_trace(rt.to_device(one), d_tab, abi.SG_RUN_SATURATED, keep=True)
        assert rc == abi.SG_OK
        torch.cuda.synchronize()
        assert int(keep1[0].item()) == int(keep_mix[j].item()), j
        check_job_output(s.pool, int(rt.records(log1)["offset"][0]), tr.jobs[j], tr.tables)
    s.shutdown()
