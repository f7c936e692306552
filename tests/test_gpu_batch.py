"""Batching: a trace admitted as a whole by the device engine (replay plan)
and run as one CUDA graph and by the persistent grouped kernel. Each job's
output must equal the one-launch-per-job run (output digests), triads
bit-exact against the oracle; in a pool that holds every job at once, the
output arrays of each kind and size (the batch kernel's own tcgen05 GEMM
tiles and chunked SpMV included) are compared with the oracle."""
import numpy as np
import pytest
import torch

from job_outputs import check_job_output, pick_jobs
from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

MIB = 1 << 20


def _digest_f32(a: np.ndarray) -> int:
    w = a.view(np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(tg.mix64((np.arange(len(w), dtype=np.uint64) << np.uint64(32)) | w),
                          dtype=np.uint64))


def _u64(t):
    return t.cpu().numpy().astype(np.uint64)


def _check_three_ways(tr, budget, policy="first_fit", triad_check=64):
    from paper_1712_04495_b300 import abi, runtime
    pool = torch.empty(budget, dtype=torch.uint8, device="cuda")
    tab = runtime.device_tables(tr)
    pl = runtime.Planned(pool, tr.jobs, tab, policy, keep=True, budget=budget)
    assert pl.plan_stats["err"] == 0
    for _ in range(2):                      # launched twice: state is reset per launch
        assert pl.run_graph() == abi.SG_OK
        torch.cuda.synchronize()
        g_keep = _u64(pl.keep)
        assert pl.run_batch() == abi.SG_OK
        torch.cuda.synchronize()
        rc, done, err = pl.batch_status()
        assert (rc, err) == (abi.SG_OK, 0), (rc, done, err)
        assert done == len(tr)
        b_keep = _u64(pl.keep)
        assert np.array_equal(g_keep, b_keep)
    s = runtime.Scheduler(budget, policy, pool=pool)
    rc, log, keep, st = s.run_trace(runtime.to_device(tr.jobs), tab, abi.SG_RUN_SATURATED, keep=True)
    assert rc == abi.SG_OK
    assert np.array_equal(_u64(keep), b_keep)
    s.shutdown()
    tri = np.nonzero(tr.jobs["kind"] == tg.KIND_TRIAD)[0][:triad_check]
    for j in tri:
        ref = K.triad(int(tr.jobs["key"][j]), int(tr.jobs["p0"][j]))
        assert int(b_keep[j]) == _digest_f32(ref)
    info = abi.sg_batch_info(pl.batch)
    pl.close()
    return info


def test_small_mixed_batch():
    tr = tg.trace_mixed(9, 300, None, 64 * MIB, "batch_small", triad_rng=(4096, 1 << 18),
                        spmv_rng=(1000, 65536), gemm_set=(64, 128, 256, 512), lam=8.0)
    info = _check_three_ways(tr, 64 * MIB)
    assert info["jobs"] == 300


def test_tiny_jobs_10k():
    tr = tg.trace_c4()
    info = _check_three_ways(tr, tr.budget, triad_check=16)
    assert info["jobs"] == len(tr)


def test_batch_with_ragged_gemms_and_fifo():
    jobs = tg.make_jobs([tg.KIND_GEMM] * 6 + [tg.KIND_TRIAD] * 2, [64, 72, 200, 136, 8, 520, 4160, 70000],
                        np.zeros(8, np.int64), 3, (8.0,))
    tr = tg.Trace("ragged", jobs, 16 * MIB, np.stack([tg.poisson_cdf_table(8.0)]), (8.0,))
    _check_three_ways(tr, 16 * MIB, policy="fifo")


def _online(tr, budget, policy, keep=True):
    from paper_1712_04495_b300 import abi, runtime
    from oracle import invariants
    pool = torch.empty(budget, dtype=torch.uint8, device="cuda")
    tab = runtime.device_tables(tr)
    ob = runtime.OnlineBatch(pool, tr.jobs, tab, policy, keep=keep, budget=budget)
    keeps = []
    for _ in range(2):                      # launched twice: the engine is reset per launch
        assert ob.run() == abi.SG_OK
        torch.cuda.synchronize()
        rc, done, err = ob.status()
        assert (rc, err) == (abi.SG_OK, 0), (rc, done, err)
        assert done == len(tr)
        keeps.append(_u64(ob.keep))
    assert np.array_equal(keeps[0], keeps[1])
    rec = ob.records()
    # memory safety of a real run: no overcommit, extents held at the same
    # time are disjoint, every job granted once and finished
    assert np.all(rec["status"] == 3)
    assert sorted(rec["grant_seq"].tolist()) == list(range(len(tr)))
    need_g = (tr.jobs["need"].astype(np.int64) + 255) // 256 * 256
    ev = sorted([(int(rec["grant_t"][j]), 1, j) for j in range(len(tr))] +
                [(int(rec["done_t"][j]), 0, j) for j in range(len(tr))])
    used, held = 0, {}
    for t, kind, j in ev:
        if kind == 0:
            used -= need_g[j]
            held.pop(j)
        else:
            o = int(rec["offset"][j])
            for k, (o2, g2) in held.items():
                assert o + need_g[j] <= o2 or o2 + g2 <= o, (j, k)
            held[j] = (o, int(need_g[j]))
            used += need_g[j]
            assert used <= budget
    ob.close()
    return keeps[0], pool, tab


def test_online_batch_admits_on_the_device():
    """The batch's own engine admits the 10,000 tiny jobs inside the
    persistent kernel; each job's output equals the planned batch's."""
    from paper_1712_04495_b300 import abi, runtime
    tr = tg.trace_c4()
    keep_online, pool, tab = _online(tr, tr.budget, "first_fit")
    pl = runtime.Planned(pool, tr.jobs, tab, "first_fit", keep=True, budget=tr.budget, graph=False)
    assert pl.run_batch() == abi.SG_OK
    torch.cuda.synchronize()
    assert np.array_equal(_u64(pl.keep), keep_online)
    pl.close()
    tri = np.nonzero(tr.jobs["kind"] == tg.KIND_TRIAD)[0][:16]
    for j in tri:
        ref = K.triad(int(tr.jobs["key"][j]), int(tr.jobs["p0"][j]))
        assert int(keep_online[j]) == _digest_f32(ref)


@pytest.mark.parametrize("policy", ["fifo", "prio_first_fit"])
def test_online_batch_other_policies(policy):
    tr = tg.trace_mixed(9, 300, None, 64 * MIB, "batch_small", triad_rng=(4096, 1 << 18),
                        spmv_rng=(1000, 65536), gemm_set=(64, 128, 256, 512), lam=8.0)
    jobs = tr.jobs.copy()
    jobs["prio"] = jobs["kind"].astype(np.int64) % 2
    tr = tg.Trace(tr.name, jobs, tr.budget, tr.tables, tr.lambdas)
    _online(tr, 64 * MIB, policy)


def test_online_batch_rejects_a_job_that_never_fits():
    from paper_1712_04495_b300 import abi, runtime
    jobs = tg.make_jobs([tg.KIND_TRIAD] * 2, [1 << 20, 1 << 20], np.zeros(2, np.int64), 1, (8.0,))
    pool = torch.empty(4 * MIB, dtype=torch.uint8, device="cuda")
    tab = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(abi.SgError):
        abi.sg_batch_build_online(pool.data_ptr(), pool.numel(), jobs, tab.data_ptr(), "first_fit")


def test_batch_outputs_match_the_oracle():
    """The 10,000 tiny jobs in a pool that holds them all, so no job's memory
    is reused and every output stays in its grant: the persistent grouped
    kernel (planned and admitting online) and the CUDA graph each run the
    batch on a cleared pool, and the outputs of the smallest, largest and
    spread-out jobs of every kind (every GEMM size) are compared with the
    oracle array by array."""
    from paper_1712_04495_b300 import abi, runtime
    tr = tg.trace_c4()
    need_g = (tr.jobs["need"].astype(np.int64) + 255) // 256 * 256
    budget = int(need_g.sum()) + MIB
    pool = torch.zeros(budget, dtype=torch.uint8, device="cuda")
    tab = runtime.device_tables(tr)
    picks = pick_jobs(tr.jobs, per_kind=8)
    assert {int(k) for k in tr.jobs["kind"][picks]} == {tg.KIND_TRIAD, tg.KIND_SPMV, tg.KIND_GEMM}
    pl = runtime.Planned(pool, tr.jobs, tab, "first_fit", keep=False, budget=budget)
    assert pl.plan_stats["err"] == 0
    assert np.all(pl.plan["grant_t"] == 0)                 # everything granted at once
    offs = pl.plan["offset"].astype(np.int64)
    errs = {}
    for name, run in (("batch", pl.run_batch), ("graph", pl.run_graph)):
        pool.zero_()
        assert run() == abi.SG_OK
        torch.cuda.synchronize()
        if name == "batch":
            rc, done, err = pl.batch_status()
            assert (rc, err, done) == (abi.SG_OK, 0, len(tr))
        for j in picks:
            errs[(name, j)] = check_job_output(pool, int(offs[j]), tr.jobs[j], tr.tables)
    pl.close()
    ob = runtime.OnlineBatch(pool, tr.jobs, tab, "first_fit", keep=False, budget=budget)
    pool.zero_()
    assert ob.run() == abi.SG_OK
    torch.cuda.synchronize()
    rc, done, err = ob.status()
    assert (rc, err, done) == (abi.SG_OK, 0, len(tr))
    rec = ob.records()
    for j in picks:
        check_job_output(pool, int(rec["offset"][j]), tr.jobs[j], tr.tables)
    ob.close()
    gemm_err = max(v for (n, j), v in errs.items() if tr.jobs["kind"][j] == tg.KIND_GEMM)
    assert gemm_err < 1e-4                                   # FP32 accumulation of exact bf16 products
