"""The mixed 256-job trace the benchmark measures (all arrivals at t=0,
16 GiB pool, first fit), co-scheduled by the trace runner. The real log keeps
the invariants (no overcommit, disjoint extents inside the pool, no lost
waiter). Jobs of each kind, and of every GEMM size, then run again alone:
each one's output digest equals the one it had in the co-scheduled run, and
its output arrays meet the oracle -- whole arrays for the smaller jobs,
sampled entries for the large ones (a triad bit-exact; an SpMV row within
1e-5 of sum |a_ij x_j|; a GEMM within 2e-2 relative Frobenius error)."""
import numpy as np
import pytest
import torch

from job_outputs import check_job_output, pick_jobs
from oracle import invariants
from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(1200)]

SPMV_FULL_ROWS = 1_000_000     # larger SpMVs are checked on sampled rows
GEMM_FULL_SIZE = 1024          # larger GEMMs on a sampled block


def _read(pool, off, nbytes, dtype, idx):
    t = pool[off:off + nbytes].view(dtype)
    return t[torch.from_numpy(np.asarray(idx, dtype=np.int64)).cuda()].cpu().numpy()


def _check_sampled(pool, off, job, tables, rng):
    kind, key = int(job["kind"]), int(job["key"])
    if kind == tg.KIND_SPMV:
        rows, cap, tid = int(job["p0"]), int(job["p1"]), int(job["p2"])
        lay = tg.spmv_layout(rows, cap)
        sample = np.unique(np.concatenate([[0, rows - 1], rng.integers(0, rows, 1024)]))
        y, mag, ptr = K.spmv_sampled(key, rows, tables[tid], sample)
        esz, pdt = (8, torch.int64) if lay["ptr64"] else (4, torch.int32)
        g_ptr = _read(pool, off + lay["row_ptr"], esz * (rows + 1), pdt, np.arange(rows + 1)).astype(np.int64)
        assert np.array_equal(g_ptr, ptr)
        gy = _read(pool, off + lay["y"], 4 * rows, torch.float32, sample).astype(np.float64)
        assert np.all(np.abs(gy - y) <= 1e-5 * mag + 1e-30), ("spmv", key, rows)
        return
    m = int(job["p0"])
    lay = tg.gemm_layout(m, m, m)
    ii = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 30)]))
    jj = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 30)]))
    I, J = np.meshgrid(ii, jj, indexing="ij")
    I, J = I.ravel(), J.ravel()
    ref = K.gemm_sampled(key, m, m, m, I, J)
    got = _read(pool, off + lay["C"], 4 * m * m, torch.float32, I * m + J).astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 2e-2, ("gemm", key, m, err)


def test_mixed_trace_outputs_match_the_oracle():
    from paper_1712_04495_b300 import abi, runtime
    tr = tg.trace_c2(saturated=True)
    s = runtime.Scheduler(tr.budget, "first_fit")
    d_jobs, d_tab = runtime.to_device(tr.jobs), runtime.device_tables(tr)
    rc, log, keep_mix, st = s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED, keep=True)
    assert rc == abi.SG_OK, st
    assert st["jobs_done"] == len(tr) and st["peak_used"] <= tr.budget
    rec = runtime.records(log)
    out = np.zeros(len(tr), dtype=[("status", "<i4"), ("grant_seq", "<i8"), ("grant_t", "<u8"),
                                   ("offset", "<u8"), ("done_t", "<u8")])
    for f in out.dtype.names:
        out[f] = rec[f]
    jobs = tr.jobs.copy()
    jobs["arrival_ns"] = rec["arrival_t"]
    invariants.check_log(jobs, out, tr.budget, "first_fit", replay=False)
    assert abi.sg_kernel_errors() == 0
    rng = np.random.default_rng(11)
    picks = pick_jobs(tr.jobs, per_kind=3)
    kinds = {int(tr.jobs["kind"][j]) for j in picks}
    assert kinds == {tg.KIND_TRIAD, tg.KIND_SPMV, tg.KIND_GEMM}
    gemm_sizes = {int(tr.jobs["p0"][j]) for j in picks if int(tr.jobs["kind"][j]) == tg.KIND_GEMM}
    assert gemm_sizes == {256, 512, 1024, 2048, 4096, 8192}
    for j in picks:
        one = tr.jobs[[j]].copy()
        one["arrival_ns"] = 0
        rc, log1, keep1, _ = s.run_trace(runtime.to_device(one), d_tab, abi.SG_RUN_SATURATED, keep=True)
        assert rc == abi.SG_OK
        torch.cuda.synchronize()
        assert int(keep1[0].item()) == int(keep_mix[j].item()), j
        off = int(runtime.records(log1)["offset"][0])
        job = tr.jobs[j]
        kind = int(job["kind"])
        large = (kind == tg.KIND_SPMV and int(job["p0"]) > SPMV_FULL_ROWS) or \
                (kind == tg.KIND_GEMM and int(job["p0"]) > GEMM_FULL_SIZE)
        if large:
            _check_sampled(s.pool, off, job, tr.tables, rng)
        else:
            check_job_output(s.pool, off, job, tr.tables)
    s.shutdown()
