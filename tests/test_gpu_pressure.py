"""Memory pressure: 128 jobs declaring 2-60 GiB in a 170 GiB pool, arriving
in bursts of 16 (the needs of a burst exceed the pool), co-scheduled with
wake-on-release. Checks no overcommit, disjoint extents and no lost waiter
on the real log, that jobs did wait for memory, and that every job's output
is the same as when it runs alone. Exercises 64-bit sizes: triads of 5.4e9
elements, int64 row_ptr SpMV, GEMMs up to N = 86,144; sampled outputs of
one job of each kind at those sizes are compared with the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import invariants
from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(1500)]


@pytest.fixture(scope="module")
def c3_mix():
    from paper_1712_04495_b300 import abi, runtime
    tr = tg.trace_c3()
    free, total = torch.cuda.mem_get_info()
    if free < tr.budget + (8 << 30):
        pytest.skip("needs a 170 GiB pool")
    s = runtime.Scheduler(tr.budget, "first_fit")
    d_jobs, d_tab = runtime.to_device(tr.jobs), runtime.device_tables(tr)
    rc, log, keep_mix, st = s.run_trace(d_jobs, d_tab, abi.SG_RUN_TIMED, keep=True)
    yield {"tr": tr, "s": s, "d_jobs": d_jobs, "d_tab": d_tab, "rc": rc, "log": log, "keep": keep_mix,
           "st": st}
    s.shutdown()


def test_pressure_trace_co_scheduled_equals_alone(c3_mix):
    from paper_1712_04495_b300 import abi, runtime
    tr, s, st = c3_mix["tr"], c3_mix["s"], c3_mix["st"]
    assert c3_mix["rc"] == abi.SG_OK, st
    rec = runtime.records(c3_mix["log"])
    assert np.all(rec["status"] == abi.SG_ST_DONE)
    out = np.zeros(len(tr), dtype=[("status", "<i4"), ("grant_seq", "<i8"), ("grant_t", "<u8"),
                                   ("offset", "<u8"), ("done_t", "<u8")])
    for f in out.dtype.names:
        out[f] = rec[f]
    jobs = tr.jobs.copy()
    jobs["arrival_ns"] = rec["arrival_t"]
    peak = invariants.check_log(jobs, out, tr.budget, "first_fit", replay=False)
    assert peak <= tr.budget and st["peak_used"] <= tr.budget
    waited = int(np.sum(rec["grant_t"] > rec["arrival_t"] + 1_000_000))   # > 1 ms for memory
    assert waited >= 16
    assert abi.sg_kernel_errors() == 0
    rc, _, keep_alone, st2 = s.run_trace(c3_mix["d_jobs"], c3_mix["d_tab"],
                                         abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE, keep=True)
    assert rc == abi.SG_OK
    assert torch.equal(c3_mix["keep"], keep_alone)


def _largest(tr, kind, pred=lambda j: True):
    idx = [int(j) for j in np.nonzero(tr.jobs["kind"] == kind)[0] if pred(int(j))]
    return max(idx, key=lambda j: int(tr.jobs["p0"][j]))


def _run_alone(c3_mix, j):
    """Job j alone in the pool; returns its grant offset. Its output digest
    must equal the one it had in the co-scheduled run."""
    from paper_1712_04495_b300 import abi, runtime
    jobs = c3_mix["tr"].jobs[[j]].copy()
    jobs["arrival_ns"] = 0
    rc, log, keep, st = c3_mix["s"].run_trace(runtime.to_device(jobs), c3_mix["d_tab"],
                                              abi.SG_RUN_SATURATED, keep=True)
    assert rc == abi.SG_OK, st
    torch.cuda.synchronize()
    assert int(keep[0].item()) == int(c3_mix["keep"][j].item()), j
    return int(runtime.records(log)["offset"][0])


def _read(pool, off, nbytes, dtype, idx):
    t = pool[off:off + nbytes].view(dtype)
    return t[torch.from_numpy(np.asarray(idx, dtype=np.int64)).cuda()].cpu().numpy()


def test_pressure_outputs_at_64bit_sizes_match_the_oracle(c3_mix):
    """One job of each kind at the sizes only this trace reaches, run alone
    with the digest of its co-scheduled output, and sampled outputs against
    the oracle: a triad above 2^32 elements (bit-exact), an SpMV whose row
    pointers are int64 (per row, 1e-5 of sum |a x|) and the GEMM with
    N = 86,144 (relative Frobenius error of the sampled block within 2e-2)."""
    tr, pool = c3_mix["tr"], c3_mix["s"].pool
    rng = np.random.default_rng(3)
    # triad, n > 2^32
    j = _largest(tr, tg.KIND_TRIAD)
    n, key = int(tr.jobs["p0"][j]), int(tr.jobs["key"][j])
    assert n > 1 << 32
    off = _run_alone(c3_mix, j)
    idx = np.unique(np.concatenate([[0, 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, n - 1],
                                    rng.integers(0, n, 4096), rng.integers(1 << 32, n, 1024)]))
    got = _read(pool, off, 4 * n, torch.float32, idx)
    assert np.array_equal(got.view(np.uint32), K.triad_sampled(key, idx).view(np.uint32))
    # SpMV with int64 row pointers (nnz above 2^31): the smallest such job
    cands = [int(i) for i in np.nonzero((tr.jobs["kind"] == tg.KIND_SPMV) &
                                        (tr.jobs["p1"] >= (1 << 31)))[0]]
    j = min(cands, key=lambda i: int(tr.jobs["p0"][i]))
    rows, cap, key = int(tr.jobs["p0"][j]), int(tr.jobs["p1"][j]), int(tr.jobs["key"][j])
    lay = tg.spmv_layout(rows, cap)
    assert lay["ptr64"]
    off = _run_alone(c3_mix, j)
    sample = np.unique(np.concatenate([[0, 1, rows - 2, rows - 1], rng.integers(0, rows, 512),
                                       rng.integers(rows - rows // 16, rows, 512)]))
    y, mag, starts, ends, nnz = K.spmv_sampled_streamed(key, rows, tr.tables[int(tr.jobs["p2"][j])], sample)
    assert nnz > 1 << 31 and ends.max() > 1 << 31
    g_start = _read(pool, off + lay["row_ptr"], 8 * (rows + 1), torch.int64, sample)
    g_end = _read(pool, off + lay["row_ptr"], 8 * (rows + 1), torch.int64, sample + 1)
    assert np.array_equal(g_start, starts) and np.array_equal(g_end, ends)
    assert int(_read(pool, off + lay["row_ptr"], 8 * (rows + 1), torch.int64, [rows])[0]) == nnz
    gy = _read(pool, off + lay["y"], 4 * rows, torch.float32, sample).astype(np.float64)
    assert np.all(np.abs(gy - y) <= 1e-5 * mag + 1e-30)
    # GEMM, N >= 65,536
    j = _largest(tr, tg.KIND_GEMM)
    N, key = int(tr.jobs["p0"][j]), int(tr.jobs["key"][j])
    assert N >= 65536
    lay = tg.gemm_layout(N, N, N)
    off = _run_alone(c3_mix, j)
    ii = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 40)]))
    jj = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 40)]))
    I, J = np.meshgrid(ii, jj, indexing="ij")
    I, J = I.ravel(), J.ravel()
    ref = K.gemm_sampled(key, N, N, N, I, J)
    got = _read(pool, off + lay["C"], 4 * N * N, torch.float32, I * N + J).astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 2e-2, err
