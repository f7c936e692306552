"""Batching: a trace admitted as a whole by the device engine (replay plan)
and run as one CUDA graph and by the persistent grouped kernel. Each job's
output must equal the one-launch-per-job run (output digests), triads
bit-exact against the oracle."""
import numpy as np
import pytest
import torch

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
