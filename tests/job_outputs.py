"""Compare one job's output arrays, read from its grant in the pool, with the
CPU oracle (test helper, used by the GPU tests).

Tolerances are the ones every parity test states: the FP32 triad is
bit-exact; the CSR SpMV is within 1e-5 of sum_j |a_ij x_j| on every row (and
within 1e-5 relative 2-norm); the BF16 GEMM is within 2e-2 relative
Frobenius error of the fp64 product of the bf16-rounded inputs.
"""
import numpy as np
import torch

from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg


def _region(pool: torch.Tensor, off: int, nbytes: int, dtype) -> np.ndarray:
    return pool[off:off + nbytes].view(dtype).cpu().numpy()


def check_job_output(pool: torch.Tensor, off: int, job, tables: np.ndarray) -> float:
    """Assert that the output of `job` (a tracegen job record) found at byte
    offset `off` of `pool` matches the oracle; return its error measure
    (0 for the triad, the relative 2-norm / Frobenius error otherwise)."""
    kind, key = int(job["kind"]), int(job["key"])
    if kind == tg.KIND_TRIAD:
        n = int(job["p0"])
        a = _region(pool, off + tg.triad_layout(n)["a"], 4 * n, torch.float32)
        assert np.array_equal(a.view(np.uint32), K.triad(key, n).view(np.uint32)), ("triad", key, n)
        return 0.0
    if kind == tg.KIND_SPMV:
        rows, cap, tid = int(job["p0"]), int(job["p1"]), int(job["p2"])
        lay = tg.spmv_layout(rows, cap)
        y, mag = K.spmv(key, rows, tables[tid])
        gy = _region(pool, off + lay["y"], 4 * rows, torch.float32).astype(np.float64)
        assert np.all(np.abs(gy - y) <= 1e-5 * mag + 1e-30), ("spmv", key, rows)
        ny = np.linalg.norm(y)
        err = float(np.linalg.norm(gy - y) / ny) if ny > 0 else 0.0
        assert err <= 1e-5, ("spmv", key, rows, err)
        return err
    m, n, k = int(job["p0"]), int(job["p1"]), int(job["p2"])
    lay = tg.gemm_layout(m, n, k)
    c = _region(pool, off + lay["C"], 4 * m * n, torch.float32).astype(np.float64).reshape(m, n)
    ref = K.gemm(key, m, n, k)
    err = float(np.linalg.norm(c - ref) / np.linalg.norm(ref))
    assert err <= 2e-2, ("gemm", key, m, err)
    return err


def pick_jobs(jobs: np.ndarray, per_kind: int = 8) -> list:
    """Jobs to check: for each kind the smallest and the largest and, for the
    GEMM, each size present; then evenly spread ones, `per_kind` at most
    per kind (GEMM: per size)."""
    out = []
    for kind in (tg.KIND_TRIAD, tg.KIND_SPMV, tg.KIND_GEMM):
        idx = np.nonzero(jobs["kind"] == kind)[0]
        if len(idx) == 0:
            continue
        groups = ([idx[jobs["p0"][idx] == s] for s in np.unique(jobs["p0"][idx])]
                  if kind == tg.KIND_GEMM else [idx])
        for g in groups:
            order = g[np.argsort(jobs["p0"][g], kind="stable")]
            take = np.unique(np.linspace(0, len(order) - 1, min(per_kind, len(order))).round().astype(int))
            out.extend(int(order[t]) for t in take)
    return sorted(set(out))
