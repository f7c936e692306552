"""CPU reference results of the three job kinds (test infrastructure only).

Each function regenerates a job's inputs from ``tracegen`` (the seeded
input generator) and computes the plain definition of the job:

* triad  a = b + s*c in FP32 with two roundings (product rounded, then sum),
         the STREAM definition with no fused multiply-add;
* SpMV   y = A x over CSR, products and sums in fp64 on the FP32 inputs;
* GEMM   C = A B^T, fp64 accumulation of the BF16-rounded inputs.

Sampled variants compute a chosen subset of outputs one by one, for job
sizes the host cannot hold whole.
"""
from __future__ import annotations

import numpy as np

from paper_1712_04495_b300 import tracegen as tg


# ------------------------------------------------------------------- triad
def triad_inputs(key: int, idx):
    b = tg.uniform_stream_f32(tg.stream_key(key, 1), idx)
    c = tg.uniform_stream_f32(tg.stream_key(key, 2), idx)
    return b, c


def triad(key: int, n: int, s: float = tg.TRIAD_SCALE) -> np.ndarray:
    """Whole output a[0:n]."""
    b, c = triad_inputs(key, np.arange(n, dtype=np.uint64))
    prod = np.multiply(np.float32(s), c, dtype=np.float32)     # first rounding
    return np.add(b, prod, dtype=np.float32)                   # second rounding


def triad_sampled(key: int, idx, s: float = tg.TRIAD_SCALE) -> np.ndarray:
    b, c = triad_inputs(key, np.asarray(idx, dtype=np.uint64))
    return np.add(b, np.multiply(np.float32(s), c, dtype=np.float32), dtype=np.float32)


# -------------------------------------------------------------------- SpMV
def spmv_row_ptr(key: int, rows: int, table) -> np.ndarray:
    lens = tg.row_lengths(tg.stream_key(key, 1), np.arange(rows, dtype=np.uint64), table)
    ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    return ptr


def spmv_csr(key: int, rows: int, table):
    """CSR arrays (row_ptr int64, col int64, val fp32) and x (fp32)."""
    ptr = spmv_row_ptr(key, rows, table)
    e = np.arange(ptr[-1], dtype=np.uint64)
    col = tg.spmv_columns(tg.stream_key(key, 2), e, rows)
    val = tg.spmv_values(tg.stream_key(key, 3), e)
    x = tg.uniform_stream_f32(tg.stream_key(key, 4), np.arange(rows, dtype=np.uint64))
    return ptr, col, val, x


def spmv(key: int, rows: int, table):
    """y (fp64) and the per-row magnitude sum_j |a_ij x_j| (for error bounds)."""
    ptr, col, val, x = spmv_csr(key, rows, table)
    prod = val.astype(np.float64) * x[col].astype(np.float64)
    row_of = np.repeat(np.arange(rows), np.diff(ptr))
    y = np.zeros(rows, dtype=np.float64)
    mag = np.zeros(rows, dtype=np.float64)
    np.add.at(y, row_of, prod)
    np.add.at(mag, row_of, np.abs(prod))
    return y, mag


def spmv_sampled(key: int, rows: int, table, sample_rows):
    """y and |.|-sums for chosen rows; row_ptr needs the prefix of row lengths."""
    sample_rows = np.asarray(sample_rows, dtype=np.int64)
    ptr = spmv_row_ptr(key, rows, table)
    kx = tg.stream_key(key, 4)
    kc = tg.stream_key(key, 2)
    kv = tg.stream_key(key, 3)
    y = np.zeros(len(sample_rows))
    mag = np.zeros(len(sample_rows))
    for t, r in enumerate(sample_rows):
        e = np.arange(ptr[r], ptr[r + 1], dtype=np.uint64)
        col = tg.spmv_columns(kc, e, rows)
        val = tg.spmv_values(kv, e).astype(np.float64)
        x = tg.uniform_stream_f32(kx, col.astype(np.uint64)).astype(np.float64)
        y[t] = float(np.sum(val * x))
        mag[t] = float(np.sum(np.abs(val * x)))
    return y, mag, ptr


def spmv_sampled_streamed(key: int, rows: int, table, sample_rows, chunk: int = 1 << 22):
    """spmv_sampled for matrices too large to hold row_ptr on the host: the
    row lengths are summed chunk by chunk, and only the chosen rows' start
    and end offsets are kept. Returns y, |.|-sums, starts, ends and nnz."""
    sample_rows = np.asarray(sample_rows, dtype=np.int64)
    starts = np.zeros(len(sample_rows), dtype=np.int64)
    ends = np.zeros(len(sample_rows), dtype=np.int64)
    kl = tg.stream_key(key, 1)
    base = 0
    for s in range(0, rows, chunk):
        e = min(rows, s + chunk)
        lens = tg.row_lengths(kl, np.arange(s, e, dtype=np.uint64), table)
        sel = (sample_rows >= s) & (sample_rows < e)
        if np.any(sel):
            cs = np.zeros(e - s + 1, dtype=np.int64)
            np.cumsum(lens, out=cs[1:])
            starts[sel] = base + cs[sample_rows[sel] - s]
            ends[sel] = base + cs[sample_rows[sel] - s + 1]
        base += int(lens.sum())
    kx = tg.stream_key(key, 4)
    kc = tg.stream_key(key, 2)
    kv = tg.stream_key(key, 3)
    y = np.zeros(len(sample_rows))
    mag = np.zeros(len(sample_rows))
    for t in range(len(sample_rows)):
        e = np.arange(starts[t], ends[t], dtype=np.uint64)
        col = tg.spmv_columns(kc, e, rows)
        val = tg.spmv_values(kv, e).astype(np.float64)
        x = tg.uniform_stream_f32(kx, col.astype(np.uint64)).astype(np.float64)
        y[t] = float(np.sum(val * x))
        mag[t] = float(np.sum(np.abs(val * x)))
    return y, mag, starts, ends, base


# -------------------------------------------------------------------- GEMM
def gemm_a(key: int, m: int, k: int, rows=None) -> np.ndarray:
    """A[i, :] as fp64 values of the bf16 inputs (rows defaults to all m)."""
    rows = np.arange(m) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = (rows[:, None].astype(np.uint64) * np.uint64(k) + np.arange(k, dtype=np.uint64)[None, :])
    u = tg.bf16_stream_f32(tg.stream_key(key, 1), idx)
    return tg.bf16_bits_to_f64(tg.bf16_bits_rne(u))


def gemm_bt(key: int, n: int, k: int, rows=None) -> np.ndarray:
    """B^T[j, :] (B stored N x K, K contiguous) as fp64 of the bf16 inputs."""
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = (rows[:, None].astype(np.uint64) * np.uint64(k) + np.arange(k, dtype=np.uint64)[None, :])
    u = tg.bf16_stream_f32(tg.stream_key(key, 2), idx)
    return tg.bf16_bits_to_f64(tg.bf16_bits_rne(u))


def gemm(key: int, m: int, n: int, k: int) -> np.ndarray:
    """C = A B^T in fp64 (M x N)."""
    return gemm_a(key, m, k) @ gemm_bt(key, n, k).T


def gemm_sampled(key: int, m: int, n: int, k: int, ii, jj) -> np.ndarray:
    """C[ii[t], jj[t]] one by one, each a length-K fp64 dot product."""
    ii = np.asarray(ii, dtype=np.int64)
    jj = np.asarray(jj, dtype=np.int64)
    out = np.empty(len(ii))
    ua = np.unique(ii)
    ub = np.unique(jj)
    a = dict(zip(ua.tolist(), gemm_a(key, m, k, ua)))
    b = dict(zip(ub.tolist(), gemm_bt(key, n, k, ub)))
    for t in range(len(ii)):
        out[t] = float(np.dot(a[int(ii[t])], b[int(jj[t])]))
    return out
