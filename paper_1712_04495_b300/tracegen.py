"""Seeded synthetic inputs: job traces and the counter-based element generator.

This module is input generation only. It decides what jobs arrive, when,
what they declare and what data they hold. It admits nothing, schedules
nothing and computes no job result. Both the CUDA path (through the job
records it builds) and the CPU oracle read it; the CUDA kernels carry their
own implementation of the same element generator.

Element generator
-----------------
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output (0-based) of the stream seeded
with state ``k`` is ``mix64(k + (i + 1) * GAMMA)``, where ``mix64`` is the
published finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27,
multiply 0x94D049BB133111EB, xor-shift 31) and GAMMA = 0x9E3779B97F4A7C15.

A job of trace seed ``S`` and index ``j`` has data key ``K_j = out(S, j)``;
its data stream ``s`` has key ``K_{j,s} = out(K_j, s)``; element ``i`` of that
stream is drawn from ``h = out(K_{j,s}, i)``.

  row length      L = #{k : T[k] <= (h >> 32)}, T the Poisson CDF table below

Uniform streams give two elements per hash, h = out(K, m) for elements
e = 2m, 2m + 1:
  uniform[-1, 1)  u = b * 2^-23 - 1 (exact in fp32), b = h >> 40 for e even,
                  b = (h >> 8) & 0xFFFFFF for e odd (24 bits each)
bf16 streams (the GEMM operands) give four elements per hash, h = out(K, m)
for e = 4m + j, j = 0..3, 16 bits each (a bf16 keeps 8 significant bits):
  bf16 uniform    u = b * 2^-15 - 1 (exact in fp32), b = (h >> 16 j) & 0xFFFF,
                  then rounded to nearest, ties to even, to bf16

SpMV non-zeros come in pairs (e = 2m, 2m + 1), one hash per pair and per
quantity, h = out(K, m):
  column in [0,n) c = (w * n) >> 32 with w = h >> 32 for e even, h & 0xFFFFFFFF
                  for e odd (multiply-shift)
  value N(0,1)    u1 = ((h >> 40) + 1) * 2^-24, u2 = ((h >> 16) & 0xFFFFFF) * 2^-24,
                  r = sqrt(-2 ln u1); v = r cos(2 pi u2) for e even, r sin(2 pi u2)
                  for e odd (Box-Muller's two independent normals)

Streams: triad b=1, c=2 (element i); GEMM A=1 (element i*K+k), B^T=2
(element j*K+k); SpMV row lengths=1 (hash index row), columns=2 (hash
index e // 2), values=3 (hash index e // 2), x=4 (element col). The
uniform streams (b, c, x) are addressed by element, two per hash, and the
bf16 streams (A, B^T) by element, four per hash.

Job record (``JOB_DTYPE``, 64 bytes, the C struct ``sg_job``): arrival,
declared bytes, declared duration (replay clock), timeout, data key, kind
parameters and priority.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_U64 = np.uint64

KIND_TRIAD, KIND_SPMV, KIND_GEMM = 0, 1, 2
KIND_NAMES = {KIND_TRIAD: "triad", KIND_SPMV: "spmv", KIND_GEMM: "gemm"}
NO_TIMEOUT = (1 << 64) - 1
GRANULE = 256
TRIAD_SCALE = 3.0
SPMV_CHUNK_ROWS = 4096  # rows per chunk of the CSR build's scan workspace
POISSON_TABLE_LEN = 64

# Reference rates that turn a job's algorithmic cost into its declared
# replay duration (integer ns): B300 copy bandwidth and sustained bf16 rate.
REF_BYTES_PER_US = 6_492_100          # 6492.1 GB/s
REF_FLOP_PER_NS = 1_366_300           # 1366.3 TFLOP/s

JOB_DTYPE = np.dtype([
    ("arrival_ns", "<u8"),
    ("need", "<u8"),
    ("duration_ns", "<u8"),
    ("timeout_ns", "<u8"),
    ("key", "<u8"),
    ("p0", "<u8"),     # triad n | spmv rows | gemm M
    ("p1", "<u8"),     # spmv nnz capacity | gemm N
    ("p2", "<u4"),     # spmv Poisson table id | gemm K
    ("kind", "<u2"),
    ("prio", "<i2"),
])
assert JOB_DTYPE.itemsize == 64


# ---------------------------------------------------------------- SplitMix64
def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=_U64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


def sm64_at(key, i):
    """The i-th output (0-based) of the SplitMix64 stream seeded with ``key``."""
    k = np.asarray(key, dtype=_U64)
    i = np.asarray(i, dtype=_U64)
    with np.errstate(over="ignore"):
        return mix64(k + (i + _U64(1)) * _U64(GAMMA))


def stream_key(job_key: int, stream: int) -> int:
    return int(sm64_at(job_key, stream))


def job_keys(seed: int, n: int) -> np.ndarray:
    return sm64_at(seed, np.arange(n, dtype=np.uint64))


# ------------------------------------------------------------ element values
def uniform_pm1_f32(h, odd=False) -> np.ndarray:
    """The uniform of an even (bits 40..63 of h) or odd (bits 8..31) element."""
    h = np.asarray(h, dtype=_U64)
    b = np.where(np.asarray(odd, bool), (h >> _U64(8)) & _U64(0xFFFFFF), h >> _U64(40))
    return (b.astype(np.float64) * 2.0 ** -23 - 1.0).astype(np.float32)


def uniform_stream_f32(key: int, e) -> np.ndarray:
    """Elements e of the uniform stream with key ``key`` (two per hash)."""
    e = np.asarray(e, dtype=_U64)
    return uniform_pm1_f32(sm64_at(key, e >> _U64(1)), (e & _U64(1)) == _U64(1))


def normal_pair_f32(h, odd) -> np.ndarray:
    """Box-Muller: the cos branch for even elements, the sin branch for odd."""
    h = np.asarray(h, dtype=_U64)
    u1 = ((h >> _U64(40)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = ((h >> _U64(16)) & _U64(0xFFFFFF)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return np.where(np.asarray(odd, bool), r * np.sin(ang), r * np.cos(ang)).astype(np.float32)


def column_pair(h, odd, n: int) -> np.ndarray:
    """Multiply-shift of the high (even element) or low (odd) 32 bits."""
    h = np.asarray(h, dtype=_U64)
    w = np.where(np.asarray(odd, bool), h & _U64(0xFFFFFFFF), h >> _U64(32))
    with np.errstate(over="ignore"):
        return ((w * _U64(n)) >> _U64(32)).astype(np.int64)


def spmv_columns(col_key: int, e, n: int) -> np.ndarray:
    e = np.asarray(e, dtype=_U64)
    return column_pair(sm64_at(col_key, e >> _U64(1)), (e & _U64(1)) == _U64(1), n)


def spmv_values(val_key: int, e) -> np.ndarray:
    e = np.asarray(e, dtype=_U64)
    return normal_pair_f32(sm64_at(val_key, e >> _U64(1)), (e & _U64(1)) == _U64(1))


def bf16_stream_f32(key: int, e) -> np.ndarray:
    """Elements e of the bf16 stream with key ``key`` as the fp32 uniforms
    they round from (four per hash, 16 bits each)."""
    e = np.asarray(e, dtype=_U64)
    h = sm64_at(key, e >> _U64(2))
    b = (h >> (_U64(16) * (e & _U64(3)))) & _U64(0xFFFF)
    return (b.astype(np.float64) * 2.0 ** -15 - 1.0).astype(np.float32)


def bf16_bits_rne(x_f32) -> np.ndarray:
    """bf16 bit patterns of fp32 values, round to nearest, ties to even."""
    b = np.asarray(x_f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> _U64(16)) & _U64(1)
    return (((b + _U64(0x7FFF) + lsb) >> _U64(16)) & _U64(0xFFFF)).astype(np.uint16)


def bf16_bits_to_f64(bits) -> np.ndarray:
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def poisson_cdf_table(lam: float) -> np.ndarray:
    """Inverse-CDF thresholds of Poisson(lam) on 32-bit uniforms.

    T[k] = ceil(F(k) * 2^32) = 2^32 - floor(S(k) * 2^32), with F the CDF and
    S(k) = P(X > k) summed from the far tail down so it stays accurate where
    F is near 1; T[63] = 2^32 caps a row at 63 entries. A row whose 32-bit
    uniform is u gets length #{k : T[k] <= u}, the smallest k with
    F(k) > u / 2^32.
    """
    top = 400
    p = [math.exp(-lam + i * math.log(lam) - math.lgamma(i + 1)) for i in range(top)]
    sf = [0.0] * top
    acc = 0.0
    for i in range(top - 1, -1, -1):
        sf[i] = acc
        acc += p[i]
    t = np.zeros(POISSON_TABLE_LEN, dtype=np.uint64)
    for k in range(POISSON_TABLE_LEN - 1):
        t[k] = (1 << 32) - int(math.floor(sf[k] * 4294967296.0))
    t[POISSON_TABLE_LEN - 1] = 1 << 32
    return t


def row_lengths(len_key: int, rows_idx, table: np.ndarray) -> np.ndarray:
    u = sm64_at(len_key, rows_idx) >> _U64(32)
    return np.searchsorted(table, u, side="right").astype(np.int64)


def spmv_nnz_cap(rows: int, lam: float) -> int:
    """Declared capacity for the non-zeros of an SpMV job.

    The row lengths are iid Poisson(lam), so nnz ~ Poisson(rows * lam); the
    job sizes its col / val arrays for mean + 8 standard deviations + 64
    (exceeded with probability below 1e-14), the way an application sizes
    its buffers before it knows the exact count.
    """
    mu = rows * lam
    return int(math.ceil(mu + 8.0 * math.sqrt(mu) + 64))


def spmv_nnz(job_key: int, rows: int, table: np.ndarray, chunk: int = 1 << 22) -> int:
    k = stream_key(job_key, 1)
    total = 0
    for s in range(0, rows, chunk):
        idx = np.arange(s, min(rows, s + chunk), dtype=np.uint64)
        total += int(row_lengths(k, idx, table).sum())
    return total


# ------------------------------------------------------- declared job layout
def r256(x: int) -> int:
    return (x + 255) // 256 * 256


def triad_layout(n: int) -> dict:
    """a, b, c contiguous: offsets 0, 4n, 8n (n a multiple of 64)."""
    return {"a": 0, "b": 4 * n, "c": 8 * n, "total": 12 * n}


def spmv_layout(rows: int, nnz: int) -> dict:
    ptr_bytes = (8 if nnz >= (1 << 31) else 4) * (rows + 1)
    chunks = (rows + SPMV_CHUNK_ROWS - 1) // SPMV_CHUNK_ROWS
    off = 0
    lay = {}
    for name, size in (("row_ptr", ptr_bytes), ("col", 4 * nnz), ("val", 4 * nnz),
                       ("x", 4 * rows), ("y", 4 * rows), ("scan", 8 * (chunks + 1))):
        lay[name] = off
        off += r256(size)
    lay["total"] = off
    lay["ptr64"] = nnz >= (1 << 31)
    return lay


def gemm_layout(m: int, n: int, k: int) -> dict:
    a = r256(2 * m * k)
    b = r256(2 * n * k)
    c = r256(4 * m * n)
    return {"A": 0, "B": a, "C": a + b, "total": a + b + c}


def triad_alg_bytes(n: int) -> int:
    return 12 * n


def spmv_alg_bytes(rows: int, nnz: int) -> int:
    ptr = 8 if nnz >= (1 << 31) else 4
    return ptr * (rows + 1) + 8 * nnz + 4 * rows + 4 * rows


def gemm_flops(m: int, n: int, k: int) -> int:
    return 2 * m * n * k


def declared_duration(kind: int, p0: int, p1: int, p2: int) -> int:
    if kind == KIND_TRIAD:
        b = triad_alg_bytes(p0)
        return -(-b * 1000 // REF_BYTES_PER_US)
    if kind == KIND_SPMV:
        b = spmv_alg_bytes(p0, p1)
        return -(-b * 1000 // REF_BYTES_PER_US)
    return -(-gemm_flops(p0, p1, p2) // REF_FLOP_PER_NS)


# --------------------------------------------------------------- trace build
@dataclass
class Trace:
    name: str
    jobs: np.ndarray          # JOB_DTYPE records, job id = index
    budget: int               # pool bytes
    tables: np.ndarray        # (n_tables, 64) uint64 Poisson CDF tables
    lambdas: tuple

    def __len__(self):
        return len(self.jobs)


def _u01(key: int, idx) -> np.ndarray:
    """Uniform [0,1) doubles from a SplitMix64 stream (53-bit)."""
    return (sm64_at(key, idx) >> _U64(11)).astype(np.float64) * 2.0 ** -53


def _log_uniform_int(u: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def _floor64(x):
    return np.maximum(64, (np.asarray(x, np.int64) // 64) * 64)


def make_jobs(kinds, sizes, arrivals, seed: int, lams, lam_id=None, prio=None,
              timeout=None) -> np.ndarray:
    n = len(kinds)
    jobs = np.zeros(n, dtype=JOB_DTYPE)
    keys = job_keys(seed, n)
    for j in range(n):
        kind = int(kinds[j])
        rec = jobs[j]
        rec["kind"] = kind
        rec["key"] = keys[j]
        rec["arrival_ns"] = int(arrivals[j])
        rec["prio"] = 0 if prio is None else int(prio[j])
        rec["timeout_ns"] = NO_TIMEOUT if timeout is None else int(timeout[j])
        if kind == KIND_TRIAD:
            nn = int(sizes[j])
            rec["p0"] = nn
            need = triad_layout(nn)["total"]
            dur = declared_duration(kind, nn, 0, 0)
        elif kind == KIND_SPMV:
            rows = int(sizes[j])
            tid = 0 if lam_id is None else int(lam_id[j])
            cap = spmv_nnz_cap(rows, lams[tid])
            rec["p0"], rec["p1"], rec["p2"] = rows, cap, tid
            need = spmv_layout(rows, cap)["total"]
            dur = declared_duration(kind, rows, int(round(rows * lams[tid])), 0)
        else:
            s = int(sizes[j])
            rec["p0"], rec["p1"], rec["p2"] = s, s, s
            need = gemm_layout(s, s, s)["total"]
            dur = declared_duration(kind, s, s, s)
        rec["need"] = need
        rec["duration_ns"] = dur
    return jobs


def trace_single_kind_t0(seed: int, n_jobs: int, lo: int, hi: int, budget: int,
                         name: str) -> Trace:
    """Triad jobs all arriving at t=0 with n log-uniform in [lo, hi]."""
    tkey = int(sm64_at(seed ^ 0xC1, 0))
    n = _floor64(_log_uniform_int(_u01(tkey, np.arange(n_jobs)), lo, hi))
    tables = np.stack([poisson_cdf_table(16.0)])
    jobs = make_jobs([KIND_TRIAD] * n_jobs, n, np.zeros(n_jobs, np.int64), seed, (16.0,))
    return Trace(name, jobs, budget, tables, (16.0,))


def trace_c1(seed: int = 0) -> Trace:
    """8 FP32 triads at t=0, n log-uniform [2^20, 2^24], budget 1 GiB."""
    return trace_single_kind_t0(seed, 8, 1 << 20, 1 << 24, 1 << 30, "triad8_t0_1GiB")


def _mixed_kinds_sizes(tkey: int, n_jobs: int, triad_rng, spmv_rng, gemm_set):
    idx = np.arange(n_jobs)
    uk = _u01(tkey, 3 * idx)
    us = _u01(tkey, 3 * idx + 1)
    kinds = np.where(uk < 0.4, KIND_TRIAD, np.where(uk < 0.7, KIND_SPMV, KIND_GEMM))
    sizes = np.zeros(n_jobs, np.int64)
    t = kinds == KIND_TRIAD
    sizes[t] = _floor64(_log_uniform_int(us[t], *triad_rng))
    s = kinds == KIND_SPMV
    sizes[s] = _log_uniform_int(us[s], *spmv_rng)
    g = kinds == KIND_GEMM
    gs = np.asarray(gemm_set, np.int64)
    sizes[g] = gs[np.minimum((us[g] * len(gs)).astype(np.int64), len(gs) - 1)]
    return kinds, sizes


def poisson_arrivals(tkey: int, n_jobs: int, rate_per_s: float) -> np.ndarray:
    u = _u01(tkey, 3 * np.arange(n_jobs) + 2)
    gaps = np.rint(-np.log1p(-u) / rate_per_s * 1e9).astype(np.int64)
    return np.cumsum(gaps) - gaps[0]


def trace_mixed(seed: int = 0, n_jobs: int = 256, rate_per_s: float | None = 200.0,
                budget: int = 16 << 30, name: str = "mixed256_16GiB",
                triad_rng=(1 << 20, 1 << 26), spmv_rng=(1e5, 1e7),
                gemm_set=(256, 512, 1024, 2048, 4096, 8192), lam: float = 16.0) -> Trace:
    """Mixed trace: 40% triad, 30% CSR SpMV, 30% BF16 GEMM, Poisson arrivals.

    ``rate_per_s=None`` puts every arrival at t=0 (the saturated trace).
    """
    tkey = int(sm64_at(seed ^ 0xC2, 0))
    kinds, sizes = _mixed_kinds_sizes(tkey, n_jobs, triad_rng, spmv_rng, gemm_set)
    if rate_per_s is None:
        arr = np.zeros(n_jobs, np.int64)
    else:
        arr = poisson_arrivals(tkey, n_jobs, rate_per_s)
    tables = np.stack([poisson_cdf_table(lam)])
    jobs = make_jobs(kinds, sizes, arr, seed, (lam,))
    return Trace(name, jobs, budget, tables, (lam,))


def trace_c2(seed: int = 0, saturated: bool = False) -> Trace:
    return trace_mixed(seed, 256, None if saturated else 200.0, 16 << 30,
                       "mixed256_16GiB_" + ("t0" if saturated else "poisson200"))


def trace_c3(seed: int = 0, n_jobs: int = 128, burst: int = 16,
             gap_ns: int = 200_000_000, budget: int = 170 << 30,
             need_rng=(2 << 30, 60 << 30)) -> Trace:
    """Memory pressure: needs log-uniform [2, 60] GiB, bursts of 16."""
    tkey = int(sm64_at(seed ^ 0xC3, 0))
    idx = np.arange(n_jobs)
    uk = _u01(tkey, 3 * idx)
    un = _u01(tkey, 3 * idx + 1)
    target = _log_uniform_int(un, *need_rng)
    kinds = np.where(uk < 0.4, KIND_TRIAD, np.where(uk < 0.7, KIND_SPMV, KIND_GEMM))
    sizes = np.zeros(n_jobs, np.int64)
    for j in range(n_jobs):
        if kinds[j] == KIND_TRIAD:
            sizes[j] = max(64, target[j] // 12 // 64 * 64)
        elif kinds[j] == KIND_SPMV:
            sizes[j] = max(1024, target[j] // (8 * 17 + 12 + 8))
        else:
            sizes[j] = max(128, int(math.isqrt(int(target[j]) // 8)) // 128 * 128)
    arr = (idx // burst) * gap_ns
    tables = np.stack([poisson_cdf_table(16.0)])
    jobs = make_jobs(kinds, sizes, arr, seed, (16.0,))
    return Trace("pressure128_170GiB", jobs, budget, tables, (16.0,))


def trace_c4(seed: int = 0, n_jobs: int = 10_000, budget: int = 2 << 30) -> Trace:
    """Batching: tiny jobs, all at t=0."""
    tkey = int(sm64_at(seed ^ 0xC4, 0))
    kinds, sizes = _mixed_kinds_sizes(tkey, n_jobs, (4096, 262144), (1024, 65536),
                                      (64, 128, 256, 512))
    tables = np.stack([poisson_cdf_table(8.0)])
    jobs = make_jobs(kinds, sizes, np.zeros(n_jobs, np.int64), seed, (8.0,))
    return Trace("tiny10k_2GiB", jobs, budget, tables, (8.0,))


def trace_c5(seed: int = 0, n_jobs: int = 100_000, rate_per_s: float = 1000.0,
             budget: int = 64 << 30) -> Trace:
    """Serving: open-loop Poisson stream with the mixed-trace size mix."""
    tr = trace_mixed(seed, n_jobs, rate_per_s, budget, f"serve{n_jobs}_{int(rate_per_s)}rps")
    return tr


def trace_identical(n_jobs: int, need: int, duration: int, budget: int) -> np.ndarray:
    """k identical triad-shaped records at t=0 (for admission-only tests)."""
    jobs = np.zeros(n_jobs, dtype=JOB_DTYPE)
    jobs["need"] = need
    jobs["duration_ns"] = duration
    jobs["timeout_ns"] = NO_TIMEOUT
    jobs["kind"] = KIND_TRIAD
    return jobs


def random_admission_trace(seed: int, n_jobs: int, budget: int, max_arrival: int = 50,
                           max_dur: int = 40, prio_levels: int = 1,
                           timeout_frac: float = 0.0) -> np.ndarray:
    """Small integer-time traces for admission-only tests (no job data)."""
    key = int(sm64_at(seed ^ 0xAD, 0))
    idx = np.arange(n_jobs)
    u = [_u01(key, 5 * idx + s) for s in range(5)]
    jobs = np.zeros(n_jobs, dtype=JOB_DTYPE)
    arr = np.sort(np.floor(u[0] * max_arrival).astype(np.int64))
    jobs["arrival_ns"] = arr
    gran = budget // GRANULE
    jobs["need"] = (1 + np.floor(u[1] * gran).astype(np.int64)) * GRANULE - np.floor(u[2] * 200).astype(np.int64)
    jobs["need"] = np.maximum(jobs["need"], 1)
    jobs["duration_ns"] = 1 + np.floor(u[3] * max_dur).astype(np.int64)
    jobs["prio"] = np.floor(u[4] * prio_levels).astype(np.int64)
    to = np.where(u[2] < timeout_frac, 1 + np.floor(u[3] * max_dur).astype(np.int64), 0)
    tmo = np.full(n_jobs, NO_TIMEOUT, dtype=np.uint64)
    tmo[to > 0] = to[to > 0].astype(np.uint64)
    jobs["timeout_ns"] = tmo
    jobs["kind"] = KIND_TRIAD
    return jobs


def random_lifecycle_calls(seed: int, n_ops: int, budget: int, prio_levels: int = 1,
                           p_declare: float = 0.45, p_release: float = 0.35) -> list:
    """A seeded sequence of life-cycle calls by many clients, for step-by-step
    tests of a live scheduler: ("declare", need, prio), ("release", ticket,
    bytes) and ("cancel", ticket). Tickets are numbered in declare order.

    Needs are log-uniform between 1 byte and half the pool, with a few of 0
    bytes and a few of the whole pool; none is larger than the pool, so every
    declare gets a ticket. A release or cancel names a ticket declared
    earlier, whatever its state (the scheduler refuses what is not valid).
    Release sizes: 0 (all), a part of the declared need, or more than it.
    """
    key = int(sm64_at(seed ^ 0x11FE, 0))
    idx = np.arange(n_ops)
    u = [_u01(key, 6 * idx + s) for s in range(6)]
    calls = []
    declared = []                         # declared need of each ticket
    for k in range(n_ops):
        r = float(u[0][k])
        if not declared or r < p_declare:
            w = float(u[1][k])
            if w < 0.04:
                need = 0
            elif w < 0.07:
                need = budget
            else:
                need = int(math.floor(math.exp(float(u[2][k]) * math.log(max(budget // 2, 2)))))
            prio = int(math.floor(float(u[3][k]) * prio_levels))
            calls.append(("declare", need, prio))
            declared.append(need)
            continue
        t = int(math.floor(float(u[4][k]) * len(declared)))
        if r < p_declare + p_release:
            v = float(u[5][k])
            need = declared[t]
            if v < 0.35 or need < 2:
                nbytes = 0
            elif v < 0.85:
                nbytes = 1 + int(math.floor((v - 0.35) / 0.5 * (need - 1)))
            else:
                nbytes = need + 1 + int(math.floor((v - 0.85) * 1e4))
            calls.append(("release", t, nbytes))
        else:
            calls.append(("cancel", t))
    return calls
