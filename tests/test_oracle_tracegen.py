"""Pins of the seeded input generator against published definitions."""
import math
import struct

import numpy as np
import pytest
import torch

from paper_1712_04495_b300 import tracegen as tg


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 0 (the reference test vector
    # of Steele et al.'s generator, also Java's SplittableRandom mix64).
    out = tg.sm64_at(0, np.arange(3))
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_scalar_definition():
    # random access equals stepping the state by GAMMA
    M = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    state = 12345
    seq = []
    for _ in range(10):
        state = (state + tg.GAMMA) & M
        seq.append(mix(state))
    assert [int(x) for x in tg.sm64_at(12345, np.arange(10))] == seq


def test_uniform_exact_and_range():
    h = tg.sm64_at(7, np.arange(100000))
    u = tg.uniform_pm1_f32(h)
    assert u.min() >= -1.0 and u.max() < 1.0
    # exactness: u + 1 is a multiple of 2^-23
    k = (u.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.all(k == np.floor(k))
    assert np.array_equal(k.astype(np.uint64), (h >> np.uint64(40)))
    assert abs(float(u.mean())) < 0.01
    # odd elements: bits 8..31 of the same hash
    v = tg.uniform_pm1_f32(h, odd=True)
    kv = (v.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.all(kv == np.floor(kv)) and v.min() >= -1.0 and v.max() < 1.0
    assert np.array_equal(kv.astype(np.uint64), (h >> np.uint64(8)) & np.uint64(0xFFFFFF))
    assert abs(float(v.mean())) < 0.01
    # the two halves of one hash are uncorrelated
    assert abs(float(np.corrcoef(u, v)[0, 1])) < 0.01


def test_uniform_stream_two_elements_per_hash():
    """Element e of a uniform stream, from a scalar restatement: the SplitMix64
    output e // 2, its bits 40..63 (e even) or 8..31 (e odd), times 2^-23, minus 1."""
    M = (1 << 64) - 1
    key = 0x1234_5678_9ABC_DEF0

    def out(k, i):
        z = (k + (i + 1) * tg.GAMMA) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    e = np.array([0, 1, 2, 3, 4, 5, 1000, 1001, (1 << 33) + 6, (1 << 33) + 7], dtype=np.uint64)
    got = tg.uniform_stream_f32(key, e)
    for ei, g in zip(e.tolist(), got.tolist()):
        h = out(key, ei // 2)
        b = (h >> 8) & 0xFFFFFF if ei % 2 else h >> 40
        assert g == np.float32(b * 2.0 ** -23 - 1.0), ei
    u = tg.uniform_stream_f32(key, np.arange(200000, dtype=np.uint64))
    assert abs(float(u.mean())) < 0.01 and abs(float(u.var()) - 1.0 / 3.0) < 0.01
    assert abs(float(np.corrcoef(u[0::2], u[1::2])[0, 1])) < 0.01


def test_bf16_stream_four_elements_per_hash():
    """Element e of a bf16 stream, from a scalar restatement: SplitMix64 output
    e // 4, its 16-bit field number e % 4 (from the low end), times 2^-15, minus 1."""
    M = (1 << 64) - 1
    key = 0x0F1E_2D3C_4B5A_6978

    def out(k, i):
        z = (k + (i + 1) * tg.GAMMA) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    e = np.array([0, 1, 2, 3, 4, 7, 4001, 4002, (1 << 34) + 5], dtype=np.uint64)
    got = tg.bf16_stream_f32(key, e)
    for ei, g in zip(e.tolist(), got.tolist()):
        b = (out(key, ei // 4) >> (16 * (ei % 4))) & 0xFFFF
        assert g == np.float32(b * 2.0 ** -15 - 1.0), ei
    u = tg.bf16_stream_f32(key, np.arange(400000, dtype=np.uint64))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(float(u.mean())) < 0.01 and abs(float(u.var()) - 1.0 / 3.0) < 0.01
    for j in range(1, 4):   # the fields of one hash are uncorrelated
        assert abs(float(np.corrcoef(u[0::4], u[j::4])[0, 1])) < 0.01
    # and the bf16 values carry the whole 16-bit grid: 2^16 distinct uniforms
    assert len(np.unique(tg.bf16_stream_f32(key, np.arange(1 << 20, dtype=np.uint64)))) > 60000


def test_bf16_rne_matches_torch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(200000).astype(np.float32)
    # add exact ties: low 16 bits = 0x8000
    ties = np.uint32(0x3F800000) + (rng.integers(0, 128, 2000, dtype=np.uint32) << np.uint32(16)) + np.uint32(0x8000)
    x = np.concatenate([x, ties.view(np.float32)])
    ours = tg.bf16_bits_rne(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_poisson_table_matches_scipy_quantiles():
    from scipy.stats import poisson
    for lam in (8.0, 16.0):
        t = tg.poisson_cdf_table(lam)
        assert t[-1] == 1 << 32 and np.all(np.diff(t.astype(np.int64)) >= 0)
        u = np.array([0, 1, 12345, 1 << 31, (1 << 32) - 1, 3_000_000_000], dtype=np.uint64)
        lens = np.searchsorted(t, u, side="right")
        q = np.nextafter(u.astype(np.float64) / 2 ** 32, 2.0)   # F(k) > u/2^32
        ref = poisson.ppf(q, lam)
        assert np.array_equal(lens, ref.astype(np.int64))


def test_row_length_search_in_32_bits_is_exact():
    """The CUDA CSR build counts a row's length with 32-bit compares against
    the table saturated to 2^32 - 1, and with the 64-bit table only for the
    uniform 2^32 - 1. A model of that search gives the 64-bit count for every
    uniform at and around each threshold of both Poisson tables used."""
    for lam in (8.0, 16.0):
        T = tg.poisson_cdf_table(lam).astype(np.uint64)
        T32 = np.where(T >> np.uint64(32), np.uint64(0xFFFFFFFF), T)
        cand = {0, 1, 0xFFFFFFFE, 0xFFFFFFFF}
        for t in T.tolist():
            cand.update(v for v in (t - 1, t, t + 1) if 0 <= v <= 0xFFFFFFFF)
        for u in sorted(cand):
            want = int(np.sum(T <= np.uint64(u)))
            pos = 0
            step = 32
            while step:
                if u != 0xFFFFFFFF:
                    if T32[pos + step - 1] <= u:
                        pos += step
                elif T[pos + step - 1] <= u:
                    pos += step
                step >>= 1
            assert pos == want, (lam, u, pos, want)


def test_row_length_statistics():
    t = tg.poisson_cdf_table(16.0)
    lens = tg.row_lengths(99, np.arange(200000, dtype=np.uint64), t)
    assert abs(lens.mean() - 16.0) < 0.05
    assert abs(lens.var() - 16.0) < 0.3


def test_columns_in_range_and_uniform():
    e = np.arange(200000)
    for n in (1, 7, 1000, 10_000_000):
        c = tg.spmv_columns(3, e, n)
        assert c.min() >= 0 and c.max() < n
    c = tg.spmv_columns(3, e, 10)
    counts = np.bincount(c, minlength=10)
    assert np.all(np.abs(counts - 20000) < 5 * np.sqrt(20000))
    # an even and an odd element share a hash but use different halves
    assert np.mean(tg.spmv_columns(3, e[0::2], 1 << 20) == tg.spmv_columns(3, e[1::2], 1 << 20)) < 1e-3


def test_normal_pair_moments_and_independence():
    v = tg.spmv_values(5, np.arange(400000)).astype(np.float64)
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01
    assert np.all(np.isfinite(v))
    even, odd = v[0::2], v[1::2]
    assert abs(np.corrcoef(even, odd)[0, 1]) < 0.01
    # the pair lies on one circle: even^2 + odd^2 = -2 ln u1
    h = tg.sm64_at(5, np.arange(200000))
    u1 = ((h >> np.uint64(40)).astype(np.float64) + 1.0) * 2.0 ** -24
    assert np.allclose(even ** 2 + odd ** 2, -2.0 * np.log(u1), rtol=1e-5, atol=1e-5)


def test_layouts_aligned():
    for n in (64, 1 << 20, 5 << 20):
        lay = tg.triad_layout(n)
        assert lay["b"] % 256 == 0 and lay["c"] % 256 == 0 and lay["total"] == 12 * n
    lay = tg.spmv_layout(100003, 1600000)
    for k in ("row_ptr", "col", "val", "x", "y", "scan"):
        assert lay[k] % 256 == 0
    assert not lay["ptr64"]
    assert tg.spmv_layout(10, 1 << 31)["ptr64"]
    lay = tg.gemm_layout(256, 512, 128)
    assert lay["B"] == 2 * 256 * 128 and lay["C"] == lay["B"] + 2 * 512 * 128


def test_declared_duration_integer_ceil():
    assert tg.declared_duration(tg.KIND_GEMM, 8192, 8192, 8192) == -(-2 * 8192 ** 3 // 1_366_300)
    assert tg.declared_duration(tg.KIND_TRIAD, 64, 0, 0) == 1   # 768 B at 6.49 kB/us -> 0.118 ns -> 1


def test_c1_trace_shape():
    tr = tg.trace_c1()
    assert len(tr) == 8 and np.all(tr.jobs["arrival_ns"] == 0)
    n = tr.jobs["p0"]
    assert np.all(n % 64 == 0) and n.min() >= 1 << 20 - 0 and n.max() <= 1 << 24
    assert np.all(tr.jobs["need"] == 12 * n)


def test_mixed_trace_mix_and_rate():
    tr = tg.trace_mixed(0, 2000, 200.0, 16 << 30, spmv_rng=(1e3, 1e4))
    k = tr.jobs["kind"]
    frac = np.bincount(k, minlength=3) / len(k)
    assert abs(frac[0] - 0.4) < 0.04 and abs(frac[1] - 0.3) < 0.04
    gaps = np.diff(tr.jobs["arrival_ns"].astype(np.int64))
    assert abs(gaps.mean() - 5e6) < 0.5e6
    assert np.all(gaps >= 0)
