"""Pins of the CPU reference kernels against independent arithmetic."""
import struct
from fractions import Fraction

import numpy as np

from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg


def _f32(x: float) -> float:
    """Round a Python float (fp64) to fp32, nearest-even, via struct."""
    return struct.unpack("<f", struct.pack("<f", x))[0]


def test_triad_two_roundings_match_scalar_definition():
    key = 0x1234
    a = K.triad(key, 4096)
    b, c = K.triad_inputs(key, np.arange(4096, dtype=np.uint64))
    for i in range(0, 4096, 7):
        want = _f32(float(b[i]) + _f32(3.0 * float(c[i])))
        assert a[i] == np.float32(want)
    # and it is not the single-rounding (fused) result everywhere
    fused = (b.astype(np.float64) + 3.0 * c.astype(np.float64)).astype(np.float32)
    assert np.any(fused != a)


def test_triad_sampled_equals_full():
    key = 99
    a = K.triad(key, 10000)
    idx = np.array([0, 1, 777, 9999])
    assert np.array_equal(K.triad_sampled(key, idx), a[idx])


def test_spmv_matches_dense_product():
    table = tg.poisson_cdf_table(16.0)
    rows = 300
    ptr, col, val, x = K.spmv_csr(7, rows, table)
    dense = np.zeros((rows, rows))
    for r in range(rows):
        for e in range(ptr[r], ptr[r + 1]):
            dense[r, col[e]] += float(val[e])          # duplicates add up
    y, mag = K.spmv(7, rows, table)
    ref = dense @ x.astype(np.float64)
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)
    assert np.all(mag >= np.abs(y) - 1e-12)
    assert ptr[-1] == tg.spmv_nnz(7, rows, table)


def test_spmv_sampled_equals_full():
    table = tg.poisson_cdf_table(8.0)
    y, mag = K.spmv(11, 2000, table)
    rows = np.array([0, 5, 1999, 1234])
    ys, ms, _ = K.spmv_sampled(11, 2000, table, rows)
    assert np.allclose(ys, y[rows], rtol=1e-14, atol=1e-14)
    assert np.allclose(ms, mag[rows], rtol=1e-14)


def test_spmv_streamed_equals_sampled():
    table = tg.poisson_cdf_table(16.0)
    rows = 5000
    sample = np.array([0, 1, 17, 2047, 2048, 4095, 4999])
    ys, ms, ptr = K.spmv_sampled(3, rows, table, sample)
    y2, m2, st, en, nnz = K.spmv_sampled_streamed(3, rows, table, sample, chunk=1024)
    assert np.array_equal(ys, y2) and np.array_equal(ms, m2)
    assert np.array_equal(st, ptr[sample]) and np.array_equal(en, ptr[sample + 1]) and nnz == ptr[-1]


def test_gemm_exact_for_small_k():
    # bf16 products are exact in fp64 and sums of 32 of them stay exact:
    # compare with rational arithmetic
    m, n, k = 8, 6, 32
    c = K.gemm(5, m, n, k)
    a = K.gemm_a(5, m, k)
    bt = K.gemm_bt(5, n, k)
    for i in range(m):
        for j in range(n):
            exact = sum(Fraction(float(a[i, q])) * Fraction(float(bt[j, q])) for q in range(k))
            assert Fraction(float(c[i, j])) == exact


def test_gemm_transposed_operand_is_detected():
    m = n = k = 16
    c = K.gemm(3, m, n, k)
    a = K.gemm_a(3, m, k)
    bt = K.gemm_bt(3, n, k)
    assert not np.allclose(c, a @ bt)          # B^T used as B would differ
    assert np.allclose(c, np.einsum("ik,jk->ij", a, bt))


def test_gemm_sampled_equals_full():
    c = K.gemm(8, 64, 48, 40)
    ii = np.array([0, 63, 17, 5])
    jj = np.array([0, 47, 3, 40])
    assert np.allclose(K.gemm_sampled(8, 64, 48, 40, ii, jj), c[ii, jj], rtol=1e-15, atol=0)


def test_gemm_inputs_are_bf16_rounded_uniforms():
    a = K.gemm_a(2, 4, 64)
    assert np.all(np.abs(a) <= 1.0)
    bits = a.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)          # representable in bf16
