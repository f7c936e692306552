"""The OpenMP form of the oracle's job results (the CPU baseline) gives the
same results as the plain definitions in oracle/kernels.py, which carry the
pins (closed forms, dense and rational references): the triad bit for bit,
the SpMV within a few float ulps of a value per product (libm and numpy may
round the Box-Muller transcendentals differently in the last place) and the
GEMM operands bit for bit."""
import numpy as np

from oracle import kernels as K
from oracle import omp
from paper_1712_04495_b300 import tracegen as tg


def test_triad_equals_definition():
    for key, n in ((3, 1), (5, 100_003), (9, 1 << 16)):
        assert np.array_equal(omp.triad(key, n).view(np.uint32), K.triad(key, n).view(np.uint32))


def test_spmv_equals_definition():
    table = tg.poisson_cdf_table(16.0)
    rows = 20_000
    y, mag, ptr = omp.spmv(7, rows, table)
    assert np.array_equal(ptr, K.spmv_row_ptr(7, rows, table))
    y_ref, mag_ref = K.spmv(7, rows, table)
    assert np.all(np.abs(y - y_ref) <= 1e-6 * mag_ref + 1e-300)
    assert np.allclose(mag, mag_ref, rtol=1e-6, atol=0)


def test_gemm_equals_definition():
    c = omp.gemm(4, 72, 40, 96)
    assert np.array_equal(c, K.gemm(4, 72, 40, 96))


def test_runs_on_several_threads():
    assert omp.threads() >= 1
