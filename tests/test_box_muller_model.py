"""The SpMV generator's Box-Muller (normal_pair in csrc/common.cuh) computes
its logarithm, sine and cosine from series. This is an fp32 model of those
steps, run over every input of each half of a hash (2^24 values of b1 and of
b2), checked against the fp64 definition the oracle uses. A wrong quadrant,
sign, coefficient or constant fails here; the device's own values are checked
against the oracle on the GPU (tests/test_gpu_kernels.py).

Model: products and fused multiply-adds are rounded to fp32 once; the division
and the reciprocal square root are taken correctly rounded (the device's
approximate forms add at most 2 units in the last place, inside the GPU
test's 1e-6 relative bound)."""
import math

import numpy as np

F32 = np.float32


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def _hexf(s):
    return F32(float.fromhex(s))


S1, S3, S5, S7, S9 = (_hexf(x) for x in ("0x1.921fb6p+0", "-0x1.4abbcep-1", "0x1.466bc6p-4",
                                          "-0x1.32d2ccp-8", "0x1.507834p-13"))
C2, C4, C6, C8, C10 = (_hexf(x) for x in ("-0x1.3bd3ccp+0", "0x1.03c1f0p-2", "-0x1.55d3c8p-6",
                                           "0x1.e1f506p-11", "-0x1.a6d1f2p-16"))
L3, L5, L7, L9 = (_hexf(x) for x in ("0x1.555556p-1", "0x1.99999ap-2", "0x1.24924ap-2", "0x1.c71c72p-3"))
LN2_HI, LN2_LO = _hexf("0x1.62e4p-1"), _hexf("0x1.7f7d1cp-20")


def _ulps(got, ref):
    """|got - ref| in units in the last place of ref rounded to fp32."""
    sp = np.spacing(np.abs(ref.astype(F32))).astype(np.float64)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(sp, np.finfo(F32).tiny)


def test_constants_are_the_series_coefficients():
    h = math.pi / 2
    for got, want in ((S1, h), (S3, -h ** 3 / 6), (S5, h ** 5 / 120), (S7, -h ** 7 / 5040),
                      (S9, h ** 9 / 362880), (C2, -h ** 2 / 2), (C4, h ** 4 / 24), (C6, -h ** 6 / 720),
                      (C8, h ** 8 / 40320), (C10, -h ** 10 / 3628800), (L3, 2 / 3), (L5, 2 / 5),
                      (L7, 2 / 7), (L9, 2 / 9)):
        assert got == F32(want)
    assert LN2_LO == F32(math.log(2) - float(LN2_HI))
    assert abs(float(LN2_HI) + float(LN2_LO) - math.log(2)) < 1e-12
    assert float(LN2_HI) * 2 ** 16 == int(float(LN2_HI) * 2 ** 16)   # 16 significant bits: k ln2_hi exact


def test_sin_cos_of_2pi_u2_every_input():
    b2 = np.arange(1 << 24, dtype=np.int64)
    q = (b2 + (1 << 21)) >> 22
    x = ((b2 - (q << 22)).astype(F32) * F32(2.0 ** -22)).astype(F32)
    x2 = (x * x).astype(F32)
    ps = _fma(x2, S9, S7)
    for c in (S5, S3, S1):
        ps = _fma(x2, ps, c)
    sn = (x * ps).astype(F32)
    pc = _fma(x2, C10, C8)
    for c in (C6, C4, C2):
        pc = _fma(x2, pc, c)
    cs = _fma(x2, pc, F32(1.0))
    odd, neg_s, neg_c = (q & 1) == 1, (q & 2) == 2, ((q + 1) & 2) == 2
    sv, cv = np.where(odd, cs, sn), np.where(odd, sn, cs)
    sin_v, cos_v = np.where(neg_s, -sv, sv), np.where(neg_c, -cv, cv)
    ang = 2.0 * np.pi * b2.astype(np.float64) * 2.0 ** -24
    rs, rc = np.sin(ang), np.cos(ang)
    big_s, big_c = np.abs(rs) > 1e-6, np.abs(rc) > 1e-6
    assert _ulps(sin_v[big_s], rs[big_s]).max() <= 2.0
    assert _ulps(cos_v[big_c], rc[big_c]).max() <= 2.0
    # at the zeros of sine and cosine (angles at multiples of pi/2) the model gives exact
    # zeros where fp64 leaves a remainder below 1e-12
    assert np.abs(sin_v.astype(np.float64) - rs).max() < 1e-6
    assert np.abs(sin_v[~big_s].astype(np.float64) - rs[~big_s]).max() < 1e-12
    assert np.abs(cos_v[~big_c].astype(np.float64) - rc[~big_c]).max() < 1e-12


def test_minus_two_ln_u1_every_input():
    b1 = np.arange(1 << 24, dtype=np.int64)
    v = (b1 + 1).astype(F32)                            # exact
    vb = v.view(np.uint32).astype(np.int64)
    mb = vb & 0x7FFFFF
    big = mb > 0x3504F3
    m = np.where(big, mb | 0x3F000000, mb | 0x3F800000).astype(np.uint32).view(F32)
    k = ((vb >> 23) - 127 + big.astype(np.int64) - 24).astype(F32)
    sq = ((m - F32(1)).astype(F32) / (m + F32(1)).astype(F32)).astype(F32)
    s2 = (sq * sq).astype(F32)
    pl = _fma(s2, L9, L7)
    for c in (L5, L3, F32(2.0)):
        pl = _fma(s2, pl, c)
    lnu = _fma(k, LN2_HI, _fma(k, LN2_LO, (sq * pl).astype(F32)))
    L = (F32(-2.0) * lnu).astype(F32)
    ref = -2.0 * np.log((b1 + 1).astype(np.float64) * 2.0 ** -24)
    assert L[-1] == 0.0 and ref[-1] == 0.0              # u1 = 1
    assert _ulps(L[:-1], ref[:-1]).max() <= 3.0
    # the radius as the device forms it, L * rsqrt(L), within a few units of sqrt(L)
    r = (L[:-1] * (1.0 / np.sqrt(L[:-1].astype(np.float64))).astype(F32)).astype(F32)
    assert _ulps(r, np.sqrt(ref[:-1])).max() <= 4.0
