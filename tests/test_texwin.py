"""The texture windows a pool gets for the SpMV's x gathers (csrc/texwin.h),
on the CPU, against a brute-force model: windows of the largest power-of-two
element count the device allows, every half window, clipped to the pool;
every byte of the pool in some window; an array is given a window exactly
when some window holds it whole, and the window given holds it; every
array of at most half a window inside the pool gets one."""
import ctypes
import os
import sys
import tempfile

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "texwin_harness"))
import texwin_build  # noqa: E402

MiB, GiB = 1 << 20, 1 << 30
B300 = (1 << 28, 512)          # elements a 1-D linear texture spans, texture alignment


@pytest.fixture(scope="module")
def tw():
    L = ctypes.CDLL(texwin_build.build(tempfile.mkdtemp(prefix="sg_texwin_")))
    U = ctypes.c_uint64
    L.tw_layout.argtypes = [U, U, U, ctypes.POINTER(U)]
    L.tw_layout.restype = None
    L.tw_size.argtypes = [U, U, U, U]
    L.tw_size.restype = U
    L.tw_pick.argtypes = [U, U, U, U, U]
    L.tw_pick.restype = ctypes.c_int64

    class H:
        @staticmethod
        def layout(b, e, a):
            out = (U * 3)()
            L.tw_layout(b, e, a, out)
            return tuple(out)

        size = staticmethod(L.tw_size)
        pick = staticmethod(L.tw_pick)
    return H


def _model_windows(bytes_, max_elems, align):
    """The windows by their definition: (start, end) byte ranges."""
    if bytes_ < 4 or max_elems < (1 << 16):
        return []
    elems = 1 << (min(max_elems, 1 << 30).bit_length() - 1)
    win = 4 * elems
    step = win // 2
    if step % align:
        return []
    out, start = [], 0
    while True:
        end = min(start + win, bytes_)
        out.append((start, start + ((end - start) & ~3)))
        if start + win >= bytes_:
            return out
        start += step


@pytest.mark.parametrize("bytes_,max_elems,align", [
    (16 * GiB, *B300), (GiB, *B300), (GiB + GiB // 4, *B300), (170 * GiB, *B300), (64 * MiB, *B300),
    (3 * GiB + 2, *B300), (4, *B300), (1 << 20, 1 << 16, 512), (5 * MiB + 7, 1 << 16, 512),
    ((1 << 20) + 100, (1 << 17) + 5, 256), (GiB, 1 << 15, 512), (GiB, 1 << 16, 1 << 20)])
def test_layout_matches_the_definition(tw, bytes_, max_elems, align):
    win, step, count = tw.layout(bytes_, max_elems, align)
    model = _model_windows(bytes_, max_elems, align)
    assert count == len(model)
    for i, (s, e) in enumerate(model):
        assert i * step == s
        assert tw.size(bytes_, max_elems, align, i) == e - s
    if model:
        assert win == 2 * step and win % 4 == 0 and step % align == 0
        # every byte of the pool (whole elements) is in some window
        covered = 0
        for s, e in model:
            assert s <= covered
            covered = max(covered, e)
        assert covered == bytes_ & ~3


@pytest.mark.parametrize("bytes_,max_elems,align", [
    (GiB + GiB // 4, *B300), (3 * GiB + 2, *B300), (5 * MiB + 8, 1 << 16, 512),
    ((1 << 20) + 100, (1 << 17) + 5, 256)])
def test_pick_is_exact(tw, bytes_, max_elems, align):
    model = _model_windows(bytes_, max_elems, align)
    win, step, _ = tw.layout(bytes_, max_elems, align)
    rng = np.random.default_rng(bytes_ % 1000003)
    offs = np.concatenate([rng.integers(0, bytes_ // 4, 3000) * 4,
                           np.array([s for s, _ in model] + [e - 4 for _, e in model] + [0, (bytes_ & ~3) - 4]),
                           np.array([s + step - 4 for s, _ in model])])
    for off in offs:
        off = int(off)
        if off < 0 or off >= bytes_:
            continue
        for nbytes in (0, 4, 64, step // 2, step - (off % 4096), step, step + 4, win, win + 4,
                       int(rng.integers(0, win // 4)) * 4):
            got = tw.pick(bytes_, max_elems, align, off, nbytes)
            holders = [i for i, (s, e) in enumerate(model) if s <= off and off + nbytes <= e]
            if holders:
                assert got in holders, (off, nbytes, got, holders)
            else:
                assert got == -1, (off, nbytes, got)
            if nbytes <= step and off + nbytes <= (bytes_ & ~3):
                assert got >= 0, (off, nbytes)


def test_pick_refuses_misaligned_and_outside(tw):
    b, e, a = GiB, *B300
    assert tw.pick(b, e, a, 2, 4) == -1
    assert tw.pick(b, e, a, b, 0) == -1
    assert tw.pick(b, e, a, b - 4, 8) == -1
    assert tw.pick(b, e, a, b - 4, 4) == 0
    assert tw.pick(b, 1 << 15, a, 0, 4) == -1          # device limit below 2^16 elements: no windows
