"""The SpMV's x gathers through a texture window of a context's pool.

A context registers texture windows over its pool (1 GiB windows every
512 MiB on a B300); an SpMV whose x lies wholly inside one is gathered
through it, any other x with global loads. Both paths must give the same y
bit for bit, and the same y as the CPU oracle within the SpMV tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import kernels as K
from paper_1712_04495_b300 import tracegen as tg

pytestmark = pytest.mark.gpu

MiB = 1 << 20
GiB = 1 << 30


def _mods():
    from paper_1712_04495_b300 import abi, runtime
    return abi, runtime


def test_gather_path_follows_the_windows():
    abi, runtime = _mods()
    pool_bytes = GiB + GiB // 4        # windows [0, 1 GiB) and [512 MiB, 1.25 GiB)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    p = pool.data_ptr()
    outside = torch.empty(4096, dtype=torch.float32, device="cuda")
    assert abi.sg_spmv_gather_path(p, 1000) == abi.SG_GATHER_LOAD        # no context yet
    s = runtime.Scheduler(pool_bytes, pool=pool)
    try:
        T, L = abi.SG_GATHER_TEXTURE, abi.SG_GATHER_LOAD
        assert abi.sg_spmv_gather_path(p, 1000) == T
        assert abi.sg_spmv_gather_path(p + 512 * MiB - 8, 1000) == T     # across the first half mark
        assert abi.sg_spmv_gather_path(p + pool_bytes - 4000, 1000) == T  # ends at the pool's end
        assert abi.sg_spmv_gather_path(p + pool_bytes - 3996, 1000) == L  # one float past it
        assert abi.sg_spmv_gather_path(p, GiB // 4) == T                  # a whole window
        assert abi.sg_spmv_gather_path(p, GiB // 4 + 1) == L              # longer than any window
        assert abi.sg_spmv_gather_path(p + 600 * MiB, 150 * MiB) == T     # in the second window
        assert abi.sg_spmv_gather_path(p + 2, 10) == L                    # not float-aligned
        assert abi.sg_spmv_gather_path(outside.data_ptr(), 4096) == L     # not in any pool
    finally:
        s.shutdown()
    assert abi.sg_spmv_gather_path(p, 1000) == abi.SG_GATHER_LOAD        # windows gone with the context


def test_windows_of_two_contexts():
    """Each live context's pool has its own windows; shutting one context
    down leaves the other's."""
    abi, runtime = _mods()
    a = torch.empty(64 * MiB, dtype=torch.uint8, device="cuda")
    b = torch.empty(64 * MiB, dtype=torch.uint8, device="cuda")
    sa = runtime.Scheduler(64 * MiB, pool=a)
    sb = runtime.Scheduler(64 * MiB, pool=b)
    try:
        T, L = abi.SG_GATHER_TEXTURE, abi.SG_GATHER_LOAD
        assert abi.sg_spmv_gather_path(a.data_ptr() + 4096, 1000) == T
        assert abi.sg_spmv_gather_path(b.data_ptr() + 4096, 1000) == T
        sa.shutdown()
        assert abi.sg_spmv_gather_path(a.data_ptr() + 4096, 1000) == L
        assert abi.sg_spmv_gather_path(b.data_ptr() + 4096, 1000) == T
    finally:
        sa.shutdown()
        sb.shutdown()
    assert abi.sg_spmv_gather_path(b.data_ptr() + 4096, 1000) == abi.SG_GATHER_LOAD


def test_pool_without_texture_alignment_uses_loads():
    abi, runtime = _mods()
    big = torch.empty(64 * MiB + 512, dtype=torch.uint8, device="cuda")
    assert big.data_ptr() % 512 == 0
    pool = big[256:256 + 64 * MiB]                 # 256-byte aligned: a valid pool, no texture windows
    s = runtime.Scheduler(64 * MiB, pool=pool)
    try:
        assert abi.sg_spmv_gather_path(pool.data_ptr(), 1000) == abi.SG_GATHER_LOAD
    finally:
        s.shutdown()


def _gen_in(base_ptr, rows, lam, key):
    abi, _ = _mods()
    table = tg.poisson_cdf_table(lam)
    cap = tg.spmv_nnz_cap(rows, lam)
    lay = tg.spmv_layout(rows, cap)
    d_table = torch.from_numpy(table.view(np.int64).copy()).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert abi.sg_gen_spmv(base_ptr, rows, cap, d_table.data_ptr(), key, err.data_ptr()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return lay, table


@pytest.mark.parametrize("rows,lam,ptr64", [(1, 16.0, False), (7, 16.0, False), (1000, 8.0, False),
                                            (100003, 16.0, False), (1000003, 16.0, False),
                                            (100003, 16.0, True)])
def test_spmv_texture_equals_loads_and_oracle(rows, lam, ptr64):
    """x in the second window of a 1.25 GiB pool (texture) and a copy of the
    same arrays outside the pool (loads): equal y, and y against the oracle.
    ptr64 runs the int64 row-pointer kernel on the int32 matrix widened."""
    abi, runtime = _mods()
    key = 4242 + rows
    pool_bytes = GiB + GiB // 4
    pool = torch.zeros(pool_bytes, dtype=torch.uint8, device="cuda")
    s = runtime.Scheduler(pool_bytes, pool=pool)
    try:
        cap = tg.spmv_nnz_cap(rows, lam)
        total = tg.spmv_layout(rows, cap)["total"]
        off = (pool_bytes - total - 4096) // 256 * 256          # near the end: the second window
        bp = pool.data_ptr() + off
        lay, table = _gen_in(bp, rows, lam, key)
        assert not lay["ptr64"]
        ptr = bp + lay["row_ptr"]
        if ptr64:
            rp32 = pool[off + lay["row_ptr"]:off + lay["row_ptr"] + 4 * (rows + 1)].view(torch.int32)
            rp64 = rp32.to(torch.int64)        # outside the pool; row_ptr is read with loads either way
            ptr = rp64.data_ptr()
        assert abi.sg_spmv_gather_path(bp + lay["x"], rows) == abi.SG_GATHER_TEXTURE
        assert abi.sg_spmv(ptr, ptr64, bp + lay["col"], bp + lay["val"], bp + lay["x"], bp + lay["y"], rows) == 0
        torch.cuda.synchronize()
        y_tex = pool[off + lay["y"]:off + lay["y"] + 4 * rows].clone()
        copy = pool[off:off + lay["total"]].clone()            # a separate allocation: not in any pool
        cp = copy.data_ptr()
        assert abi.sg_spmv_gather_path(cp + lay["x"], rows) == abi.SG_GATHER_LOAD
        copy[lay["y"]:lay["y"] + 4 * rows].fill_(0xFF)
        if not ptr64:
            ptr = cp + lay["row_ptr"]
        assert abi.sg_spmv(ptr, ptr64, cp + lay["col"], cp + lay["val"], cp + lay["x"], cp + lay["y"], rows) == 0
        torch.cuda.synchronize()
        y_ld = copy[lay["y"]:lay["y"] + 4 * rows]
        assert torch.equal(y_tex, y_ld)
        gy = y_tex.view(torch.float32).cpu().numpy().astype(np.float64)
        if rows <= 100003:
            y, mag = K.spmv(key, rows, table)
            assert np.all(np.abs(gy - y) <= 1e-5 * mag + 1e-30)
        else:
            sample = np.unique(np.concatenate([[0, 1, rows - 1],
                                               np.random.default_rng(rows).integers(0, rows, 2000)]))
            y, mag, _ = K.spmv_sampled(key, rows, table, sample)
            assert np.all(np.abs(gy[sample] - y) <= 1e-5 * mag + 1e-30)
    finally:
        s.shutdown()


def test_gather_sum_texture_equals_loads():
    """The gather-rate measurement kernel takes the same path as the SpMV:
    its sums through the pool's window equal those through loads."""
    abi, runtime = _mods()
    rows, n = 300_000, 1_000_003
    rng = np.random.default_rng(5)
    col = torch.from_numpy(rng.integers(0, rows, n).astype(np.int32)).cuda()
    xs = torch.from_numpy(rng.uniform(-1, 1, rows).astype(np.float32)).cuda()
    pool = torch.zeros(16 * MiB, dtype=torch.uint8, device="cuda")
    s = runtime.Scheduler(16 * MiB, pool=pool)
    try:
        xin = pool[4096:4096 + 4 * rows].view(torch.float32)
        xin.copy_(xs)
        assert abi.sg_spmv_gather_path(xin.data_ptr(), rows) == abi.SG_GATHER_TEXTURE
        chunks = (n + 1023) // 1024
        o1 = torch.empty(chunks, dtype=torch.float32, device="cuda")
        o2 = torch.empty(chunks, dtype=torch.float32, device="cuda")
        assert abi.sg_gather_sum(col.data_ptr(), xin.data_ptr(), rows, n, o1.data_ptr()) == 0
        assert abi.sg_gather_sum(col.data_ptr(), xs.data_ptr(), rows, n, o2.data_ptr()) == 0
        torch.cuda.synchronize()
        assert torch.equal(o1.view(torch.int32), o2.view(torch.int32))
    finally:
        s.shutdown()


def test_spmv_captured_in_a_graph_uses_loads():
    """An SpMV captured into a CUDA graph must not hold a context's texture
    objects (they die with the context): on a capturing stream it gathers
    with loads. The replayed graph gives the same y as the texture path."""
    abi, runtime = _mods()
    rows, lam, key = 100_003, 16.0, 77
    cap = tg.spmv_nnz_cap(rows, lam)
    total = tg.spmv_layout(rows, cap)["total"]
    pool = torch.zeros(total + 4096, dtype=torch.uint8, device="cuda")
    s = runtime.Scheduler(total + 4096, pool=pool)
    try:
        bp = pool.data_ptr()
        lay, table = _gen_in(bp, rows, lam, key)
        assert abi.sg_spmv_gather_path(bp + lay["x"], rows) == abi.SG_GATHER_TEXTURE
        args = (bp + lay["row_ptr"], False, bp + lay["col"], bp + lay["val"], bp + lay["x"], bp + lay["y"], rows)
        assert abi.sg_spmv(*args) == 0
        torch.cuda.synchronize()
        y_tex = pool[lay["y"]:lay["y"] + 4 * rows].clone()
        pool[lay["y"]:lay["y"] + 4 * rows].fill_(0xFF)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            assert abi.sg_spmv(*args, torch.cuda.current_stream().cuda_stream) == 0
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(pool[lay["y"]:lay["y"] + 4 * rows], y_tex)
        y, mag = K.spmv(key, rows, table)
        gy = y_tex.view(torch.float32).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gy - y) <= 1e-5 * mag + 1e-30)
        del g
    finally:
        s.shutdown()
