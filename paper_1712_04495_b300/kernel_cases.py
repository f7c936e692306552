"""Run one job kernel on its own, for profiling and timing.

    python -m paper_1712_04495_b300.kernel_cases gemm  [M=N=K, default 8192] [launches] [tile, e.g. 256x256]
    python -m paper_1712_04495_b300.kernel_cases spmv  [rows, default 1e7]   [launches]
    python -m paper_1712_04495_b300.kernel_cases triad [n, default 64M]      [launches]
    python -m paper_1712_04495_b300.kernel_cases fill  [rows, default 1e7]   [launches]
    python -m paper_1712_04495_b300.kernel_cases gather [rows, default 1e7]  [launches]
    python -m paper_1712_04495_b300.kernel_cases batch [jobs, default 10000] [launches]
    python -m paper_1712_04495_b300.kernel_cases replay [jobs, default 10000] [launches] [policy]

`gather` times the gather-rate measurement kernel (sg_gather_sum) on the
generated SpMV matrix's own columns and x, after one SpMV launch.
`batch` runs the tiny-job trace (10,000 jobs, 2 GiB pool) through the
persistent grouped kernel on the device engine's replay plan. `replay` runs
the device engine's replay (one warp, logical clock) of the same trace.

The inputs are built by the library's own generators first (one launch per
generator kernel), then the kernel runs `launches` times (default 3) on the
current stream. Prints the CUDA-event time per launch. The SpMV cases place
the matrix in the grant of a scheduler pool, where an SpMV job's matrix is.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from . import abi
from . import tracegen as tg


def _time(fn, launches: int) -> float:
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(launches):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / launches


def run(kind: str, size: int | None = None, launches: int = 3, tile: str | None = None) -> dict:
    st = torch.cuda.current_stream().cuda_stream
    if kind == "gemm":
        m = size or 8192
        A = torch.empty(m * m, dtype=torch.int16, device="cuda")
        B = torch.empty(m * m, dtype=torch.int16, device="cuda")
        C = torch.empty(m * m, dtype=torch.float32, device="cuda")
        assert abi.sg_gen_gemm(A.data_ptr(), B.data_ptr(), m, m, m, 42, st) == 0
        code = abi.gemm_tile(*(int(x) for x in tile.split("x"))) if tile else abi.sg_gemm_tile(m, m)
        ms = _time(lambda: abi.sg_gemm_bf16_tiled(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, m, m, code, st),
                   launches)
        return {"kernel": "gemm", "tile": abi.gemm_tile_name(code), "size": m, "ms": ms,
                "tflops": 2.0 * m ** 3 / (ms * 1e-3) / 1e12}
    if kind in ("spmv", "fill", "gather"):
        rows = size or 10_000_000
        lam = 16.0
        cap = tg.spmv_nnz_cap(rows, lam)
        lay = tg.spmv_layout(rows, cap)
        base = torch.empty(lay["total"], dtype=torch.uint8, device="cuda")
        tab = torch.from_numpy(tg.poisson_cdf_table(lam).view(np.int64).copy()).cuda()
        # the matrix in the grant of a scheduler pool, as an SpMV job's is
        # (x is then gathered through the pool's texture window)
        from . import runtime
        sched = runtime.Scheduler(lay["total"], pool=base)
        try:
            t = sched.declare(lay["total"])
            rc, grant = sched.wait(t, 10 ** 9)
            assert rc == abi.SG_OK, rc
            p = base.data_ptr() + grant.offset
            path = "texture" if abi.sg_spmv_gather_path(p + lay["x"], rows) == abi.SG_GATHER_TEXTURE else "loads"
            gen = lambda: abi.sg_gen_spmv(p, rows, cap, tab.data_ptr(), 5, 0, st)  # noqa: E731
            gen()
            torch.cuda.synchronize()
            if kind == "fill":
                ms = _time(gen, launches)
                return {"kernel": "spmv generator", "rows": rows, "ms": ms}
            ptr_t = torch.int64 if lay["ptr64"] else torch.int32
            esz = 8 if lay["ptr64"] else 4
            nnz = int(base[lay["row_ptr"] + esz * rows:lay["row_ptr"] + esz * (rows + 1)].view(ptr_t).item())
            if kind == "gather":
                assert abi.sg_spmv(p + lay["row_ptr"], lay["ptr64"], p + lay["col"], p + lay["val"],
                                   p + lay["x"], p + lay["y"], rows, st) == 0
                out = torch.empty((nnz + 1023) // 1024, dtype=torch.float32, device="cuda")
                ms = _time(lambda: abi.sg_gather_sum(p + lay["col"], p + lay["x"], rows, nnz, out.data_ptr(), st),
                           launches)
                return {"kernel": "gather", "rows": rows, "nnz": nnz, "ms": ms, "x_gathers": path,
                        "gathers_per_s": nnz / (ms * 1e-3)}
            ms = _time(lambda: abi.sg_spmv(p + lay["row_ptr"], lay["ptr64"], p + lay["col"], p + lay["val"],
                                           p + lay["x"], p + lay["y"], rows, st), launches)
            alg = esz * (rows + 1) + 8 * nnz + 8 * rows
            return {"kernel": "spmv", "rows": rows, "nnz": nnz, "ms": ms, "alg_bytes": alg, "x_gathers": path,
                    "gbs": alg / (ms * 1e-3) / 1e9}
        finally:
            torch.cuda.synchronize()
            sched.shutdown()
    if kind == "triad":
        n = size or (64 << 20)
        buf = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        a, b, c = buf[:n], buf[n:2 * n], buf[2 * n:]
        assert abi.sg_gen_triad(b.data_ptr(), c.data_ptr(), n, 7, st) == 0
        ms = _time(lambda: abi.sg_triad(a.data_ptr(), b.data_ptr(), c.data_ptr(), 3.0, n, st), launches)
        return {"kernel": "triad", "n": n, "ms": ms, "gbs": 12.0 * n / (ms * 1e-3) / 1e9}
    if kind == "batch":
        from . import runtime
        tr = tg.trace_c4(n_jobs=size or 10_000)
        pool = torch.empty(tr.budget, dtype=torch.uint8, device="cuda")
        pl = runtime.Planned(pool, tr.jobs, runtime.device_tables(tr), "first_fit", budget=tr.budget)
        ms = _time(lambda: pl.run_batch(), launches)
        rc, done, err = pl.batch_status()
        info = abi.sg_batch_info(pl.batch)
        pl.close()
        return {"kernel": "batch", "jobs": len(tr), "ms": ms, "done": done, "err": err, **info}
    if kind == "replay":
        from . import runtime
        tr = tg.trace_c4(n_jobs=size or 10_000)
        pol = tile or "first_fit"
        n = len(tr)
        d_jobs = runtime.to_device(tr.jobs)
        d_log = torch.empty(n * abi.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        ws = torch.empty(abi.sg_replay_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        stats = torch.zeros(4, dtype=torch.int64, device="cuda")
        ms = _time(lambda: abi.sg_replay(d_jobs.data_ptr(), n, tr.budget, 256, pol, 0, False, d_log.data_ptr(),
                                         ws.data_ptr(), stats.data_ptr(), st), launches)
        return {"kernel": "replay", "policy": pol, "jobs": n, "ms": ms, "us_per_event": 1e3 * ms / (2 * n),
                "stats": stats.cpu().tolist()}
    raise ValueError(kind)


if __name__ == "__main__":
    k = sys.argv[1]
    size = int(float(sys.argv[2])) if len(sys.argv) > 2 else None
    launches = int(sys.argv[3]) if len(sys.argv) > 3 else 3
    print(run(k, size, launches, sys.argv[4] if len(sys.argv) > 4 else None))
