"""Torch plumbing around the C ABI: device pool, streams, device copies of
traces and logs. PyTorch only provides memory and streams here; every
scheduling decision and every job's arithmetic runs in ``libschedgpu.so``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi
from . import tracegen as tg


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the co-scheduler has no CPU path)")


def to_device(arr: np.ndarray) -> torch.Tensor:
    """Byte copy of a numpy array in device memory."""
    _require_cuda()
    raw = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    return torch.from_numpy(raw.copy()).cuda()


def from_device(t: torch.Tensor, dtype, count: int) -> np.ndarray:
    return t.cpu().numpy().view(np.uint8)[: np.dtype(dtype).itemsize * count].view(dtype).copy()


def stream_handle(stream: torch.cuda.Stream | None = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def replay(jobs: np.ndarray, budget: int, policy, granule: int = 256, flags: int = 0,
           exclusive: bool = False):
    """Device replay of a trace (logical clock): (records, stats dict)."""
    _require_cuda()
    n = len(jobs)
    d_jobs = to_device(jobs)
    d_log = torch.empty(n * abi.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    ws = torch.empty(abi.sg_replay_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    d_stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = abi.sg_replay(d_jobs.data_ptr(), n, budget, granule, policy, flags, exclusive,
                       d_log.data_ptr(), ws.data_ptr(), d_stats.data_ptr(), stream_handle())
    if rc != abi.SG_OK:
        raise abi.SgError(rc, "sg_replay")
    torch.cuda.synchronize()
    st = d_stats.cpu().numpy().astype(np.uint64)
    return from_device(d_log, abi.RECORD_DTYPE, n), {
        "peak_used": int(st[0]), "frag_waits": int(st[1]), "passes": int(st[2]), "err": int(st[3])}


class Scheduler:
    """A context over one device pool (``sg_init`` .. ``sg_shutdown``)."""

    def __init__(self, pool_bytes: int, policy="first_fit", flags: int = 0, max_tickets: int = 0,
                 n_streams: int = 0, granule: int = 0, pool: torch.Tensor | None = None,
                 n_gemm_streams: int = 0, run_flags: int = 0, phase_jobs: int = 0):
        _require_cuda()
        self.pool = pool if pool is not None else torch.empty(pool_bytes, dtype=torch.uint8,
                                                              device="cuda")
        self.pool_bytes = pool_bytes
        self.ctx = abi.sg_init(self.pool.data_ptr(), pool_bytes, policy, flags, max_tickets,
                               n_streams, granule, n_gemm_streams, run_flags, phase_jobs)
        self._tables = None

    # -- life cycle
    def declare(self, need: int, priority: int = 0) -> int:
        return abi.sg_declare(self.ctx, need, priority)

    def try_grant(self, ticket: int):
        return abi.sg_try(self.ctx, ticket)

    def wait(self, ticket: int, timeout_ns: int):
        return abi.sg_wait(self.ctx, ticket, timeout_ns)

    def release(self, ticket: int, nbytes: int = 0, stream: torch.cuda.Stream | None = None) -> int:
        return abi.sg_release(self.ctx, ticket, nbytes, stream_handle(stream))

    def launch(self, ticket: int, job: np.ndarray, tables: torch.Tensor | None = None,
               stream: torch.cuda.Stream | None = None) -> int:
        tp = tables.data_ptr() if tables is not None else 0
        return abi.sg_launch(self.ctx, ticket, job, tp, stream_handle(stream))

    def reset(self):
        abi.sg_reset(self.ctx)

    def shutdown(self):
        if self.ctx:
            abi.sg_shutdown(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.shutdown()
        except Exception:
            pass

    # -- traces
    def run_trace(self, jobs, tables, mode: int = abi.SG_RUN_SATURATED, keep: bool = False):
        """Run a trace whose job records / tables are already device tensors.

        Returns (code, log tensor (device bytes), keep tensor or None, stats).
        """
        n = jobs.numel() // tg.JOB_DTYPE.itemsize
        log = torch.empty(n * abi.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        kp = torch.zeros(n, dtype=torch.int64, device="cuda") if keep else None
        if keep:
            mode |= abi.SG_RUN_KEEP
        rc, st = abi.sg_run_trace(self.ctx, jobs.data_ptr(), n, tables.data_ptr(), mode,
                                  log.data_ptr(), kp.data_ptr() if keep else 0)
        return rc, log, kp, st

    def run_trace_host(self, jobs: np.ndarray, tables, mode: int = abi.SG_RUN_SATURATED,
                       keep: bool = False):
        """The same through host buffers (copies inside the call)."""
        n = len(jobs)
        jobs = np.ascontiguousarray(jobs, dtype=tg.JOB_DTYPE)
        log = np.zeros(n, dtype=abi.RECORD_DTYPE)
        kp = np.zeros(n, dtype=np.uint64) if keep else None
        mode |= abi.SG_RUN_HOST_IO | (abi.SG_RUN_KEEP if keep else 0)
        rc, st = abi.sg_run_trace(self.ctx, jobs.ctypes.data, n, tables.data_ptr(), mode,
                                  log.ctypes.data, kp.ctypes.data if keep else 0)
        return rc, log, kp, st


def device_tables(trace: tg.Trace) -> torch.Tensor:
    return to_device(np.ascontiguousarray(trace.tables, dtype=np.uint64))


def records(log: torch.Tensor) -> np.ndarray:
    n = log.numel() // abi.RECORD_DTYPE.itemsize
    return from_device(log, abi.RECORD_DTYPE, n)


class Planned:
    """A batch admitted as a whole by the device engine (a replay plan), run
    either as one CUDA graph or by the persistent grouped kernel."""

    def __init__(self, pool: torch.Tensor, jobs: np.ndarray, tables: torch.Tensor, policy="first_fit",
                 keep: bool = False, budget: int | None = None, graph: bool = True, batch: bool = True):
        import time
        _require_cuda()
        self.pool = pool
        self.jobs = np.ascontiguousarray(jobs, dtype=tg.JOB_DTYPE)
        self.tables = tables
        self.budget = budget if budget is not None else pool.numel()
        t0 = time.perf_counter()
        self.plan, self.plan_stats = replay(self.jobs, self.budget, policy)
        t1 = time.perf_counter()
        self.keep = torch.zeros(len(jobs), dtype=torch.int64, device="cuda") if keep else None
        kp = self.keep.data_ptr() if keep else 0
        self.graph = (abi.sg_graph_build(pool.data_ptr(), self.budget, self.jobs, tables.data_ptr(), self.plan, kp)
                      if graph else 0)
        t2 = time.perf_counter()
        self.batch = (abi.sg_batch_build(pool.data_ptr(), self.budget, self.jobs, tables.data_ptr(), self.plan, kp)
                      if batch else 0)
        t3 = time.perf_counter()
        # host seconds: the engine's plan (device replay incl. copies), graph and batch builds
        self.build_s = {"replay": t1 - t0, "graph": t2 - t1, "batch": t3 - t2}

    def run_graph(self, stream: torch.cuda.Stream | None = None) -> int:
        if self.keep is not None:
            self.keep.zero_()
        return abi.sg_graph_launch(self.graph, stream_handle(stream))

    def run_batch(self, stream: torch.cuda.Stream | None = None) -> int:
        return abi.sg_batch_launch(self.batch, stream_handle(stream))

    def batch_status(self):
        return abi.sg_batch_status(self.batch)

    def close(self):
        if self.graph:
            abi.sg_graph_destroy(self.graph)
            self.graph = 0
        if self.batch:
            abi.sg_batch_destroy(self.batch)
            self.batch = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OnlineBatch:
    """A batch admitted on the device as it runs: the persistent grouped
    kernel holds the batch's engine, releases each finished job's memory and
    enqueues what the notification pass grants (no plan, no host step)."""

    def __init__(self, pool: torch.Tensor, jobs: np.ndarray, tables: torch.Tensor, policy="first_fit",
                 keep: bool = False, budget: int | None = None):
        _require_cuda()
        self.pool = pool
        self.jobs = np.ascontiguousarray(jobs, dtype=tg.JOB_DTYPE)
        self.tables = tables
        self.budget = budget if budget is not None else pool.numel()
        self.keep = torch.zeros(len(jobs), dtype=torch.int64, device="cuda") if keep else None
        kp = self.keep.data_ptr() if keep else 0
        self.batch = abi.sg_batch_build_online(pool.data_ptr(), self.budget, self.jobs, tables.data_ptr(), policy, kp)

    def run(self, stream: torch.cuda.Stream | None = None) -> int:
        return abi.sg_batch_launch(self.batch, stream_handle(stream))

    def status(self):
        return abi.sg_batch_status(self.batch)

    def records(self) -> np.ndarray:
        return abi.sg_batch_records(self.batch, len(self.jobs))

    def close(self):
        if self.batch:
            abi.sg_batch_destroy(self.batch)
            self.batch = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

