"""ctypes binding of ``libschedgpu.so``: the C ABI of ``include/schedgpu.h``
under the same names, argument marshalling only.

Every step of the co-scheduler runs in the library's CUDA kernels; nothing
here computes, schedules or falls back to the CPU. Loading fails loudly if
the library is missing (build it with ``paper_1712_04495_b300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import tracegen as _tg

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libschedgpu.so")

SG_OK, SG_NOT_READY, SG_ERR_TIMEOUT, SG_ERR_TOO_LARGE, SG_ERR_INVALID, SG_ERR_CUDA, \
    SG_ERR_UNKNOWN, SG_ERR_CAPACITY, SG_ERR_DEVICE = range(9)
SG_POLICY_FIFO, SG_POLICY_FIRST_FIT, SG_POLICY_PRIO_FIFO, SG_POLICY_PRIO_FIRST_FIT = range(4)
POLICIES = {"fifo": 0, "first_fit": 1, "mmu": 1, "prio_fifo": 2, "prio_first_fit": 3, "prio_mmu": 3}
SG_FLAG_FIFO_BYPASS = 1
SG_DEVERR_WAIT, SG_DEVERR_STATE, SG_DEVERR_ORDER, SG_DEVERR_EVENTS, SG_DEVERR_NNZ, \
    SG_DEVERR_CAPACITY, SG_DEVERR_ITEM = 1, 2, 4, 8, 16, 32, 64
SG_ST_PENDING, SG_ST_QUEUED, SG_ST_RUNNING, SG_ST_DONE, SG_ST_TIMEOUT, SG_ST_TOO_LARGE = range(6)
SG_RUN_SATURATED, SG_RUN_TIMED, SG_RUN_EXCLUSIVE, SG_RUN_HOST_IO, SG_RUN_KEEP = 1, 2, 4, 8, 16
SG_RUNF_OVERLAP = 1

JOB_DTYPE = _tg.JOB_DTYPE
RECORD_DTYPE = np.dtype([("status", "<i4"), ("slot", "<i4"), ("grant_seq", "<i8"),
                         ("grant_t", "<u8"), ("offset", "<u8"), ("done_t", "<u8"),
                         ("arrival_t", "<u8")])
assert RECORD_DTYPE.itemsize == 48


class SgConfig(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("max_tickets", ctypes.c_uint32), ("n_streams", ctypes.c_uint32),
                ("granule", ctypes.c_uint64), ("n_gemm_streams", ctypes.c_uint32),
                ("run_flags", ctypes.c_uint16), ("phase_jobs", ctypes.c_uint16)]


class SgGrant(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_uint64), ("ptr", ctypes.c_void_p),
                ("grant_time_ns", ctypes.c_uint64)]


class SgRunStats(ctypes.Structure):
    _fields_ = [("elapsed_ns", ctypes.c_uint64), ("makespan_ns", ctypes.c_uint64),
                ("wait_p50_ns", ctypes.c_uint64), ("wait_p99_ns", ctypes.c_uint64),
                ("turnaround_p50_ns", ctypes.c_uint64), ("turnaround_p99_ns", ctypes.c_uint64),
                ("peak_used", ctypes.c_uint64), ("frag_waits", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("jobs_done", ctypes.c_uint32), ("jobs_failed", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SgStateSummary(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_uint64), ("used", ctypes.c_uint64), ("peak_used", ctypes.c_uint64),
                ("max_free_extent", ctypes.c_uint64), ("grants", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("frag_waits", ctypes.c_uint64), ("policy", ctypes.c_uint32), ("free_extents", ctypes.c_uint32),
                ("waiting", ctypes.c_uint32), ("done", ctypes.c_uint32), ("error_flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class SgServerCounts(ctypes.Structure):
    _fields_ = [("clients_accepted", ctypes.c_uint64), ("clients_reaped", ctypes.c_uint64),
                ("declares", ctypes.c_uint64), ("grants", ctypes.c_uint64), ("timeouts", ctypes.c_uint64),
                ("releases", ctypes.c_uint64), ("protocol_errors", ctypes.c_uint64),
                ("clients_open", ctypes.c_uint32), ("tickets_open", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SgShmCounts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("budget", "granule", "used", "peak_used", "grants", "passes", "frag_waits", "reaped",
                 "rebuilt", "restored", "reset", "abandoned", "timeouts", "backups", "generation")] + \
               [(k, ctypes.c_uint32) for k in
                ("policy", "max_tickets", "waiting", "running", "free_extents", "reserved")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


SG_SHM_BAD_HEADER, SG_SHM_BAD_TICKETS, SG_SHM_BAD_USED, SG_SHM_BAD_EXTENTS, SG_SHM_BAD_QUEUE, \
    SG_SHM_BAD_SLOTS, SG_SHM_DIRTY = 1, 2, 4, 8, 16, 32, 64

NO_TIMEOUT = (1 << 64) - 1


class SgError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {sg_strerror(code)} (code {code})")
        self.code = code


_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_I32 = ctypes.c_int32

_SIGS = {
    "sg_init": ([ctypes.POINTER(_P), _P, _U64, ctypes.POINTER(SgConfig)], ctypes.c_int),
    "sg_shutdown": ([_P], ctypes.c_int),
    "sg_reset": ([_P], ctypes.c_int),
    "sg_declare": ([_P, _U64, _I32, ctypes.POINTER(_U32)], ctypes.c_int),
    "sg_try": ([_P, _U32, ctypes.POINTER(SgGrant)], ctypes.c_int),
    "sg_wait": ([_P, _U32, _U64, ctypes.POINTER(SgGrant)], ctypes.c_int),
    "sg_release": ([_P, _U32, _U64, _P], ctypes.c_int),
    "sg_launch": ([_P, _U32, _P, _P, _P], ctypes.c_int),
    "sg_run_trace": ([_P, _P, _U32, _P, _U32, _P, _P, ctypes.POINTER(SgRunStats)], ctypes.c_int),
    "sg_replay_workspace_bytes": ([_U32], _U64),
    "sg_replay": ([_P, _U32, _U64, _U64, _U32, _U32, _U32, _P, _P, _P, _P], ctypes.c_int),
    "sg_replay_noalloc": ([_P, _U32, _U64, _U64, _U32, _U32, _U32, _P, _P, _P], ctypes.c_int),
    "sg_graph_build": ([_P, _U64, _P, _U32, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sg_graph_launch": ([_P, _P], ctypes.c_int),
    "sg_graph_info": ([_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)], ctypes.c_int),
    "sg_graph_destroy": ([_P], ctypes.c_int),
    "sg_batch_build": ([_P, _U64, _P, _U32, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sg_batch_launch": ([_P, _P], ctypes.c_int),
    "sg_batch_status": ([_P, ctypes.POINTER(_U64), ctypes.POINTER(_U32)], ctypes.c_int),
    "sg_batch_info": ([_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)], ctypes.c_int),
    "sg_batch_destroy": ([_P], ctypes.c_int),
    "sg_kernel_errors": ([ctypes.POINTER(_U32)], ctypes.c_int),
    "sg_device_error": ([_P], _U32),
    "sg_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "sg_triad": ([_P, _P, _P, ctypes.c_float, _U64, _P], ctypes.c_int),
    "sg_gen_triad": ([_P, _P, _U64, _U64, _P], ctypes.c_int),
    "sg_spmv": ([_P, ctypes.c_int, _P, _P, _P, _P, _U64, _P], ctypes.c_int),
    "sg_gen_spmv": ([_P, _U64, _U64, _P, _U64, _P, _P], ctypes.c_int),
    "sg_gemm_bf16": ([_P, _P, _P, _U32, _U32, _U32, _P], ctypes.c_int),
    "sg_gemm_bf16_tiled": ([_P, _P, _P, _U32, _U32, _U32, _U32, _P], ctypes.c_int),
    "sg_gemm_tile": ([_U32, _U32], _U32),
    "sg_autotune_gemm": ([_P, _U32, _P, _U64, _P, _P, _P], ctypes.c_int),
    "sg_autotune_clear": ([], ctypes.c_int),
    "sg_gen_gemm": ([_P, _P, _U32, _U32, _U32, _U64, _P], ctypes.c_int),
    "sg_digest": ([_P, _U64, _P, _P], ctypes.c_int),
    "sg_gather_sum": ([_P, _P, _U64, _U64, _P, _P], ctypes.c_int),
    "sg_spmv_gather_path": ([_P, _U64], ctypes.c_int),
    "sg_cancel": ([_P, _U32, _P], ctypes.c_int),
    "sg_poll_grants": ([_P, _P, _P, _U32, _P], ctypes.c_int),
    "sg_server_start": ([_P, ctypes.c_char_p, _P], ctypes.c_int),
    "sg_server_counters": ([_P, _P], ctypes.c_int),
    "sg_server_stop": ([_P], ctypes.c_int),
    "sg_client_connect": ([ctypes.c_char_p, _P], ctypes.c_int),
    "sg_client_info": ([_P, _P, _P], ctypes.c_int),
    "sg_client_pool": ([_P, _P], ctypes.c_int),
    "sg_client_declare": ([_P, _U64, ctypes.c_int32, _U64, _P], ctypes.c_int),
    "sg_client_try": ([_P, _U32, _P], ctypes.c_int),
    "sg_client_wait": ([_P, _U32, _U64, _P], ctypes.c_int),
    "sg_client_release": ([_P, _U32, _U64], ctypes.c_int),
    "sg_client_close": ([_P], ctypes.c_int),
    "sg_state": ([_P, _P], ctypes.c_int),
    "sg_batch_build_online": ([_P, _U64, _P, _U32, _P, _U32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sg_batch_records": ([_P, _P], ctypes.c_int),
    "sg_shm_open": ([ctypes.c_char_p, _U64, _U32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sg_shm_declare": ([_P, _U64, ctypes.c_int32, ctypes.POINTER(_U32)], ctypes.c_int),
    "sg_shm_try": ([_P, _U32, _P], ctypes.c_int),
    "sg_shm_wait": ([_P, _U32, _U64, _P], ctypes.c_int),
    "sg_shm_release": ([_P, _U32, _U64], ctypes.c_int),
    "sg_shm_record": ([_P, _U32, _P], ctypes.c_int),
    "sg_shm_stats": ([_P, _P], ctypes.c_int),
    "sg_shm_used_by": ([_P, ctypes.c_int32, ctypes.POINTER(_U64)], ctypes.c_int),
    "sg_shm_check": ([_P, ctypes.POINTER(_U32)], ctypes.c_int),
    "sg_shm_set_pool": ([_P, _P, _U64], ctypes.c_int),
    "sg_shm_pool": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "sg_shm_close": ([_P], ctypes.c_int),
    "sg_shm_unlink": ([ctypes.c_char_p], ctypes.c_int),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1712_04495_b300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, what: str, ok=(SG_OK,)):
    if rc not in ok:
        raise SgError(rc, what)
    return rc


def sg_strerror(code: int) -> str:
    return lib().sg_strerror(code).decode()


# ------------------------------------------------------------- life cycle
def sg_init(pool_ptr: int, pool_bytes: int, policy=0, flags=0, max_tickets=0, n_streams=0,
            granule=0, n_gemm_streams=0, run_flags=0, phase_jobs=0) -> int:
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    cfg = SgConfig(pol, flags, max_tickets, n_streams, granule, n_gemm_streams, run_flags, phase_jobs)
    out = _P()
    _check(lib().sg_init(ctypes.byref(out), pool_ptr, pool_bytes, ctypes.byref(cfg)), "sg_init")
    return out.value


def sg_shutdown(ctx: int):
    _check(lib().sg_shutdown(ctx), "sg_shutdown")


def sg_reset(ctx: int):
    _check(lib().sg_reset(ctx), "sg_reset")


def sg_declare(ctx: int, need: int, priority: int = 0) -> int:
    t = _U32()
    _check(lib().sg_declare(ctx, need, priority, ctypes.byref(t)), "sg_declare")
    return t.value


def sg_try(ctx: int, ticket: int):
    """(code, grant or None): SG_OK, SG_NOT_READY, SG_ERR_TIMEOUT, ..."""
    g = SgGrant()
    rc = lib().sg_try(ctx, ticket, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_wait(ctx: int, ticket: int, timeout_ns: int):
    g = SgGrant()
    rc = lib().sg_wait(ctx, ticket, timeout_ns, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_release(ctx: int, ticket: int, nbytes: int = 0, stream: int = 0) -> int:
    return lib().sg_release(ctx, ticket, nbytes, stream)


def sg_state(ctx: int) -> dict:
    """Post-mortem summary of the device engine's scalar state."""
    st = SgStateSummary()
    _check(lib().sg_state(ctx, ctypes.byref(st)), "sg_state")
    return st.as_dict()


def sg_cancel(ctx: int, ticket: int):
    """(code, grant or None): SG_ERR_TIMEOUT if withdrawn, SG_OK if it was granted first."""
    g = SgGrant()
    rc = lib().sg_cancel(ctx, ticket, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_poll_grants(ctx: int, cursor: int, max_n: int = 1024):
    """(code, new cursor, tickets granted since `cursor`)."""
    cur = _U32(cursor)
    out = np.zeros(max(1, max_n), dtype=np.uint32)
    n = _U32()
    rc = lib().sg_poll_grants(ctx, ctypes.byref(cur), out.ctypes.data, max_n, ctypes.byref(n))
    return rc, cur.value, [int(x) for x in out[: n.value]]


# ---------------------------------------------------- server and clients
def sg_server_start(ctx: int, socket_path: str) -> int:
    out = _P()
    _check(lib().sg_server_start(ctx, socket_path.encode(), ctypes.byref(out)), "sg_server_start")
    return out.value


def sg_server_counters(srv: int) -> dict:
    c = SgServerCounts()
    _check(lib().sg_server_counters(srv, ctypes.byref(c)), "sg_server_counters")
    return c.as_dict()


def sg_server_stop(srv: int):
    _check(lib().sg_server_stop(srv), "sg_server_stop")


def sg_client_connect(socket_path: str) -> int:
    out = _P()
    _check(lib().sg_client_connect(socket_path.encode(), ctypes.byref(out)), "sg_client_connect")
    return out.value


def sg_client_info(cl: int):
    pb, gr = _U64(), _U64()
    _check(lib().sg_client_info(cl, ctypes.byref(pb), ctypes.byref(gr)), "sg_client_info")
    return pb.value, gr.value


def sg_client_pool(cl: int) -> int:
    p = _P()
    _check(lib().sg_client_pool(cl, ctypes.byref(p)), "sg_client_pool")
    return p.value


def sg_client_declare(cl: int, need: int, priority: int = 0, timeout_ns: int = NO_TIMEOUT) -> int:
    t = _U32()
    _check(lib().sg_client_declare(cl, need, priority, timeout_ns, ctypes.byref(t)), "sg_client_declare")
    return t.value


def sg_client_try(cl: int, ticket: int):
    g = SgGrant()
    rc = lib().sg_client_try(cl, ticket, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_client_wait(cl: int, ticket: int, max_block_ns: int):
    g = SgGrant()
    rc = lib().sg_client_wait(cl, ticket, max_block_ns, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_client_release(cl: int, ticket: int, nbytes: int = 0) -> int:
    return lib().sg_client_release(cl, ticket, nbytes)


def sg_client_close(cl: int):
    _check(lib().sg_client_close(cl), "sg_client_close")


def sg_launch(ctx: int, ticket: int, job: np.ndarray, tables_ptr: int = 0, stream: int = 0) -> int:
    job = np.ascontiguousarray(job, dtype=JOB_DTYPE).reshape(1)
    return lib().sg_launch(ctx, ticket, job.ctypes.data, tables_ptr or None, stream)


def sg_run_trace(ctx: int, jobs_ptr: int, n: int, tables_ptr: int, mode: int, log_ptr: int,
                 keep_ptr: int = 0):
    st = SgRunStats()
    rc = lib().sg_run_trace(ctx, jobs_ptr, n, tables_ptr or None, mode, log_ptr or None,
                            keep_ptr or None, ctypes.byref(st))
    return rc, st.as_dict()


def sg_replay_workspace_bytes(n: int) -> int:
    return lib().sg_replay_workspace_bytes(n)


def sg_replay(jobs_ptr: int, n: int, budget: int, granule: int, policy, flags: int, exclusive: bool,
              log_ptr: int, ws_ptr: int, stats_ptr: int = 0, stream: int = 0) -> int:
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    return lib().sg_replay(jobs_ptr, n, budget, granule, pol, flags, int(bool(exclusive)), log_ptr,
                           ws_ptr, stats_ptr or None, stream)


SG_REPLAY_NOALLOC_MAX_JOBS = 16384


def sg_replay_noalloc(jobs_ptr: int, n: int, budget: int, granule: int, policy, flags: int,
                      exclusive: bool, log_ptr: int, stats_ptr: int = 0, stream: int = 0) -> int:
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    return lib().sg_replay_noalloc(jobs_ptr, n, budget, granule, pol, flags, int(bool(exclusive)),
                                   log_ptr, stats_ptr or None, stream)


def sg_graph_build(pool_ptr: int, pool_bytes: int, jobs: np.ndarray, tables_ptr: int, plan: np.ndarray,
                   keep_ptr: int = 0) -> int:
    jobs = np.ascontiguousarray(jobs, dtype=JOB_DTYPE)
    plan = np.ascontiguousarray(plan, dtype=RECORD_DTYPE)
    out = _P()
    _check(lib().sg_graph_build(pool_ptr, pool_bytes, jobs.ctypes.data, len(jobs), tables_ptr or None,
                                plan.ctypes.data, keep_ptr or None, ctypes.byref(out)), "sg_graph_build")
    return out.value


def sg_graph_launch(g: int, stream: int = 0) -> int:
    return lib().sg_graph_launch(g, stream)


def sg_graph_info(g: int):
    a, b, c = _U64(), _U64(), _U64()
    _check(lib().sg_graph_info(g, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sg_graph_info")
    return {"jobs": a.value, "kernels": b.value, "edges": c.value}


def sg_graph_destroy(g: int):
    _check(lib().sg_graph_destroy(g), "sg_graph_destroy")


def sg_batch_build(pool_ptr: int, pool_bytes: int, jobs: np.ndarray, tables_ptr: int, plan: np.ndarray,
                   keep_ptr: int = 0) -> int:
    jobs = np.ascontiguousarray(jobs, dtype=JOB_DTYPE)
    plan = np.ascontiguousarray(plan, dtype=RECORD_DTYPE)
    out = _P()
    _check(lib().sg_batch_build(pool_ptr, pool_bytes, jobs.ctypes.data, len(jobs), tables_ptr or None,
                                plan.ctypes.data, keep_ptr or None, ctypes.byref(out)), "sg_batch_build")
    return out.value


def sg_batch_build_online(pool_ptr: int, pool_bytes: int, jobs: np.ndarray, tables_ptr: int, policy,
                          keep_ptr: int = 0) -> int:
    jobs = np.ascontiguousarray(jobs, dtype=JOB_DTYPE)
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    out = _P()
    _check(lib().sg_batch_build_online(pool_ptr, pool_bytes, jobs.ctypes.data, len(jobs), tables_ptr or None, pol,
                                       keep_ptr or None, ctypes.byref(out)), "sg_batch_build_online")
    return out.value


def sg_batch_records(b: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=RECORD_DTYPE)
    _check(lib().sg_batch_records(b, out.ctypes.data), "sg_batch_records")
    return out


def sg_batch_launch(b: int, stream: int = 0) -> int:
    return lib().sg_batch_launch(b, stream)


def sg_batch_status(b: int):
    d, e = _U64(), _U32()
    rc = lib().sg_batch_status(b, ctypes.byref(d), ctypes.byref(e))
    return rc, d.value, e.value


def sg_batch_info(b: int):
    a, c, k = _U64(), _U64(), _U64()
    _check(lib().sg_batch_info(b, ctypes.byref(a), ctypes.byref(c), ctypes.byref(k)), "sg_batch_info")
    return {"jobs": a.value, "chunks": c.value, "blocks": k.value}


def sg_batch_destroy(b: int):
    _check(lib().sg_batch_destroy(b), "sg_batch_destroy")


def sg_kernel_errors() -> int:
    v = _U32()
    _check(lib().sg_kernel_errors(ctypes.byref(v)), "sg_kernel_errors")
    return v.value


def sg_device_error(ctx: int) -> int:
    return lib().sg_device_error(ctx)


# ----------------------------------------------------------------- kernels
def sg_triad(a, b, c, s: float, n: int, stream: int = 0) -> int:
    return lib().sg_triad(a, b, c, s, n, stream)


def sg_gen_triad(b, c, n: int, key: int, stream: int = 0) -> int:
    return lib().sg_gen_triad(b, c, n, key, stream)


def sg_spmv(row_ptr, ptr64: bool, col, val, x, y, rows: int, stream: int = 0) -> int:
    return lib().sg_spmv(row_ptr, int(ptr64), col, val, x, y, rows, stream)


def sg_gen_spmv(base, rows: int, nnz: int, table_ptr, key: int, err_ptr=0, stream: int = 0) -> int:
    return lib().sg_gen_spmv(base, rows, nnz, table_ptr, key, err_ptr or None, stream)


def sg_gemm_bf16(A, Bt, C, M: int, N: int, K: int, stream: int = 0) -> int:
    return lib().sg_gemm_bf16(A, Bt, C, M, N, K, stream)


def gemm_tile(m: int, n: int) -> int:
    """Tile code of an m x n output tile (SG_GEMM_TILE)."""
    return (m << 16) | n


def gemm_tile_name(code: int) -> str:
    if 0 < code < 65536:
        code = gemm_tile(128, code)
    return f"{code >> 16}x{code & 0xFFFF}"


GEMM_TILES = (gemm_tile(128, 64), gemm_tile(128, 128), gemm_tile(128, 256), gemm_tile(256, 256))


def sg_gemm_bf16_tiled(A, Bt, C, M: int, N: int, K: int, tile: int, stream: int = 0) -> int:
    return lib().sg_gemm_bf16_tiled(A, Bt, C, M, N, K, tile, stream)


def sg_gemm_tile(M: int, N: int) -> int:
    return lib().sg_gemm_tile(M, N)


def sg_autotune_gemm(shapes, scratch_ptr: int, scratch_bytes: int, stream: int = 0):
    """Tune the output tile of each (M, N, K); returns [(shape, tile code, ms)]."""
    arr = np.ascontiguousarray(np.asarray(shapes, dtype=np.uint32).reshape(-1, 3))
    n = len(arr)
    chosen = np.zeros(n, dtype=np.uint32)
    best = np.zeros(n, dtype=np.float32)
    _check(lib().sg_autotune_gemm(arr.ctypes.data, n, scratch_ptr, scratch_bytes, chosen.ctypes.data,
                                  best.ctypes.data, stream), "sg_autotune_gemm")
    return [(tuple(int(x) for x in arr[i]), int(chosen[i]), float(best[i])) for i in range(n)]


def sg_autotune_clear():
    _check(lib().sg_autotune_clear(), "sg_autotune_clear")


def sg_gen_gemm(A, Bt, M: int, N: int, K: int, key: int, stream: int = 0) -> int:
    return lib().sg_gen_gemm(A, Bt, M, N, K, key, stream)


def sg_digest(ptr, words: int, out_ptr, stream: int = 0) -> int:
    return lib().sg_digest(ptr, words, out_ptr, stream)


SG_GATHER_LOAD, SG_GATHER_TEXTURE = 0, 1


def sg_spmv_gather_path(x, rows: int) -> int:
    """SG_GATHER_TEXTURE when x (rows floats) lies in a texture window of a
    live context's pool, else SG_GATHER_LOAD."""
    return lib().sg_spmv_gather_path(x, rows)


def sg_gather_sum(col, x, x_len: int, n: int, out_ptr, stream: int = 0) -> int:
    return lib().sg_gather_sum(col, x, x_len, n, out_ptr, stream)


# ------------------------------------------------ shared memory (no server)
def sg_shm_open(name: str, budget: int = 0, policy="first_fit", max_tickets: int = 0, granule: int = 0,
                flags: int = 0) -> int:
    """Create (budget > 0) or attach to (budget 0) the shared segment `name`."""
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    cfg = SgConfig(policy=pol, flags=flags, max_tickets=max_tickets, granule=granule)
    out = _P()
    _check(lib().sg_shm_open(name.encode(), budget, pol, ctypes.byref(cfg), ctypes.byref(out)), "sg_shm_open")
    return out.value


def sg_shm_declare(h: int, need: int, priority: int = 0):
    """(rc, ticket): rc is SG_OK or the refusal (SG_ERR_TOO_LARGE, ...)."""
    t = _U32()
    rc = lib().sg_shm_declare(h, need, priority, ctypes.byref(t))
    return rc, (t.value if rc == SG_OK else None)


def sg_shm_try(h: int, ticket: int):
    g = SgGrant()
    rc = lib().sg_shm_try(h, ticket, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_shm_wait(h: int, ticket: int, timeout_ns: int = NO_TIMEOUT):
    g = SgGrant()
    rc = lib().sg_shm_wait(h, ticket, timeout_ns, ctypes.byref(g))
    return rc, (g if rc == SG_OK else None)


def sg_shm_release(h: int, ticket: int, nbytes: int = 0) -> int:
    return lib().sg_shm_release(h, ticket, nbytes)


def sg_shm_record(h: int, ticket: int):
    """(rc, record): record is a RECORD_DTYPE scalar while the ticket lives."""
    r = np.zeros(1, dtype=RECORD_DTYPE)
    rc = lib().sg_shm_record(h, ticket, r.ctypes.data_as(_P))
    return rc, (r[0] if rc == SG_OK else None)


def sg_shm_stats(h: int) -> dict:
    c = SgShmCounts()
    _check(lib().sg_shm_stats(h, ctypes.byref(c)), "sg_shm_stats")
    return c.as_dict()


def sg_shm_used_by(h: int, pid: int) -> int:
    b = _U64()
    _check(lib().sg_shm_used_by(h, pid, ctypes.byref(b)), "sg_shm_used_by")
    return b.value


def sg_shm_check(h: int) -> int:
    """Integrity check (and recovery); the SG_SHM_* problems found."""
    p = _U32()
    _check(lib().sg_shm_check(h, ctypes.byref(p)), "sg_shm_check")
    return p.value


def sg_shm_set_pool(h: int, dev_ptr: int, pool_bytes: int):
    _check(lib().sg_shm_set_pool(h, dev_ptr, pool_bytes), "sg_shm_set_pool")


def sg_shm_pool(h: int) -> int:
    p = _P()
    _check(lib().sg_shm_pool(h, ctypes.byref(p)), "sg_shm_pool")
    return p.value


def sg_shm_close(h: int):
    _check(lib().sg_shm_close(h), "sg_shm_close")


def sg_shm_unlink(name: str) -> int:
    return lib().sg_shm_unlink(name.encode())
