"""ctypes front of the C discrete-event simulator (``des.c``): whole traces
(``simulate``) and sequences of life-cycle calls (``simulate_ops``)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

ST_PENDING, ST_QUEUED, ST_RUNNING, ST_DONE, ST_TIMEOUT, ST_TOO_LARGE = range(6)
POL_FIFO, POL_FIRST_FIT, POL_PRIO_FIFO, POL_PRIO_FIRST_FIT = range(4)
POLICIES = {"fifo": POL_FIFO, "first_fit": POL_FIRST_FIT, "mmu": POL_FIRST_FIT,
            "prio_fifo": POL_PRIO_FIFO, "prio_first_fit": POL_PRIO_FIRST_FIT,
            "prio_mmu": POL_PRIO_FIRST_FIT}
FLAG_FIFO_BYPASS = 1

OUT_DTYPE = np.dtype([("status", "<i4"), ("pad", "<i4"), ("grant_seq", "<i8"),
                      ("grant_t", "<u8"), ("offset", "<u8"), ("done_t", "<u8")])


class _Stats(ctypes.Structure):
    _fields_ = [("peak_used", ctypes.c_uint64), ("frag_waits", ctypes.c_uint64),
                ("passes", ctypes.c_uint64), ("makespan", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        lib.des_run.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(_Stats)]
        lib.des_run.restype = ctypes.c_int
        lib.des_ops_run.argtypes = [ctypes.c_int, P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_int)]
        lib.des_ops_run.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def simulate(jobs: np.ndarray, budget: int, policy, granule: int = 256, flags: int = 0,
             exclusive: bool = False):
    """Run the DES over job records (``tracegen.JOB_DTYPE``).

    ``exclusive`` makes every job declare the whole pool, the paper's way of
    running an application alone on the GPU (so jobs run one at a time).
    Returns ``(out, stats)``: a structured array (status, grant_seq, grant_t,
    offset, done_t) per job and a dict of counters.
    """
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    n = len(jobs)
    arrival = np.ascontiguousarray(jobs["arrival_ns"], dtype=np.uint64)
    need = np.ascontiguousarray(jobs["need"], dtype=np.uint64)
    if exclusive:
        need = np.full(n, budget // granule * granule, dtype=np.uint64)
    dur = np.ascontiguousarray(jobs["duration_ns"], dtype=np.uint64)
    tmo = np.ascontiguousarray(jobs["timeout_ns"], dtype=np.uint64)
    prio = np.ascontiguousarray(jobs["prio"], dtype=np.int32)
    out = np.zeros(n, dtype=OUT_DTYPE)
    st = _Stats()
    rc = _load().des_run(n, _ptr(arrival), _ptr(need), _ptr(dur), _ptr(tmo), _ptr(prio),
                         int(budget), int(granule), pol, int(flags), _ptr(out), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"des_run failed: {rc}")
    return out, {"peak_used": st.peak_used, "frag_waits": st.frag_waits, "passes": st.passes,
                 "makespan": st.makespan}


# ---------------------------------------------------------------- op mode
OP_DECLARE, OP_RELEASE, OP_CANCEL = range(3)
RC_OK, RC_NOT_READY, RC_TIMEOUT, RC_TOO_LARGE, RC_INVALID = range(5)

OP_DTYPE = np.dtype([("t", "<u8"), ("type", "<i4"), ("ticket", "<i4"), ("arg", "<u8"), ("prio", "<i4"),
                     ("pad", "<i4")])
OP_OUT_DTYPE = np.dtype([("rc", "<i4"), ("ticket", "<i4"), ("used", "<u8"), ("peak_used", "<u8"),
                         ("grants", "<u8"), ("passes", "<u8"), ("frag_waits", "<u8"),
                         ("max_free_extent", "<u8"), ("free_extents", "<u4"), ("waiting", "<u4"),
                         ("done", "<u4"), ("pad2", "<u4")])


def make_ops(items) -> np.ndarray:
    """Op records from tuples: ("declare", need[, prio]), ("release", ticket[, bytes]),
    ("cancel", ticket); logical time = position in the list."""
    ops = np.zeros(len(items), dtype=OP_DTYPE)
    for k, it in enumerate(items):
        ops["t"][k] = k
        kind = it[0]
        if kind == "declare":
            ops["type"][k] = OP_DECLARE
            ops["arg"][k] = it[1]
            ops["prio"][k] = it[2] if len(it) > 2 else 0
            ops["ticket"][k] = -1
        elif kind == "release":
            ops["type"][k] = OP_RELEASE
            ops["ticket"][k] = it[1]
            ops["arg"][k] = it[2] if len(it) > 2 else 0
        elif kind == "cancel":
            ops["type"][k] = OP_CANCEL
            ops["ticket"][k] = it[1]
        else:
            raise ValueError(kind)
    return ops


def simulate_ops(ops: np.ndarray, budget: int, policy, granule: int = 256, flags: int = 0):
    """Run a sequence of life-cycle calls (``OP_DTYPE`` records, or tuples for
    ``make_ops``) through the op-sequence mode of the simulator.

    Returns ``(tickets, per_op)``: one ``OUT_DTYPE`` record per ticket handed
    out (status, grant_seq, grant_t, offset, done_t) and one ``OP_OUT_DTYPE``
    record per op (its result code, the ticket a declare got, and the scalar
    state after the op).
    """
    if not isinstance(ops, np.ndarray):
        ops = make_ops(ops)
    ops = np.ascontiguousarray(ops, dtype=OP_DTYPE)
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    n = len(ops)
    tickets = np.zeros(max(n, 1), dtype=OUT_DTYPE)
    per_op = np.zeros(max(n, 1), dtype=OP_OUT_DTYPE)
    nt = ctypes.c_int(0)
    lib = _load()
    rc = lib.des_ops_run(n, _ptr(ops), int(budget), int(granule), pol, int(flags), _ptr(tickets),
                         _ptr(per_op), ctypes.byref(nt))
    if rc != 0:
        raise RuntimeError(f"des_ops_run failed: {rc}")
    return tickets[: nt.value].copy(), per_op[:n].copy()
