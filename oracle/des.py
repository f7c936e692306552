"""ctypes front of the C discrete-event simulator (``des.c``)."""
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
