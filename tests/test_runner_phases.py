"""The trace runner's start rule (csrc/phases.h), on the CPU: SpMV and GEMM
jobs are kept apart in alternating phases, triads run beside either, a
phase yields after its quota while the other kind waits, no two long jobs
(declared duration of 1 ms or more) run at once, nothing starves,
and each slot pool starts the earliest-admitted job it may start. The rule
is driven by a discrete simulation of admitted jobs on stream slots
(tests/phases_harness), which mirrors sg_run_trace's loop."""
import ctypes
import os
import sys
import tempfile

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "phases_harness"))
import phases_build  # noqa: E402

_ERRORS = {1: "pick is not the earliest admitted job the pool may start",
           2: "an SpMV and a GEMM ran at the same time",
           3: "a free slot stayed free while a job it serves could start",
           4: "without the rule a kind was held back",
           5: "a job started before it was admitted",
           6: "a job never started",
           7: "two long jobs ran at the same time"}


@pytest.fixture(scope="module")
def sim():
    L = ctypes.CDLL(phases_build.build(tempfile.mkdtemp(prefix="sg_phases_")))
    L.ph_sim.restype = ctypes.c_int
    L.ph_sim.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                         ctypes.c_int, ctypes.c_void_p]

    def run(seed, n_jobs, n_other, n_gemm, apart, quota):
        st = (ctypes.c_int64 * 3)()
        rc = L.ph_sim(seed, n_jobs, n_other, n_gemm, int(apart), quota, st)
        assert rc == 0, _ERRORS.get(rc, rc)
        return list(st)
    return run


@pytest.mark.parametrize("n_other,n_gemm", [(4, 4), (4, 0), (1, 1), (6, 2), (32, 8)])
@pytest.mark.parametrize("quota", [1, 8, 64])
def test_apart_phases_hold(sim, n_other, n_gemm, quota):
    for seed in range(20):
        ticks, phases, worst = sim(seed, 400, n_other, n_gemm, True, quota)
        assert phases >= 1
        # starts of one kind while the other waits stay within the quota
        assert worst <= quota


def test_quota_bounds_phase_length_and_alternates(sim):
    _, phases_small, _ = sim(7, 2000, 4, 4, True, 4)
    _, phases_large, _ = sim(7, 2000, 4, 4, True, 1000)
    assert phases_small > phases_large >= 1


@pytest.mark.parametrize("n_other,n_gemm", [(4, 4), (4, 0), (2, 1)])
def test_overlap_starts_every_admitted_job_when_a_slot_frees(sim, n_other, n_gemm):
    for seed in range(20):
        sim(seed, 400, n_other, n_gemm, False, 64)
