"""The live device engine against the oracle, one life-cycle call at a time
(Sec. IV pre-allocation and post-free, including partial post-free and the
withdrawal of a timed-out wait; the Sec. V policies).

Each call goes through the C ABI on a live context (the engine state shared
through GPU-scope loads and stores under the device lock, not the replay's
owned copy), and the device is synchronised before the next call, so the
result is deterministic. After every call the test compares with the
oracle's op-sequence mode: the call's result code and ticket, the tickets it
granted in grant order with their offsets, and the engine's scalar state
(used and peak bytes, grants, passes, fragmentation-blocked passes, free
extents and the largest, waiting and finished tickets). At the end every
ticket's state is compared too.
"""
import numpy as np
import pytest
import torch

from oracle import des
from paper_1712_04495_b300 import tracegen as tg

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

KIB = 1 << 10
MIB = 1 << 20
STATE = ("used", "peak_used", "grants", "passes", "frag_waits", "max_free_extent", "free_extents",
         "waiting", "done")


def _rc_map(abi):
    return {abi.SG_OK: des.RC_OK, abi.SG_NOT_READY: des.RC_NOT_READY, abi.SG_ERR_TIMEOUT: des.RC_TIMEOUT,
            abi.SG_ERR_TOO_LARGE: des.RC_TOO_LARGE, abi.SG_ERR_INVALID: des.RC_INVALID}


def _check_live(calls, budget, policy, flags=0):
    from paper_1712_04495_b300 import abi, runtime as rt
    rcm = _rc_map(abi)
    tick, per_op = des.simulate_ops(calls, budget, policy, flags=flags)
    s = rt.Scheduler(budget, policy, flags=flags, max_tickets=len(calls) + 1)
    cursor = 0
    grants_before = 0
    try:
        for k, c in enumerate(calls):
            where = (policy, k, c)
            if c[0] == "declare":
                try:
                    t = s.declare(c[1], c[2] if len(c) > 2 else 0)
                    rc = abi.SG_OK
                except abi.SgError as e:
                    t, rc = -1, e.code
                assert t == int(per_op["ticket"][k]), where
            elif c[0] == "release":
                rc = s.release(c[1], c[2] if len(c) > 2 else 0)
                torch.cuda.synchronize()
            else:
                rc, _ = abi.sg_cancel(s.ctx, c[1])
            assert rcm.get(rc, -1) == int(per_op["rc"][k]), (where, abi.sg_strerror(rc))
            st = abi.sg_state(s.ctx)                # waits for the engine's streams
            assert st["error_flags"] == 0, where
            for f in STATE:
                assert int(st[f]) == int(per_op[f][k]), (where, f, int(st[f]), int(per_op[f][k]))
            prc, cursor, granted = abi.sg_poll_grants(s.ctx, cursor)
            assert prc == abi.SG_OK
            grants_after = int(per_op["grants"][k])
            want = sorted(np.nonzero((tick["grant_seq"] >= grants_before) &
                                     (tick["grant_seq"] < grants_after))[0],
                          key=lambda j: int(tick["grant_seq"][j]))
            assert granted == [int(j) for j in want], where
            for j in granted:
                grc, g = abi.sg_try(s.ctx, j)
                assert grc == abi.SG_OK and g.offset == int(tick["offset"][j]), (where, j)
                assert g.ptr == s.pool.data_ptr() + g.offset
            grants_before = grants_after
        want_rc = {des.ST_RUNNING: abi.SG_OK, des.ST_QUEUED: abi.SG_NOT_READY,
                   des.ST_TIMEOUT: abi.SG_ERR_TIMEOUT, des.ST_DONE: abi.SG_ERR_INVALID}
        for j in range(len(tick)):
            grc, g = abi.sg_try(s.ctx, j)
            assert grc == want_rc[int(tick["status"][j])], (policy, j)
            if grc == abi.SG_OK:
                assert g.offset == int(tick["offset"][j])
        assert abi.sg_device_error(s.ctx) == 0
    finally:
        s.shutdown()
    return tick, per_op


HAND_WORKED = {
    "shrink_regrant": ([("declare", 600 * KIB), ("declare", 500 * KIB), ("release", 0, 200 * KIB),
                        ("release", 0, 400 * KIB), ("release", 0), ("release", 1, 0)], MIB, "fifo"),
    "granule_rounding": ([("declare", 1000), ("release", 0, 100), ("release", 0, 200), ("release", 0, 700),
                          ("release", 0, 1)], 4096, "first_fit"),
    "double_release": ([("declare", 5000), ("release", 0, 0), ("release", 0, 0), ("release", 0, 100)],
                       1 << 16, "fifo"),
    "withdraw_head_fifo": ([("declare", 700 * KIB), ("declare", 500 * KIB), ("declare", 100 * KIB),
                            ("cancel", 1), ("cancel", 2), ("cancel", 1), ("release", 1), ("cancel", 0),
                            ("release", 0), ("cancel", 0)], MIB, "fifo"),
    "too_large": ([("declare", MIB + 1), ("declare", MIB), ("declare", 0), ("release", 0)], MIB, "fifo"),
    "fragmentation": ([("declare", 256 * KIB)] * 4 + [("release", 1), ("release", 3, 128 * KIB),
                                                      ("declare", 300 * KIB), ("release", 2)], MIB, "first_fit"),
}


@pytest.mark.parametrize("case", sorted(HAND_WORKED))
def test_hand_worked_sequences_on_the_live_engine(case):
    calls, budget, policy = HAND_WORKED[case]
    _check_live(calls, budget, policy)


@pytest.mark.parametrize("policy,flags,prio_levels", [
    ("fifo", 0, 1), ("first_fit", 0, 1), ("prio_fifo", 0, 3), ("prio_first_fit", 0, 3),
    ("fifo", des.FLAG_FIFO_BYPASS, 1)], ids=["fifo", "first_fit", "prio_fifo", "prio_first_fit", "fifo_bypass"])
def test_random_call_sequences_match_the_oracle(policy, flags, prio_levels):
    budget = 64 * MIB
    for seed in (1, 2):
        calls = tg.random_lifecycle_calls(seed, 300, budget, prio_levels=prio_levels)
        tick, per_op = _check_live(calls, budget, policy, flags)
        # the sequence exercised what it is for
        kinds = {c[0] for c in calls}
        assert kinds == {"declare", "release", "cancel"}
        assert int(per_op["waiting"].max()) > 0 and int(per_op["grants"][-1]) > 10
        assert np.any(per_op["rc"] == des.RC_INVALID) and np.any(per_op["rc"] == des.RC_TIMEOUT)
