"""sg_replay_noalloc: the admission replay for callers that cannot allocate
device memory -- a process whose device memory all belongs to the pool
this library schedules, where one more cudaMalloc would fall outside the
accounted budget, or a latency-critical loop that must stay out of the
CUDA allocator. Its log must equal sg_replay's (bit for bit: the log is
integer data) on two calls in a row through the shared workspace array."""
import numpy as np
import pytest
import torch

from paper_1712_04495_b300 import tracegen as tg

pytestmark = pytest.mark.gpu


def _replay_both(jobs, budget, policy, timed_free_check):
    from paper_1712_04495_b300 import abi, runtime
    n = len(jobs)
    d_jobs = runtime.to_device(jobs)
    rec_sz = abi.RECORD_DTYPE.itemsize
    log_ref = torch.empty(n * rec_sz, dtype=torch.uint8, device="cuda")
    log_new = torch.full((n * rec_sz,), 0xAB, dtype=torch.uint8, device="cuda")
    st_ref = torch.zeros(4, dtype=torch.int64, device="cuda")
    st_new = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    ws = torch.empty(abi.sg_replay_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert abi.sg_replay(d_jobs.data_ptr(), n, budget, 256, policy, 0, False, log_ref.data_ptr(),
                         ws.data_ptr(), st_ref.data_ptr(), stream) == abi.SG_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    rc = abi.sg_replay_noalloc(d_jobs.data_ptr(), n, budget, 256, policy, 0, False, log_new.data_ptr(),
                               st_new.data_ptr(), stream)
    torch.cuda.synchronize()
    assert rc == abi.SG_OK
    if timed_free_check:
        # nothing was allocated: torch's pool is unchanged, and the device's
        # free memory did not drop by an allocation's granularity (2 MiB; the
        # reading is device-wide, so it assumes no other process allocates
        # on this GPU meanwhile)
        assert torch.cuda.memory_allocated() == alloc0
        assert free0 - torch.cuda.mem_get_info()[0] < (2 << 20)
    assert torch.equal(log_new, log_ref)
    assert torch.equal(st_new, st_ref)
    assert int(st_ref[3].item()) == 0
    rec = runtime.from_device(log_ref, abi.RECORD_DTYPE, n)
    assert np.all(rec["status"] >= 3)


def test_two_calls_in_a_row_match_sg_replay():
    # a larger trace first, then a smaller one: the second call runs over
    # the first call's leftovers in the shared array
    big = tg.random_admission_trace(11, 3000, 1 << 20, max_arrival=20000, max_dur=900,
                                    timeout_frac=0.1)
    _replay_both(big, 1 << 20, "first_fit", timed_free_check=False)
    small = tg.trace_c2(saturated=True)
    _replay_both(small.jobs, small.budget, "fifo", timed_free_check=True)


def test_rejects_traces_beyond_the_limit():
    from paper_1712_04495_b300 import abi
    assert abi.sg_replay_noalloc(0, abi.SG_REPLAY_NOALLOC_MAX_JOBS + 1, 1 << 20, 256, "fifo", 0, False,
                                 0) == abi.SG_ERR_TOO_LARGE


def test_a_trace_of_exactly_the_limit_matches_sg_replay():
    from paper_1712_04495_b300 import abi
    n = abi.SG_REPLAY_NOALLOC_MAX_JOBS
    jobs = tg.random_admission_trace(5, n, 1 << 24, max_arrival=200000, max_dur=4000)
    _replay_both(jobs, 1 << 24, "first_fit", timed_free_check=True)
