"""CPU oracle for the co-scheduler: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import anything from here. The
product path (``paper_1712_04495_b300``) never imports, links or runs it,
and this package never imports the product's CUDA library.

Contents, each written from arXiv 1712.04495 and the plain definition of
each job's arithmetic:

* ``des``        discrete-event simulator of admission and notification
                 (Sec. III-B state, Sec. IV life cycle, Sec. V policies), in C.
* ``kernels``    CPU reference results of the three job kinds: FP32 STREAM
                 triad (two roundings), CSR SpMV (fp64 accumulation) and
                 BF16 GEMM (fp64 accumulation), plus sampled variants.
* ``invariants`` checks every admission log must satisfy.
* ``brute``      brute-force schedule enumeration for traces of 3-5 jobs.
* ``metrics``    makespan, nearest-rank wait / turnaround percentiles.

Job data come from ``paper_1712_04495_b300.tracegen``, the seeded input
generator module that holds none of the scheduling or job arithmetic.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, brute force, invariants or values the paper prints
(the concurrency arithmetic of Sec. VI-C); no trace-level admission log is
printed in the paper, so the DES is pinned by those and not by a paper
trace.
"""
