"""Benchmark: co-scheduled job execution on one B300 (arXiv 1712.04495).

A step is one pass of the whole path over the mixed 256-job trace (40%
FP32 triad, 30% CSR SpMV, 30% BF16 GEMM; 16 GiB pool, seed 0): every job
is declared, admitted by the device engine (first fit), generated and run
in its grant on a stream slot, and released from its kernel's last block,
which wakes the waiters. Arrivals are compressed to t = 0 (the saturated
trace): at the paper-style 200 jobs/s the run is arrival-bound, so that
literal run is reported beside it.

Prints one JSON line (rank 0). Extra keys: makespan of FIFO / first fit /
exclusive-serial, p50 / p99 wait, the literal 200 jobs/s run, the roofline
of the dominant kernel, the oracle's CPU baseline and the end-to-end
number through host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1712_04495_b300 import tracegen as tg  # noqa: E402

WORKLOAD = "mixed256_16GiB"
METRIC = "jobs/s, co-scheduled (first fit) mixed 256-job trace, 16 GiB pool, 1 B300"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "source": "fallback"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 20 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- distributed
def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(jobs_local: int, seconds_local: float, world: int, backend_ops=None):
    """Whole-job throughput: jobs over all ranks / slowest rank's time."""
    if world == 1 or backend_ops is None:
        return jobs_local / seconds_local, seconds_local
    total_jobs, max_s = backend_ops(jobs_local, seconds_local)
    return total_jobs / max_s, max_s


def _torch_ops(device):
    import torch
    import torch.distributed as dist

    def ops(jobs, secs):
        t = torch.tensor([float(jobs)], device=device, dtype=torch.float64)
        s = torch.tensor([secs], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        dist.all_reduce(s, op=dist.ReduceOp.MAX)
        return float(t.item()), float(s.item())
    return ops


# ----------------------------------------------------------- CPU oracle
def stratified_samples(trace: tg.Trace, parts: int) -> list:
    """Split the trace's jobs into `parts` samples that each keep its kind mix
    and size spread: the jobs of each kind, in size order, are dealt out in
    turn, each kind continuing where the previous one stopped."""
    out = [[] for _ in range(parts)]
    k = 0
    for kind in (tg.KIND_TRIAD, tg.KIND_SPMV, tg.KIND_GEMM):
        idx = np.nonzero(trace.jobs["kind"] == kind)[0]
        idx = idx[np.argsort(trace.jobs["p0"][idx], kind="stable")]
        for i, j in enumerate(idx):
            out[(k + i) % parts].append(int(j))
        k += len(idx)
    return [sorted(o) for o in out]


def oracle_sample(trace: tg.Trace, sample: list):
    """The oracle as it stands over a sample of the trace: the admission DES
    over the whole trace (one thread), then each sampled job's CPU reference
    result with OpenMP over the host cores (the GEMM's product by a BLAS
    matrix multiply on the same cores). Returns (jobs, seconds)."""
    from oracle import des
    from oracle import omp
    t0 = time.perf_counter()
    des.simulate(trace.jobs, trace.budget, "first_fit")
    for j in sample:
        job = trace.jobs[j]
        kind, key = int(job["kind"]), int(job["key"])
        if kind == tg.KIND_TRIAD:
            omp.triad(key, int(job["p0"]))
        elif kind == tg.KIND_SPMV:
            omp.spmv(key, int(job["p0"]), trace.tables[int(job["p2"])])
        else:
            s = int(job["p0"])
            omp.gemm(key, s, s, s)
    return len(sample), time.perf_counter() - t0


def _oracle_threads() -> int:
    """Host threads the oracle's job results run on (OpenMP and BLAS)."""
    from oracle import omp
    n = omp.threads()
    try:
        import threadpoolctl
        for d in threadpoolctl.threadpool_info():
            if d.get("user_api") == "blas":
                n = max(n, int(d.get("num_threads", 1)))
    except Exception:
        pass
    return n


def _sample_desc(trace: tg.Trace, sample: list, parts: int) -> str:
    kinds = trace.jobs["kind"][sample]
    return (f"admission DES over all {len(trace)} jobs + CPU reference results of a stratified 1/{parts} "
            f"of the jobs ({int(np.sum(kinds == tg.KIND_TRIAD))} triad, {int(np.sum(kinds == tg.KIND_SPMV))} "
            f"SpMV, {int(np.sum(kinds == tg.KIND_GEMM))} GEMM: each kind in size order, every {parts}th job), "
            f"OpenMP + BLAS on the host cores")


def _threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload_config(ws: int) -> dict:
    """The workload both arms report (the same trace; the oracle arm runs a sample of it)."""
    return {"workload": WORKLOAD + "_t0", "jobs": 256, "pool_gib": 16, "policy": "first_fit",
            "arrivals": "t=0 (saturated)", "seed": 0,
            "start_rule": "SpMV and GEMM jobs in alternating phases (<= 64 starts), "
                          "triads beside either; jobs declared >= 1 ms one at a time; "
                          "stream slots 4 + 4 GEMM",
            "l2": "inputs larger than L2 (about 50 GB of job data per step)",
            "parallelism": f"replicas x{ws}"}


def reference_arm(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return 0
    trace = tg.trace_c2(saturated=True)
    # each step a different stratified part of the trace; the parts together
    # cover it once (a whole step is about a minute of host work)
    parts = stratified_samples(trace, max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        oracle_sample(trace, parts[w])
    jobs, secs = 0, 0.0
    for k in range(args.steps):
        d, e = oracle_sample(trace, parts[args.warmup + k])
        jobs += d
        secs += e
    v = jobs / secs
    sample = (f"admission DES over all {len(trace)} jobs + CPU reference results of one of "
              f"{len(parts)} stratified parts of the trace per step (each kind in size order, dealt out in "
              f"turn), OpenMP + BLAS on the host cores")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "jobs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(ws),
            "cpu_baseline": {"value": v, "unit": "jobs/s", "cores": _oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "jobs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ kernels
def profiled_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary `profiles/<name>.traffic.json`,
    or None once the kernel's sources no longer hash to the recorded value."""
    import hashlib
    p = os.path.join(ROOT, "profiles", name + ".traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for src in d["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return d["traffic_bytes_per_launch"] if h.hexdigest() == d["sha256"] else None


def kernel_roofline(torch, abi, runtime, peaks):
    """Standalone timing of the job kernels on a torch stream (CUDA events),
    the same launch configuration the trace uses."""
    s = torch.cuda.current_stream()
    out = {}
    # BF16 GEMM 8192^3
    M = N = Kd = 8192
    A = torch.empty(M * Kd, dtype=torch.int16, device="cuda")
    B = torch.empty(N * Kd, dtype=torch.int16, device="cuda")
    C = torch.empty(M * N, dtype=torch.float32, device="cuda")
    assert abi.sg_gen_gemm(A.data_ptr(), B.data_ptr(), M, N, Kd, 42, s.cuda_stream) == 0
    for _ in range(3):
        abi.sg_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, Kd, s.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        abi.sg_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, Kd, s.cuda_stream)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * M * N * Kd
    tf = flops / (ms * 1e-3) / 1e12
    out["gemm"] = {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                   "frac": tf / peaks["bf16_tflops"], "traffic": profiled_traffic("gemm_tc_8192_bf16"), "ms": ms,
                   "kernel": f"k_gemm_tc {abi.gemm_tile_name(abi.sg_gemm_tile(M, N))} tile, 8192^3 bf16",
                   "flops_per_launch": flops}
    del A, B, C
    # FP32 triad, n = 64M (768 MB per launch, larger than L2)
    n = 64 << 20
    buf = torch.empty(3 * n, dtype=torch.float32, device="cuda")
    a, b, c = buf[:n], buf[n:2 * n], buf[2 * n:]
    abi.sg_gen_triad(b.data_ptr(), c.data_ptr(), n, 7, s.cuda_stream)
    for _ in range(3):
        abi.sg_triad(a.data_ptr(), b.data_ptr(), c.data_ptr(), 3.0, n, s.cuda_stream)
    reps = 20
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        abi.sg_triad(a.data_ptr(), b.data_ptr(), c.data_ptr(), 3.0, n, s.cuda_stream)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = 12.0 * n / (ms * 1e-3) / 1e9
    out["triad"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "traffic": profiled_traffic("triad_fp32_64M"), "ms": ms,
                    "kernel": "k_triad n=64M", "bytes_per_launch": 12 * n}
    del buf
    # FP32 CSR SpMV, 1e7 rows, Poisson(16) non-zeros per row
    rows, lam = 10_000_000, 16.0
    cap = tg.spmv_nnz_cap(rows, lam)
    lay = tg.spmv_layout(rows, cap)
    base = torch.empty(lay["total"], dtype=torch.uint8, device="cuda")
    tab = torch.from_numpy(tg.poisson_cdf_table(lam).view(np.int64).copy()).cuda()
    # the arrays in a grant of a scheduler pool, where an SpMV job's arrays
    # are: x is then gathered through the pool's texture window, as in a job
    sp = runtime.Scheduler(lay["total"], pool=base)
    sp_t = sp.declare(lay["total"])
    rc, grant = sp.wait(sp_t, 10 ** 9)
    assert rc == abi.SG_OK, rc
    p = base.data_ptr() + grant.offset
    gather_path = abi.sg_spmv_gather_path(p + lay["x"], rows)
    abi.sg_gen_spmv(p, rows, cap, tab.data_ptr(), 5, 0, s.cuda_stream)
    torch.cuda.synchronize()
    nnz = int(base[lay["row_ptr"] + 4 * rows:lay["row_ptr"] + 4 * rows + 4].view(torch.int32).item())
    args_ = (p + lay["row_ptr"], False, p + lay["col"], p + lay["val"], p + lay["x"], p + lay["y"], rows,
             s.cuda_stream)
    for _ in range(3):
        abi.sg_spmv(*args_)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        abi.sg_spmv(*args_)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    alg = 4 * (rows + 1) + 8 * nnz + 8 * rows
    gbs = alg / (ms * 1e-3) / 1e9
    # the ceiling that binds it: x[col] gathers alone over the same columns and
    # x (sg_gather_sum, a measurement kernel), timed the same way
    gout = torch.empty((nnz + 1023) // 1024, dtype=torch.float32, device="cuda")
    gargs = (p + lay["col"], p + lay["x"], rows, nnz, gout.data_ptr(), s.cuda_stream)
    for _ in range(3):
        abi.sg_gather_sum(*gargs)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        abi.sg_gather_sum(*gargs)
    e1.record(s)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / reps
    del gout
    sp.release(sp_t)
    sp.shutdown()
    gpath = "texture window of the pool" if gather_path == abi.SG_GATHER_TEXTURE else "global loads"
    out["spmv"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": gbs / peaks["hbm_gbs"], "traffic": profiled_traffic("spmv_csr_1e7rows_poisson16"),
                   "ms": ms,
                   "kernel": f"k_spmv<int, {'XTex' if gather_path == abi.SG_GATHER_TEXTURE else 'XLoad'}> rows=1e7 "
                             "nnz/row~Poisson(16)", "bytes_per_launch": alg,
                   "x_gathers": gpath,
                   "target": 0.70, "target_met": gbs / peaks["hbm_gbs"] >= 0.70,
                   "why_not": "each non-zero gathers x[col] at a uniform random column of a 40 MB x: one 32-byte "
                              "L2 sector per 4-byte value (texture hit rate 0%); the kernel keeps the SM-to-crossbar "
                              "request path 94% busy (97% for the gathers alone), with HBM traffic equal to the "
                              "algorithmic bytes",
                   "gathers_per_s": nnz / (ms * 1e-3),
                   "gather_ceiling": {"gathers_per_s": nnz / (g_ms * 1e-3), "ms": g_ms,
                                      "kernel": "sg_gather_sum: x[col] alone over the SpMV's own columns "
                                                "(4 per thread from one 128-bit column load, 8 blocks per SM; "
                                                f"x through the {gpath})",
                                      "spmv_frac": g_ms / ms}}
    # the input generators, alone at the same sizes (instruction-issue and ALU bound)
    tab_ptr = tab.data_ptr()
    del base
    base = torch.empty(lay["total"], dtype=torch.uint8, device="cuda")
    p = base.data_ptr()
    A = torch.empty(8192 * 8192, dtype=torch.int16, device="cuda")
    B = torch.empty(8192 * 8192, dtype=torch.int16, device="cuda")
    buf = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    gens = {"spmv": (lambda: abi.sg_gen_spmv(p, rows, cap, tab_ptr, 5, 0, s.cuda_stream), nnz, "non-zero"),
            "gemm": (lambda: abi.sg_gen_gemm(A.data_ptr(), B.data_ptr(), 8192, 8192, 8192, 42, s.cuda_stream),
                     2 * 8192 * 8192, "bf16 element"),
            "triad": (lambda: abi.sg_gen_triad(buf[:n].data_ptr(), buf[n:].data_ptr(), n, 7, s.cuda_stream),
                      n, "element")}
    out["generators"] = {}
    for name, (fn, units, what) in gens.items():
        fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(5):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out["generators"][name] = {"ms": ms, "ns_per_unit": 1e6 * ms / units, "unit": what}
    del base, A, B, buf
    torch.cuda.synchronize()
    return out


def makespan_bound(trace: tg.Trace, kr: dict, peaks: dict, serial_ms: float) -> dict:
    """Lower bounds on a step's makespan, against the measured exclusive-serial one.

    disjoint_resources: the step's work on each resource at that resource's
    rate, if every kind's bottleneck were a resource of its own and all of it
    overlapped: HBM bytes (kernels' algorithmic bytes plus the generators'
    writes) at the measured copy bandwidth; GEMM flops at the sustained bf16
    peak; SpMV gathers (expected rows x lambda) at the SpMV's own gather rate
    measured above; generator time at the generators' measured rates.
    unit_counters: the largest per-unit busy time of a step from ncu unit
    counters of each kernel and its time per step in the launch list (a
    committed profile): no schedule packs a unit beyond 100%."""
    hbm, flops, gathers, gen_ms = 0.0, 0.0, 0.0, 0.0
    g = kr["generators"]
    for job in trace.jobs:
        kind = int(job["kind"])
        if kind == tg.KIND_TRIAD:
            nn = int(job["p0"])
            hbm += tg.triad_alg_bytes(nn) + 8 * nn
            gen_ms += g["triad"]["ns_per_unit"] * nn * 1e-6
        elif kind == tg.KIND_SPMV:
            rows = int(job["p0"])
            nnz = rows * trace.lambdas[int(job["p2"])]
            hbm += tg.spmv_alg_bytes(rows, int(nnz)) + 8 * nnz + 4 * (rows + 1) + 4 * rows
            gathers += nnz
            gen_ms += g["spmv"]["ns_per_unit"] * nnz * 1e-6
        else:
            m = int(job["p0"])
            hbm += 2 * m * m + 2 * m * m + 4 * m * m + 4 * m * m
            flops += tg.gemm_flops(m, m, m)
            gen_ms += g["gemm"]["ns_per_unit"] * 2 * m * m * 1e-6
    parts = {"hbm_ms": hbm / (peaks["hbm_gbs"] * 1e9) * 1e3,
             "tensor_ms": flops / ((peaks["bf16_tflops_sustained"] or peaks["bf16_tflops"]) * 1e12) * 1e3,
             "gathers_ms": gathers / kr["spmv"]["gathers_per_s"] * 1e3,
             "generators_ms": gen_ms}
    disjoint = max(parts.values())
    out = {"exclusive_serial_ms": serial_ms,
           "disjoint_resources": {"ms": disjoint, "ratio_vs_serial": disjoint / serial_ms, **parts}}
    p = os.path.join(ROOT, "profiles", "units_per_kernel_mixed256.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        busy = {}
        for u in d["units"]:
            tot = 0.0
            for k, t in d["per_step_ms"].items():
                ref = d["same_units_as"].get(k, k)
                tot += t * d["pct"][ref][u] / 100.0
            busy[u] = tot
        u_max = max(busy, key=busy.get)
        out["unit_counters"] = {"ms": busy[u_max], "unit": u_max, "ratio_vs_serial": busy[u_max] / serial_ms,
                                "source": "ncu unit counters per kernel x kernel time per step of the launch list"}
    return out


# ------------------------------------------------------------ batching
def batching_section(torch, abi, runtime, reps: int = 3) -> dict:
    """10,000 tiny jobs: one launch per job (online admission) vs one CUDA
    graph vs the persistent grouped kernel (both on the engine's replay plan)."""
    tr = tg.trace_c4()
    n = len(tr)
    pool = torch.empty(tr.budget, dtype=torch.uint8, device="cuda")
    tab = runtime.device_tables(tr)
    out = {"workload": tr.name, "jobs": n}
    s = runtime.Scheduler(tr.budget, "first_fit", pool=pool)
    d_jobs = runtime.to_device(tr.jobs)
    t = []
    for i in range(reps + 1):
        rc, _, _, st = s.run_trace(d_jobs, tab, abi.SG_RUN_SATURATED)
        assert rc == abi.SG_OK
        if i:
            t.append(st["elapsed_ns"] * 1e-9)
    launches = st["launches"]
    rc, _, _, st = s.run_trace(d_jobs, tab, abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE)
    assert rc == abi.SG_OK
    serial_s = st["elapsed_ns"] * 1e-9
    s.shutdown()
    out["exclusive_serial"] = {"jobs_per_s": n / serial_s, "ms": 1e3 * serial_s}
    out["per_job_launch"] = {"jobs_per_s": n / statistics.median(t), "ms": 1e3 * statistics.median(t),
                             "launches": launches}
    t0 = time.perf_counter()
    pl = runtime.Planned(pool, tr.jobs, tab, "first_fit", keep=False, budget=tr.budget)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    ms_g = timed(lambda: pl.run_graph())
    ms_b = timed(lambda: pl.run_batch())
    rc, done, err = pl.batch_status()
    assert rc == abi.SG_OK and done == n, (rc, done, err)
    ginfo = abi.sg_graph_info(pl.graph)
    binfo = abi.sg_batch_info(pl.batch)
    out["cuda_graph"] = {"jobs_per_s": n / (ms_g * 1e-3), "ms": ms_g, "kernel_nodes": ginfo["kernels"],
                         "edges": ginfo["edges"]}
    out["persistent_kernel"] = {"jobs_per_s": n / (ms_b * 1e-3), "ms": ms_b, "chunks": binfo["chunks"],
                                "blocks": binfo["blocks"], "launches": 1}
    out["plan_build_s"] = build_s
    out["plan_build_parts_s"] = pl.build_s
    # admission inside the persistent kernel: no plan, the batch's engine
    # releases and grants as jobs finish
    for pol in ("first_fit", "fifo"):
        ob = runtime.OnlineBatch(pool, tr.jobs, tab, pol, budget=tr.budget)
        ms_o = timed(lambda: ob.run())
        rc, done, err = ob.status()
        assert rc == abi.SG_OK and done == n, (rc, done, err)
        ob.close()
        out[f"persistent_online_{pol}"] = {"jobs_per_s": n / (ms_o * 1e-3), "ms": ms_o, "plan": "none",
                                           "ratio_vs_serial": ms_o * 1e-3 / serial_s}
    # single-shot cost: the plan (device replay of the batch, with its copies)
    # and the graph or batch build are host steps outside the timed launches
    # above; exclusive-serial and one launch per job admit inside their time
    plan_ms = 1e3 * pl.build_s["replay"]
    out["cuda_graph"]["ms_incl_plan_and_build"] = plan_ms + 1e3 * pl.build_s["graph"] + ms_g
    out["persistent_kernel"]["ms_incl_plan_and_build"] = plan_ms + 1e3 * pl.build_s["batch"] + ms_b
    out["makespan_ratio_vs_serial"] = {"per_job_launch": statistics.median(t) / serial_s,
                                       "cuda_graph": ms_g * 1e-3 / serial_s,
                                       "persistent_kernel": ms_b * 1e-3 / serial_s,
                                       "cuda_graph_incl_plan_and_build":
                                           out["cuda_graph"]["ms_incl_plan_and_build"] * 1e-3 / serial_s,
                                       "persistent_kernel_incl_plan_and_build":
                                           out["persistent_kernel"]["ms_incl_plan_and_build"] * 1e-3 / serial_s}
    pl.close()
    del pool
    torch.cuda.empty_cache()
    return out


def serving_section(torch, abi, runtime, requests: int, rates=(1000, 2000, 5000, 10000, 20000),
                    overlap_rates=(5000, 10000), short_requests: int = 20000) -> dict:
    """Open-loop serving: Poisson arrivals at each rate, the mixed size mix,
    64 GiB pool, first fit; requests are declared at their arrival time and
    admitted as memory frees up while earlier ones run. `requests` per rate
    from 5k req/s up; the 1k and 2k req/s streams would take 100 s and 50 s
    of arrivals at that count, so they run `short_requests` (nothing waits at
    those rates either way). `overlap` repeats two rates with the runner
    starting SpMV and GEMM jobs side by side, also at `short_requests`."""
    out = {"requests_per_rate": {}, "pool_gib": 64, "policy": "first_fit", "rates": {}, "overlap": {},
           "note": f"{requests} requests per rate from 5k req/s up; 1k and 2k req/s run {short_requests} (at "
                   f"{requests} they would take {requests // 1000} s and {requests // 2000} s of arrivals, and "
                   "nothing waits at those rates); overlap: the runner starting SpMV and GEMM jobs side by side"}
    pool = torch.empty(64 << 30, dtype=torch.uint8, device="cuda")
    for run_flags, rs, key in ((0, rates, "rates"), (abi.SG_RUNF_OVERLAP, overlap_rates, "overlap")):
        s = runtime.Scheduler(64 << 30, "first_fit", pool=pool, run_flags=run_flags)
        for r in rs:
            nreq = requests if (key == "rates" and r >= 5000) else min(requests, short_requests)
            out["requests_per_rate"][f"{key}/{r}"] = nreq
            tr = tg.trace_c5(n_jobs=nreq, rate_per_s=float(r))
            rc, _, _, st = s.run_trace(runtime.to_device(tr.jobs), runtime.device_tables(tr), abi.SG_RUN_TIMED)
            assert rc == abi.SG_OK, st
            out[key][str(r)] = {
                "requests": nreq, "jobs_per_s": nreq / (st["makespan_ns"] * 1e-9),
                "wait_p50_ms": st["wait_p50_ns"] / 1e6, "wait_p99_ms": st["wait_p99_ns"] / 1e6,
                "turnaround_p50_ms": st["turnaround_p50_ns"] / 1e6,
                "turnaround_p99_ms": st["turnaround_p99_ns"] / 1e6,
                "makespan_ms": st["makespan_ns"] / 1e6, "peak_used_gib": st["peak_used"] / 2 ** 30}
        s.shutdown()
    del pool
    torch.cuda.empty_cache()
    return out


def _run_summary(st: dict, n: int) -> dict:
    return {"makespan_ms": st["makespan_ns"] / 1e6, "jobs_per_s": n / (st["makespan_ns"] * 1e-9),
            "wait_p50_ms": st["wait_p50_ns"] / 1e6, "wait_p99_ms": st["wait_p99_ns"] / 1e6,
            "turnaround_p99_ms": st["turnaround_p99_ns"] / 1e6, "peak_used_gib": st["peak_used"] / 2 ** 30,
            "frag_waits": st["frag_waits"]}


def configs_section(torch, abi, runtime) -> dict:
    """The two other admission workloads, co-scheduled against exclusive-serial
    (one run each): 8 triads at t=0 in a 1 GiB pool under FIFO, and memory
    pressure -- 128 jobs of 2-60 GiB in a 170 GiB pool arriving in bursts of
    16 every 200 ms, first fit, where waiters are woken by releases."""
    out = {}
    tr = tg.trace_c1()
    s = runtime.Scheduler(tr.budget, "fifo")
    d_jobs, d_tab = runtime.to_device(tr.jobs), runtime.device_tables(tr)
    row = {"workload": tr.name, "jobs": len(tr), "policy": "fifo"}
    for name, mode in (("co_scheduled", abi.SG_RUN_SATURATED),
                       ("exclusive_serial", abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE)):
        runs = []
        for _ in range(5):
            rc, _, _, st = s.run_trace(d_jobs, d_tab, mode)
            assert rc == abi.SG_OK, st
            runs.append(st)
        row[name] = _run_summary(sorted(runs, key=lambda r: r["makespan_ns"])[2], len(tr))
    row["makespan_ratio"] = row["co_scheduled"]["makespan_ms"] / row["exclusive_serial"]["makespan_ms"]
    out["triad8"] = row
    s.shutdown()
    del s
    tr = tg.trace_c3()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < tr.budget + (8 << 30):
        out["pressure"] = {"workload": tr.name, "skipped": f"needs {tr.budget >> 30} GiB free"}
        return out
    s = runtime.Scheduler(tr.budget, "first_fit")
    d_jobs, d_tab = runtime.to_device(tr.jobs), runtime.device_tables(tr)
    row = {"workload": tr.name, "jobs": len(tr), "policy": "first_fit",
           "need_gib": [round(float(tr.jobs["need"].min()) / 2 ** 30, 1),
                        round(float(tr.jobs["need"].max()) / 2 ** 30, 1)]}
    for name, mode in (("co_scheduled", abi.SG_RUN_TIMED),
                       ("exclusive_serial", abi.SG_RUN_TIMED | abi.SG_RUN_EXCLUSIVE),
                       ("co_scheduled_t0", abi.SG_RUN_SATURATED),
                       ("exclusive_serial_t0", abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE)):
        rc, _, _, st = s.run_trace(d_jobs, d_tab, mode)
        assert rc == abi.SG_OK, st
        row[name] = _run_summary(st, len(tr))
    row["makespan_ratio"] = row["co_scheduled"]["makespan_ms"] / row["exclusive_serial"]["makespan_ms"]
    row["makespan_ratio_t0"] = row["co_scheduled_t0"]["makespan_ms"] / row["exclusive_serial_t0"]["makespan_ms"]
    out["pressure"] = row
    s.shutdown()
    del s, d_jobs, d_tab
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------ paper experiments
def lifecycle_section(torch, abi, runtime, reps: int = 200) -> dict:
    """Per-stage cost of the life cycle through the C ABI (the paper's
    overhead comparison of init / pre-allocation / post-free / shutdown):
    median microseconds per call, host clock, device synchronised."""
    pool = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    t_init, t_decl, t_rel, t_shut = [], [], [], []
    for i in range(max(5, reps // 20)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = abi.sg_init(pool.data_ptr(), pool.numel(), "first_fit", 0, 4096, 4, 0)
        t_init.append(time.perf_counter() - t0)
        for _ in range(reps // 10):
            t0 = time.perf_counter()
            tk = abi.sg_declare(ctx, 1 << 20, 0)
            rc, g = abi.sg_wait(ctx, tk, 10 ** 9)
            t_decl.append(time.perf_counter() - t0)
            assert rc == abi.SG_OK
            t0 = time.perf_counter()
            assert abi.sg_release(ctx, tk, 0, 0) == abi.SG_OK
            torch.cuda.synchronize()
            t_rel.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        abi.sg_shutdown(ctx)
        t_shut.append(time.perf_counter() - t0)
    med = lambda v: 1e6 * statistics.median(v)  # noqa: E731
    return {"init_us": med(t_init), "pre_allocation_us": med(t_decl), "post_free_us": med(t_rel),
            "shutdown_us": med(t_shut), "note": "declare + wait for the grant; release + device sync"}


class _Transport:
    """The client calls of one of the two multi-process designs: the
    scheduler server ("server": UNIX socket, device engine) or the shared
    segment ("shm": host shared memory, decisions made by each client)."""

    def __init__(self, a, kind: str, where: str):
        self.a, self.kind = a, kind
        self.h = a.sg_client_connect(where) if kind == "server" else a.sg_shm_open(where)

    def pool(self):
        return self.a.sg_client_pool(self.h) if self.kind == "server" else self.a.sg_shm_pool(self.h)

    def declare(self, need: int) -> int:
        if self.kind == "server":
            return self.a.sg_client_declare(self.h, need, 0)
        rc, t = self.a.sg_shm_declare(self.h, need, 0)
        assert rc == self.a.SG_OK, rc
        return t

    def wait(self, t: int, ns: int):
        return (self.a.sg_client_wait if self.kind == "server" else self.a.sg_shm_wait)(self.h, t, ns)

    def release(self, t: int) -> int:
        return (self.a.sg_client_release if self.kind == "server" else self.a.sg_shm_release)(self.h, t, 0)

    def close(self):
        (self.a.sg_client_close if self.kind == "server" else self.a.sg_shm_close)(self.h)


def _latency_client(kind: str, where: str, reps: int, q) -> None:
    """Client process of `client_server_section` (no CUDA work of its own)."""
    sys.path.insert(0, ROOT)
    from paper_1712_04495_b300 import abi as a
    t0 = time.perf_counter()
    cl = _Transport(a, kind, where)
    t_conn = time.perf_counter() - t0
    t_decl, t_rel = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        tk = cl.declare(1 << 20)
        rc, _ = cl.wait(tk, 10 ** 9)
        t_decl.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        rc2 = cl.release(tk)
        t_rel.append(time.perf_counter() - t0)
        if rc != a.SG_OK or rc2 != a.SG_OK:
            q.put({"error": f"codes {rc} {rc2}"})
            return
    cl.close()
    med = lambda v: 1e6 * statistics.median(v)  # noqa: E731
    q.put({"connect_us": 1e6 * t_conn, "pre_allocation_us": med(t_decl), "post_free_us": med(t_rel)})


def _serving_client(kind: str, where: str, jobs: list, go, q) -> None:
    """Client process of `processes_section`: triad jobs (n, key) one after
    another on its own stream, each declared, run on the IPC-mapped grant,
    synchronised and released."""
    sys.path.insert(0, ROOT)
    import torch
    from paper_1712_04495_b300 import abi as a
    torch.cuda.set_device(0)
    torch.zeros(1, device="cuda")
    cl = _Transport(a, kind, where)
    cl.pool()
    st = torch.cuda.Stream()
    q.put(("ready", 0.0, []))
    go.wait()
    t_start = time.perf_counter()
    turn = []
    for n, key in jobs:
        t0 = time.perf_counter()
        tk = cl.declare(12 * n)
        rc, g = cl.wait(tk, 60 * 10 ** 9)
        if rc != a.SG_OK:
            q.put(("error", 0.0, [rc]))
            return
        b, c = g.ptr + 4 * n, g.ptr + 8 * n
        a.sg_gen_triad(b, c, n, key, st.cuda_stream)
        a.sg_triad(g.ptr, b, c, 3.0, n, st.cuda_stream)
        st.synchronize()
        cl.release(tk)
        turn.append(time.perf_counter() - t0)
    q.put(("done", time.perf_counter() - t_start, turn))
    cl.close()


def _shm_name(tag: str) -> str:
    return f"/sg_bench_{tag}_{os.getpid()}"


def _run_clients(ctx, kind: str, where: str, work: list, timeout: float = 600):
    """Start one client process per work list, release them together and
    collect (wall seconds, per-job turnaround seconds)."""
    q, go = ctx.Queue(), ctx.Event()
    procs = [ctx.Process(target=_serving_client, args=(kind, where, w, go, q)) for w in work]
    for p in procs:
        p.start()
    try:
        for _ in procs:
            assert q.get(timeout=300)[0] == "ready"
        t0 = time.perf_counter()
        go.set()
        turns = []
        for _ in procs:
            kind_, _, turn = q.get(timeout=timeout)
            assert kind_ == "done", (kind_, turn)
            turns += turn
        wall = time.perf_counter() - t0
    finally:
        for p in procs:
            p.join(60)
    return wall, np.sort(np.array(turns))


def processes_section(torch, abi, runtime, clients: int = 4, jobs_per_client: int = 50) -> dict:
    """The paper's setting: separate client processes sharing one GPU through
    the scheduler, in both designs of Sec. III: the scheduler server (UNIX
    socket, device engine) and the shared segment (host shared memory, each
    client decides). Clients run triad jobs with n log-uniform in [1M, 64M],
    all ready at once, on grants in one pool mapped by CUDA IPC. The same jobs
    run in one process through the trace runner, co-scheduled and
    exclusive-serial."""
    import multiprocessing as mp
    import tempfile
    n_jobs = clients * jobs_per_client
    tr = tg.trace_single_kind_t0(7, n_jobs, 1 << 20, 1 << 26, 16 << 30, f"triad{n_jobs}_t0_16GiB")
    pool = torch.empty(tr.budget, dtype=torch.uint8, device="cuda")
    ctx = mp.get_context("spawn")
    work = [[] for _ in range(clients)]
    for j in range(n_jobs):
        work[j % clients].append((int(tr.jobs["p0"][j]), int(tr.jobs["key"][j])))
    out = {"workload": tr.name, "clients": clients, "jobs": n_jobs}

    def summary(wall, turns):
        return {"jobs_per_s": n_jobs / wall, "ms": 1e3 * wall,
                "turnaround_p50_ms": 1e3 * float(turns[len(turns) // 2]),
                "turnaround_p99_ms": 1e3 * float(turns[min(len(turns) - 1, int(0.99 * len(turns)))])}

    sched = runtime.Scheduler(tr.budget, "first_fit", pool=pool)
    path = os.path.join(tempfile.mkdtemp(prefix="sg_bench_"), "sock")
    srv = abi.sg_server_start(sched.ctx, path)
    try:
        out["processes"] = summary(*_run_clients(ctx, "server", path, work))
    finally:
        abi.sg_server_stop(srv)
        sched.shutdown()
    name = _shm_name("proc")
    abi.sg_shm_unlink(name)
    h = abi.sg_shm_open(name, tr.budget, "first_fit")
    try:
        abi.sg_shm_set_pool(h, pool.data_ptr(), pool.numel())
        out["processes_shared_memory"] = summary(*_run_clients(ctx, "shm", name, work))
        st = abi.sg_shm_stats(h)
        assert st["used"] == 0 and st["grants"] == n_jobs, st
    finally:
        abi.sg_shm_close(h)
        abi.sg_shm_unlink(name)
    s = runtime.Scheduler(tr.budget, "first_fit", pool=pool)
    d_jobs, d_tab = runtime.to_device(tr.jobs), runtime.device_tables(tr)
    for nm, mode in (("one_process", abi.SG_RUN_SATURATED),
                     ("one_process_exclusive", abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE)):
        s.run_trace(d_jobs, d_tab, mode)
        rc, _, _, st = s.run_trace(d_jobs, d_tab, mode)
        assert rc == abi.SG_OK
        out[nm] = {"jobs_per_s": n_jobs / (st["makespan_ns"] * 1e-9), "ms": st["makespan_ns"] / 1e6}
    s.shutdown()
    del pool
    torch.cuda.empty_cache()
    return out


def client_server_section(torch, abi, runtime, reps: int = 300) -> dict:
    """The life-cycle stages from a separate client process, in both designs
    of Sec. III: through the scheduler server (UNIX socket; grants pushed by
    the server) and through the shared segment (the client decides under the
    file lock). The paper compares the two by their overhead."""
    import multiprocessing as mp
    import tempfile
    pool = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    sched = runtime.Scheduler(pool.numel(), "first_fit", pool=pool, max_tickets=reps + 16)
    path = os.path.join(tempfile.mkdtemp(prefix="sg_bench_"), "sock")
    srv = abi.sg_server_start(sched.ctx, path)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_latency_client, args=("server", path, reps, q))
    p.start()
    try:
        out = q.get(timeout=300)
    finally:
        p.join(30)
        abi.sg_server_stop(srv)
        sched.shutdown()
    out["note"] = ("client process -> server: declare + wait for the pushed grant; "
                   "release round trip (the release kernel runs after the reply)")
    name = _shm_name("lat")
    abi.sg_shm_unlink(name)
    h = abi.sg_shm_open(name, pool.numel(), "first_fit")
    try:
        p = ctx.Process(target=_latency_client, args=("shm", name, reps, q))
        p.start()
        try:
            shm = q.get(timeout=300)
        finally:
            p.join(30)
    finally:
        abi.sg_shm_close(h)
        abi.sg_shm_unlink(name)
    shm["note"] = "client process on the shared segment: declare (decided in the call) + wait; release"
    out["shared_memory"] = shm
    return out


def policies_section(torch, abi, runtime, prioritised=tg.KIND_SPMV) -> dict:
    """The four notification policies on the mixed trace (arrivals at t=0),
    one job kind prioritised (priority 0, the rest 1), as in the paper's
    workload experiment with one application prioritised."""
    tr = tg.trace_c2(saturated=True)
    jobs = tr.jobs.copy()
    jobs["prio"] = np.where(jobs["kind"] == prioritised, 0, 1)
    pool = torch.empty(tr.budget, dtype=torch.uint8, device="cuda")
    d_jobs, d_tab = runtime.to_device(jobs), runtime.device_tables(tr)
    out = {"prioritised": tg.KIND_NAMES[prioritised]}
    for pol in ("fifo", "first_fit", "prio_fifo", "prio_first_fit"):
        s = runtime.Scheduler(tr.budget, pol, pool=pool)
        s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED)
        rc, log, _, st = s.run_trace(d_jobs, d_tab, abi.SG_RUN_SATURATED)
        assert rc == abi.SG_OK
        rec = runtime.records(log)
        s.shutdown()
        pr = jobs["kind"] == prioritised
        wait = (rec["grant_t"].astype(np.int64) - rec["arrival_t"].astype(np.int64)) / 1e6
        out[pol] = {"makespan_ms": st["makespan_ns"] / 1e6,
                    "wait_mean_ms_prioritised": float(wait[pr].mean()),
                    "wait_mean_ms_others": float(wait[~pr].mean())}
    del pool
    torch.cuda.empty_cache()
    return out


def engine_section(torch, abi, runtime) -> dict:
    """Decision rate of the device engine alone: the replay of the 10,000-job
    batch and of the 100,000-request serving trace (one warp, logical clock)."""
    out = {}
    for name, tr, pol in (("tiny10k", tg.trace_c4(), "first_fit"),
                          ("serve100k_20000rps", tg.trace_c5(rate_per_s=20000.0), "first_fit")):
        n = len(tr)
        d_jobs = runtime.to_device(tr.jobs)
        d_log = torch.empty(n * abi.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        ws = torch.empty(abi.sg_replay_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        st = torch.zeros(4, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        abi.sg_replay(d_jobs.data_ptr(), n, tr.budget, 256, pol, 0, False, d_log.data_ptr(), ws.data_ptr(),
                      st.data_ptr(), stream.cuda_stream)
        e0.record(stream)
        abi.sg_replay(d_jobs.data_ptr(), n, tr.budget, 256, pol, 0, False, d_log.data_ptr(), ws.data_ptr(),
                      st.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        passes = int(st[2].item())
        events = 2 * n   # every job arrives and completes
        out[name] = {"jobs": n, "ms": ms, "events_per_s": events / (ms * 1e-3), "us_per_event": 1e3 * ms / events,
                     "passes": passes, "err": int(st[3].item())}
    return out


def kinds_section(torch, abi, runtime, reps: int = 3) -> dict:
    """Co-scheduled vs exclusive-serial makespan on the mixed trace's jobs of
    one kind, of two kinds, and of all three (arrivals at t=0, first fit):
    where co-scheduling pays on this GPU and where the kernels contend."""
    tr = tg.trace_c2(saturated=True)
    tab = runtime.device_tables(tr)
    s = runtime.Scheduler(tr.budget, "first_fit")
    ov = runtime.Scheduler(tr.budget, "first_fit", pool=s.pool, run_flags=abi.SG_RUNF_OVERLAP)
    out = {}
    for kinds in ((tg.KIND_TRIAD,), (tg.KIND_SPMV,), (tg.KIND_GEMM,), (tg.KIND_TRIAD, tg.KIND_SPMV),
                  (tg.KIND_TRIAD, tg.KIND_GEMM), (tg.KIND_SPMV, tg.KIND_GEMM),
                  (tg.KIND_TRIAD, tg.KIND_SPMV, tg.KIND_GEMM)):
        jobs = tr.jobs[np.isin(tr.jobs["kind"], kinds)].copy()
        d = runtime.to_device(jobs)
        ms = {}
        both = tg.KIND_SPMV in kinds and tg.KIND_GEMM in kinds
        for name, sch, mode in (("co", s, abi.SG_RUN_SATURATED), ("overlap", ov, abi.SG_RUN_SATURATED),
                                ("exclusive", s, abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE)):
            if name == "overlap" and not both:
                continue   # the start rule only separates SpMV from GEMM
            t = []
            for _ in range(reps):
                rc, _, _, st = sch.run_trace(d, tab, mode)
                assert rc == abi.SG_OK
                t.append(st["makespan_ns"] / 1e6)
            ms[name] = statistics.median(t)
        row = {"jobs": len(jobs), "co_ms": ms["co"], "exclusive_ms": ms["exclusive"],
               "ratio": ms["co"] / ms["exclusive"]}
        if both:
            row["overlap_ms"] = ms["overlap"]
        out["+".join(tg.KIND_NAMES[k] for k in kinds)] = row
    ov.shutdown()
    s.shutdown()
    return out


def mixed_plan_section(torch, abi, runtime, reps: int = 3) -> dict:
    """The mixed trace (t=0) run as one CUDA graph on the engine's replay plan:
    no host round trip and no admission at run time."""
    tr = tg.trace_c2(saturated=True)
    pool = torch.empty(tr.budget, dtype=torch.uint8, device="cuda")
    pl = runtime.Planned(pool, tr.jobs, runtime.device_tables(tr), "first_fit", budget=tr.budget)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pl.run_graph()
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        e0.record(stream)
        pl.run_graph()
        e1.record(stream)
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    pl.close()
    del pool
    torch.cuda.empty_cache()
    ms = statistics.median(t)
    return {"cuda_graph_ms": ms, "jobs_per_s": len(tr) / (ms * 1e-3)}


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batching and serving sections")
    ap.add_argument("--serving-requests", type=int, default=100_000)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    ws, rank, local = _dist_env()
    import torch
    from paper_1712_04495_b300 import abi, runtime
    torch.cuda.set_device(local)
    ops = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        ops = _torch_ops(torch.device("cuda", local))
    peaks = _peaks()

    # the project's autotuner picks the GEMM output tile of every shape the
    # workloads use (outside any timed region)
    shapes = sorted({(s_, s_, s_) for s_ in (64, 128, 256, 512, 1024, 2048, 4096, 8192)})
    scratch = torch.empty(600 << 20, dtype=torch.uint8, device="cuda")
    tuned = abi.sg_autotune_gemm(shapes, scratch.data_ptr(), scratch.numel(),
                                 torch.cuda.current_stream().cuda_stream)
    del scratch
    torch.cuda.empty_cache()

    # the job kernels timed alone, first: in the same burst conditions as the
    # measured peaks they are compared with, before the long runs heat the GPU
    # and its power cap lowers the clocks
    kr = kernel_roofline(torch, abi, runtime, peaks) if rank == 0 else None
    torch.cuda.empty_cache()

    trace = tg.trace_c2(saturated=True)
    n = len(trace)
    assert n == workload_config(1)["jobs"]
    sched = runtime.Scheduler(trace.budget, "first_fit")
    d_jobs = runtime.to_device(trace.jobs)
    d_tab = runtime.device_tables(trace)

    def step(mode=abi.SG_RUN_SATURATED, s=sched):
        rc, log, _, st = s.run_trace(d_jobs, d_tab, mode)
        if rc != abi.SG_OK:
            raise RuntimeError(f"sg_run_trace: {abi.sg_strerror(rc)} {st}")
        return st

    for _ in range(args.warmup):
        step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    elapsed, launches, stats = [], 0, []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        st = step()
        elapsed.append(st["elapsed_ns"] * 1e-9)
        launches += st["launches"]
        stats.append(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    if ws > 1:
        torch.distributed.barrier()
    secs = sum(elapsed)
    value, max_secs = aggregate(n * args.steps, secs, ws, ops)

    extra = {}
    if rank == 0:
        # policies side by side (same trace, same pool)
        ms = {"first_fit": statistics.median(s["makespan_ns"] for s in stats) / 1e6}
        fifo = runtime.Scheduler(trace.budget, "fifo", pool=sched.pool)
        sched_fifo = [step(s=fifo) for _ in range(5)]
        fifo.shutdown()
        ms["fifo"] = statistics.median(s["makespan_ns"] for s in sched_fifo) / 1e6
        # the runner starting SpMV and GEMM jobs side by side (SG_RUNF_OVERLAP)
        for name, pol in (("first_fit_overlap", "first_fit"), ("fifo_overlap", "fifo")):
            ov = runtime.Scheduler(trace.budget, pol, pool=sched.pool, run_flags=abi.SG_RUNF_OVERLAP)
            ms[name] = statistics.median(step(s=ov)["makespan_ns"] for _ in range(5)) / 1e6
            ov.shutdown()
        ser = [step(abi.SG_RUN_SATURATED | abi.SG_RUN_EXCLUSIVE) for _ in range(5)]
        ms["exclusive_serial"] = statistics.median(s["makespan_ns"] for s in ser) / 1e6
        extra["makespan_ms"] = ms
        extra["makespan_ratio_vs_serial"] = {k: ms[k] / ms["exclusive_serial"] for k in
                                             ("first_fit", "fifo", "first_fit_overlap", "fifo_overlap")}
        extra["wait_p50_ms"] = statistics.median(s["wait_p50_ns"] for s in stats) / 1e6
        extra["wait_p99_ms"] = statistics.median(s["wait_p99_ns"] for s in stats) / 1e6
        extra["turnaround_p99_ms"] = statistics.median(s["turnaround_p99_ns"] for s in stats) / 1e6
        extra["peak_used_gib"] = max(s["peak_used"] for s in stats) / 2 ** 30
        # the literal trace: Poisson arrivals at 200 jobs/s
        lit = tg.trace_c2(saturated=False)
        rc, _, _, st = sched.run_trace(runtime.to_device(lit.jobs), runtime.device_tables(lit),
                                       abi.SG_RUN_TIMED)
        stl = sched.run_trace(runtime.to_device(lit.jobs), runtime.device_tables(lit),
                              abi.SG_RUN_TIMED | abi.SG_RUN_EXCLUSIVE)[3]
        extra["poisson200"] = {"makespan_ms": st["makespan_ns"] / 1e6,
                               "jobs_per_s": n / (st["makespan_ns"] * 1e-9),
                               "wait_p50_ms": st["wait_p50_ns"] / 1e6, "wait_p99_ms": st["wait_p99_ns"] / 1e6,
                               "turnaround_p99_ms": st["turnaround_p99_ns"] / 1e6,
                               "exclusive_serial_makespan_ms": stl["makespan_ns"] / 1e6,
                               "arrival_span_ms": int(lit.jobs["arrival_ns"][-1]) / 1e6}
        # end to end: the same step through host buffers (copies inside the call)
        e2e_t = []
        for _ in range(max(2, args.steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, rec, _, st = sched.run_trace_host(trace.jobs, d_tab, abi.SG_RUN_SATURATED)
            e2e_t.append(time.perf_counter() - t0)
            assert rc == abi.SG_OK
        extra["e2e"] = {"value": n * len(e2e_t) / sum(e2e_t), "unit": "jobs/s",
                        "h2d_bytes_per_step": int(trace.jobs.nbytes),
                        "d2h_bytes_per_step": int(n * abi.RECORD_DTYPE.itemsize)}
        sched.shutdown()
        del sched
        torch.cuda.empty_cache()
        extra["kernels"] = kr
        extra["makespan_bound"] = makespan_bound(trace, kr, peaks, ms["exclusive_serial"])
        if not args.no_extras:
            extra["lifecycle"] = lifecycle_section(torch, abi, runtime)
            extra["client_server"] = client_server_section(torch, abi, runtime)
            extra["processes"] = processes_section(torch, abi, runtime)
            extra["policies"] = policies_section(torch, abi, runtime)
            extra["engine"] = engine_section(torch, abi, runtime)
            extra["kinds"] = kinds_section(torch, abi, runtime)
            extra["mixed_plan_graph"] = mixed_plan_section(torch, abi, runtime)
            extra["batching"] = batching_section(torch, abi, runtime)
            extra["serving"] = serving_section(torch, abi, runtime, args.serving_requests)
            extra["configs"] = configs_section(torch, abi, runtime)
        # the single kernel with the largest share of a step's ncu launch list
        # is the CSR SpMV (28.8% of a step's kernel time); the GEMM's 256 x 256
        # tile has 26.9% (30.0% over all its tiles), reported in kernels.gemm
        extra["roofline"] = {k: kr["spmv"][k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                        "traffic")}
        extra["roofline"]["kernel"] = kr["spmv"]["kernel"]
        extra["roofline"]["peak_source"] = peaks["source"] + " (copy bandwidth, kernel timed alone)"
        extra["roofline"]["target"] = kr["spmv"]["target"]
        extra["roofline"]["target_met"] = kr["spmv"]["target_met"]
        extra["roofline"]["gather_ceiling"] = kr["spmv"]["gather_ceiling"]
        extra["roofline"]["note"] = ("below the 0.70 target: bound by random x gathers (SM-to-crossbar request "
                                     "rate), not "
                                     "by HBM; HBM traffic equals the algorithmic bytes; gather_ceiling is the "
                                     "same gathers alone, measured in this run (spmv_frac = the SpMV's fraction "
                                     "of that rate); kernels.gemm has the tcgen05 GEMM")
        if not args.no_cpu_baseline:
            sample = stratified_samples(trace, 2)[0]
            d, e = oracle_sample(trace, sample)
            extra["cpu_baseline"] = {"value": d / e, "unit": "jobs/s", "cores": _oracle_threads(),
                                     "host_cpus": _threads(), "kind": "oracle", "seconds": e,
                                     "sample": _sample_desc(trace, sample, 2)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "jobs/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * max_secs / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64 admission; f32 triad/spmv; bf16 in, f32 acc gemm",
                "data": "synthetic",
                "config": workload_config(ws),
                "gpu_launches": launches, "clocks": clocks, "wall_s": wall,
                "autotune_gemm_tile": {str(sh[0]): abi.gemm_tile_name(w) for sh, w, _ in tuned}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
