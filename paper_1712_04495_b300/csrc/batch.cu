// Batching in one persistent grouped kernel.
//
// A batch of (typically thousands of tiny) jobs is admitted as a whole by the
// device engine: sg_replay on the declared durations gives each job its
// offset in the pool and its grant order (the plan). This kernel then runs
// the plan as a dataflow. Every job is a short program of phases (input
// generators, kernel, optional output digest); every phase is a set of
// chunks, the per-block bodies shared with the standalone kernels
// (tiles.cuh). Blocks pull chunks from one work queue; the block that
// finishes the last chunk of a phase enqueues the next phase, and the block
// that finishes a job makes each successor whose memory it was using one
// step closer to runnable. A job's chunks are enqueued only when every
// earlier job that used any byte of its extent has finished, so jobs that
// share memory never overlap in time. There is no host round trip and no
// launch per job.
//
// Admitting on the device instead (sg_batch_build_online): there is no plan.
// The batch's own engine holds every job declared at t = 0. One warp of the
// kernel (in a block of its own) owns that engine for the whole launch, so it
// reads the state through L1, as a replay does: it runs the first policy pass, then takes finished
// jobs from a completion ring in the order the workers finish them, releases
// each (post-free and its notification pass) and enqueues the first phase of
// every job the pass grants, at the offset the engine gave it. Admission and
// execution share the kernel.
//
// The work queue is a ring of exactly `total` slots (the chunk count of the
// whole batch, known in advance): slot i is written once, and its sequence
// word becomes i + 1 when the item is visible. A block claims the next slot
// with one atomic and waits (bounded) until it is filled; a block that
// claims a slot past the end has nothing left to do and leaves. All blocks
// are co-resident (cooperative launch), so a waiting block never keeps the
// producer of its slot from running.
#include <vector>

#include "engine.cuh"
#include "jobs.h"
#include "plan.h"
#include "tc.cuh"
#include "tiles.cuh"

namespace sg {
namespace {

constexpr uint64_t kBatchWaitNs = 20000000000ull;  // 20 s for one queue slot
// A kernel that allocates TMEM gets one block per SM, so each block holds
// four independent workers of kChunkThreads threads (named barriers 1..4),
// each with its own GEMM staging buffers and 128 of the SM's 512 TMEM columns.
constexpr uint32_t kGroups = 4;
constexpr uint32_t kBatchThreads = kGroups * kChunkThreads;
constexpr uint32_t kGemmSmem = 32 * 1024;           // per worker: A 16 KiB + B (<= 128 rows) 16 KiB
constexpr uint32_t kBatchSmem = kGroups * kGemmSmem + 1024;
constexpr uint32_t kBatchTmemCols = 512;
constexpr uint32_t kGemmBM = 128;
// Chunks one queue item carries, per phase: a tiny job's chunk is often
// less work than the queue round trips that hand it out. SpMV: chunks of
// kSpmvRowsChunk rows; triad and its generator: kTriadChunk elements; bf16
// generator: kBf16Chunk elements; SpMV generator: kFillChunk non-zeros.
constexpr uint64_t kSpmvChunksPerItem = 8;
constexpr uint64_t kTriadChunksPerItem = 4;
constexpr uint64_t kBf16ChunksPerItem = 8;
constexpr uint64_t kFillChunksPerItem = 4;

struct Item {
  uint32_t job, phase;
  uint64_t chunk;
};

struct BatchDev {
  const sg_job* jobs;
  uint64_t* offset;              // [n] grant offsets (the plan, or written at grant time)
  char* pool;
  const uint64_t* tables;
  uint64_t* keep;                // [n] output digests, or null
  const uint64_t* succ_ptr;      // [n + 1]
  const uint32_t* succ;
  uint32_t* dep;                 // [n] unfinished predecessors
  uint32_t* left;                // [n] unfinished chunks of the current phase
  Item* items;                   // [total]
  uint32_t* seq;                 // [total]
  unsigned long long* ctr;       // [0] head (claims), [1] tail (reservations), [2] jobs done
  uint32_t* err;
  uint64_t total;
  Eng eng;                       // the batch's engine when it admits on the device
  uint32_t online;
  uint32_t n;
  uint32_t* comp;                // [n] finished jobs, in finishing order (online)
  uint32_t* comp_seq;            // [n] slot r holds r + 1 once comp[r] is visible
  uint32_t* glist;               // [n] granted jobs, in grant order (online)
};

__host__ __device__ inline uint32_t gemm_bn_small(uint64_t n) { return n > 64 ? 128u : 64u; }

__host__ __device__ inline uint32_t job_phases(const sg_job& j, bool keep) {
  const uint32_t p = j.kind == SG_KIND_SPMV ? 4u : 2u;
  return p + (keep ? 1u : 0u);
}

__host__ __device__ inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// chunks of phase `ph` of job `j` (the digest phase comes last when kept)
__host__ __device__ inline uint64_t phase_chunks(const sg_job& j, uint32_t ph) {
  if (j.kind == SG_KIND_TRIAD) {
    if (ph <= 1) return cdiv(cdiv(j.p0, kTriadChunk), kTriadChunksPerItem);
    return cdiv(j.p0, kDigestChunk);
  }
  if (j.kind == SG_KIND_GEMM) {
    const uint64_t m = j.p0, n = j.p1, k = j.p2;
    if (ph == 0) return cdiv(cdiv(m * k, kBf16Chunk) + cdiv(n * k, kBf16Chunk), kBf16ChunksPerItem);
    if (ph == 1) return cdiv(m, kGemmBM) * cdiv(n, gemm_bn_small(n));
    return cdiv(m * n, kDigestChunk);
  }
  const uint64_t rows = j.p0, cap = j.p1;
  const uint64_t nch = cdiv(rows, kRowsPerScanChunk);
  switch (ph) {
    case 0: return nch + cdiv(cdiv(cap > 4 * rows ? cap : 4 * rows, kFillChunk), kFillChunksPerItem);
    case 1: return 1;
    case 2: return nch;
    case 3: return cdiv(rows, kSpmvRowsChunk * kSpmvChunksPerItem);
    default: return cdiv(rows, kDigestChunk);
  }
}

// ------------------------------------------------------------- queue ops
// Called by one thread: reserve and publish the chunks of one phase.
__device__ void push_phase(const BatchDev& B, uint32_t job, uint32_t ph) {
  const uint64_t cnt = phase_chunks(B.jobs[job], ph);
  st_gpu(B.left + job, (uint32_t)cnt);
  __threadfence();
  const uint64_t base = atomicAdd(&B.ctr[1], (unsigned long long)cnt);
  if (base + cnt > B.total) {
    atomicOr(B.err, ERR_CAP);
    return;
  }
  for (uint64_t i = 0; i < cnt; i++) {
    Item it;
    it.job = job;
    it.phase = ph;
    it.chunk = i;
    B.items[base + i] = it;
  }
  __threadfence();
  for (uint64_t i = 0; i < cnt; i++) atomicExch(B.seq + base + i, (uint32_t)(base + i + 1));
}

// The same, warp-wide (one full warp): the chunks of the phase are written
// and published by all 32 lanes.
__device__ void push_phase_warp(const BatchDev& B, uint32_t job, uint32_t ph) {
  const uint64_t cnt = phase_chunks(B.jobs[job], ph);
  unsigned long long base = 0;
  if (lane_id() == 0) {
    st_gpu(B.left + job, (uint32_t)cnt);
    __threadfence();
    base = atomicAdd(&B.ctr[1], (unsigned long long)cnt);
    if (base + cnt > B.total) atomicOr(B.err, ERR_CAP);
  }
  base = __shfl_sync(SG_FULL, base, 0);
  if (base + cnt > B.total) return;           // warp-uniform
  for (uint64_t i = lane_id(); i < cnt; i += 32) {
    Item it;
    it.job = job;
    it.phase = ph;
    it.chunk = i;
    B.items[base + i] = it;
  }
  __threadfence();                            // each lane's items before its sequence words
  for (uint64_t i = lane_id(); i < cnt; i += 32) st_gpu(B.seq + base + i, (uint32_t)(base + i + 1));
  __syncwarp();
}

// Online admission. The engine warp hands every job it grants to the
// block's other 31 warps: it appends the job to the batch's grant list (n
// entries, so nothing wraps) and bumps a shared-memory tail; they enqueue the
// jobs' first phases, so the engine's serial path only runs engine steps.
struct GrantQueue {                 // shared memory of the engine's block
  uint32_t tail, claim, done;
};

// bounded spin of one lane on a shared word until pred() holds; false = gave up
template <class Pred>
__device__ bool spin_until(const BatchDev& B, Pred pred) {
  uint64_t t0 = 0;
  unsigned ns = 32;
  for (uint32_t it = 0;; it++) {
    if (pred()) return true;
    if ((it & 15) == 15) {
      if (ld_gpu(B.err) != 0) return false;
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kBatchWaitNs) { atomicOr(B.err, ERR_LOCK); return false; }
    }
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
}

// the engine warp: give the jobs granted at ring positions [from, to) their
// offsets and queue them for the publishers (lane 0)
__device__ bool hand_over(const BatchDev& B, const Eng& E, GrantQueue* Q, uint32_t from, uint32_t to) {
  bool ok = true;
  if (lane_id() == 0) {
    for (uint32_t p = from; p < to && ok; p++) {
      const uint32_t j = eld(E, E.dev_ring + p % B.n);
      st_gpu(B.offset + j, eld(E, reinterpret_cast<const uint64_t*>(E.rec + j) + 3));   // sg_record.offset
      volatile GrantQueue* vq = Q;
      const uint32_t t = vq->tail;
      if (t >= B.n) { atomicOr(B.err, ERR_CAP); ok = false; break; }   // cannot happen: n grants
      st_gpu(B.glist + t, j);
      __threadfence();                        // offset and list entry before the tail moves
      vq->tail = t + 1;
    }
  }
  return __shfl_sync(SG_FULL, (int)ok, 0) != 0;
}

// The engine warp of an online batch (the only user of the batch's engine
// state during the launch).
__device__ void engine_service(const BatchDev& B, GrantQueue* Q) {
  const Eng E = eng_owned(B.eng);
  Sess s = sess_load(E);
  uint32_t from = s.ring_tail;
  policy_pass(E, s, globaltimer_ns(), nullptr, nullptr);
  bool ok = hand_over(B, E, Q, from, s.ring_tail);
  for (uint32_t r = 0; r < B.n && s.err == 0 && ok; r++) {
    uint32_t j = 0;
    if (lane_id() == 0) {                     // the r-th finished job
      ok = spin_until(B, [&] { return ld_gpu(B.comp_seq + r) == r + 1; });
      __threadfence();
      if (ok) j = ld_gpu(B.comp + r);
    }
    ok = __shfl_sync(SG_FULL, (int)ok, 0) != 0;
    j = __shfl_sync(SG_FULL, j, 0);
    if (!ok) break;
    from = s.ring_tail;
    op_release(E, s, j, 0, globaltimer_ns(), nullptr, nullptr);
    ok = hand_over(B, E, Q, from, s.ring_tail);
  }
  if (s.err && lane_id() == 0) atomicOr(B.err, s.err);
  sess_store(E, s);
  if (lane_id() == 0) {
    __threadfence_block();
    ((volatile GrantQueue*)Q)->done = 1;
  }
  __syncwarp();
}

// a publisher warp of the engine's block: enqueue the first phase of each
// queued grant until the engine warp is done
__device__ void publish_service(const BatchDev& B, GrantQueue* Q) {
  volatile GrantQueue* vq = Q;
  for (;;) {
    uint32_t c = 0;
    int have = 0;
    if (lane_id() == 0) {
      c = atomicAdd(&Q->claim, 1u);
      bool ok = spin_until(B, [&] { return c < vq->tail || vq->done; });
      have = ok && c < vq->tail;
    }
    have = __shfl_sync(SG_FULL, have, 0);
    c = __shfl_sync(SG_FULL, c, 0);
    if (!have) break;
    __threadfence();
    push_phase_warp(B, ld_gpu(B.glist + c), 0);
  }
}

// Claim the next slot of the queue (one thread).
__device__ __forceinline__ uint64_t claim(const BatchDev& B) { return atomicAdd(&B.ctr[0], 1ull); }

// The item in claimed slot pos, once published: 1 = item in *out, 0 =
// nothing left, -1 = gave up.
__device__ int fetch(const BatchDev& B, uint64_t pos, Item* out) {
  if (pos >= B.total) return 0;
  const uint32_t want = (uint32_t)(pos + 1);
  uint64_t t0 = 0;
  unsigned ns = 32;
  for (uint32_t it = 0;; it++) {
    if (ld_gpu(B.seq + pos) == want) break;
    if ((it & 15) == 15) {
      if (ld_gpu(B.err) != 0) return -1;
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kBatchWaitNs) {
        atomicOr(B.err, ERR_LOCK);
        return -1;
      }
    }
    __nanosleep(ns);
    if (ns < 2048) ns <<= 1;
  }
  __threadfence();
  const uint64_t* src = reinterpret_cast<const uint64_t*>(B.items + pos);
  uint64_t w0 = ld_gpu(src), w1 = ld_gpu(src + 1);
  out->job = (uint32_t)w0;
  out->phase = (uint32_t)(w0 >> 32);
  out->chunk = w1;
  return 1;
}

// ---------------------------------------------------------- GEMM chunk
// One 128 x BNB output tile of C = A Bt^T with the operands staged by the
// worker's threads (plain 16-byte loads into the 128-byte swizzled layout a
// TMA load would produce), one tcgen05.mma group per 64-wide k-block, the
// accumulator in the worker's TMEM columns, and a masked epilogue. Any M, N;
// K % 8 == 0.
template <uint32_t BNB, class G>
__device__ bool gemm_chunk(const G& g, const uint16_t* __restrict__ A, const uint16_t* __restrict__ Bt,
                           float* __restrict__ C, uint32_t M, uint32_t N, uint32_t K, uint64_t tile, uint32_t sa,
                           uint32_t tmem, uint32_t mbar, uint32_t& mphase, volatile uint32_t* abort, int* vote) {
  const uint32_t nt = (N + BNB - 1) / BNB;
  const uint32_t m0 = (uint32_t)(tile / nt) * kGemmBM, n0 = (uint32_t)(tile % nt) * BNB;
  const uint32_t sb = sa + kGemmBM * 128;
  const uint32_t kbn = (K + 63) / 64;
  constexpr uint32_t kIdesc = idesc_bf16(kGemmBM, BNB);
  bool ok = true;
  for (uint32_t kb = 0; kb < kbn; kb++) {
    for (uint32_t idx = g.t(); idx < (kGemmBM + BNB) * 8; idx += kChunkThreads) {
      const bool is_a = idx < kGemmBM * 8;
      const uint32_t r = (is_a ? idx : idx - kGemmBM * 8) >> 3, c = idx & 7;
      const uint32_t k = kb * 64 + c * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (is_a) {
        if (m0 + r < M && k < K) v = *reinterpret_cast<const uint4*>(A + (uint64_t)(m0 + r) * K + k);
      } else {
        if (n0 + r < N && k < K) v = *reinterpret_cast<const uint4*>(Bt + (uint64_t)(n0 + r) * K + k);
      }
      const uint32_t dst = (is_a ? sa : sb) + r * 128 + ((c ^ (r & 7)) << 4);
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(v.x), "r"(v.y), "r"(v.z),
                   "r"(v.w)
                   : "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor core
    g.sync();
    if (g.t() == 0) {
      tc_fence_after();
#pragma unroll
      for (uint32_t kk = 0; kk < 4; kk++)
        mma_bf16(tmem, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), kIdesc, (kb | kk) != 0);
      mma_commit(mbar);
    }
    // every thread waits for the MMAs: the next k-block overwrites the operands
    const bool done = mbar_wait(mbar, mphase, abort);
    mphase ^= 1u;
    tc_fence_after();
    if (g.t() == 0) *vote = 1;
    g.sync();
    if (!done) *vote = 0;
    g.sync();
    const bool all = *vote != 0;
    g.sync();
    if (!all) { ok = false; break; }
  }
  if (ok) {
    const uint32_t warp = g.t() >> 5, lane = g.t() & 31;
    const uint32_t q = warp & 3u, half = warp >> 2;   // the group's warps start at a multiple of 4
    const uint32_t row = m0 + q * 32 + lane;
    for (uint32_t c = half * (BNB / 64); c < (half + 1) * (BNB / 64); c++) {
      if (n0 + c * 32 >= N) break;
      uint32_t r[32];
      tmem_ld_32cols(tmem + ((q * 32u) << 16) + c * 32, r);
      if (row < M) {
        float* crow = C + (uint64_t)row * N + n0 + c * 32;
#pragma unroll
        for (int v = 0; v < 32; v++)
          if (n0 + c * 32 + v < N) crow[v] = __uint_as_float(r[v]);
      }
    }
  }
  tc_fence_before();
  g.sync();
  return ok;
}

// ---------------------------------------------------------------- kernel
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch(BatchDev B) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t T[kGroups][64];
  __shared__ uint32_t T32[kGroups][64];
  __shared__ uint64_t red[kGroups][kChunkThreads / 32 + 1];
  __shared__ uint64_t carry[kGroups];
  __shared__ Item cur[kGroups];
  __shared__ int action[kGroups];
  __shared__ uint32_t s_last[kGroups];
  __shared__ int vote[kGroups];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[kGroups];
  __shared__ volatile uint32_t s_abort;
  __shared__ GrantQueue gq;

  const uint32_t gi = threadIdx.x / kChunkThreads;
  const SubGroup g{gi * kChunkThreads, 1u + gi};
  const uint32_t sa = ((smem_u32(smem_raw) + 1023u) & ~1023u) + gi * kGemmSmem;
  if (threadIdx.x == 0) {
    for (uint32_t k = 0; k < kGroups; k++) mbar_init(smem_u32(&mbar[k]), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kBatchTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base + gi * (kBatchTmemCols / kGroups);
  uint32_t mphase = 0;
  // admitting on the device: block 0 serves the engine (warp 0) and
  // publishes what it grants (the other warps); no chunk work shares the L1
  // that holds the engine state
  const bool service = B.online && blockIdx.x == 0;
  if (service) {
    if (threadIdx.x == 0) gq.tail = gq.claim = gq.done = 0;
    __syncthreads();
    if (threadIdx.x < 32) engine_service(B, &gq);
    else publish_service(B, &gq);
  }

  // Thread 0 of a worker claims its next slot as soon as it has its current
  // item, so the claim's round trip overlaps the item's work. A claimed slot
  // is waited for only after the current item is done, as before: every
  // worker holds at most one slot that is not yet published.
  uint64_t next_slot = 0;
  bool have_next = false;
  for (; !service;) {
    if (g.t() == 0) {
      const uint64_t pos = have_next ? next_slot : claim(B);
      action[gi] = fetch(B, pos, &cur[gi]);
      have_next = action[gi] == 1;
      if (have_next) next_slot = claim(B);
    }
    g.sync();
    if (action[gi] != 1) break;
    const Item it = cur[gi];
    const sg_job& job = B.jobs[it.job];
    char* base = B.pool + ld_gpu(B.offset + it.job);
    const bool keep = B.keep != nullptr;
    const uint32_t nph = job_phases(job, keep);
    const bool digest = keep && it.phase == nph - 1;
    bool ok = true;
    if (job.kind == SG_KIND_TRIAD) {
      const uint64_t n = job.p0;
      float* a = (float*)base;
      float* b = a + n;
      float* c = b + n;
      const int vec = (n & 3) == 0;            // b and c 16-byte aligned (the grant is)
      if (digest) {
        digest_chunk(g, (const uint32_t*)a, n, B.keep + it.job, it.chunk);
      } else {
        const uint64_t c1 = cdiv(n, kTriadChunk);
        for (uint64_t q = it.chunk * kTriadChunksPerItem; q < c1 && q < (it.chunk + 1) * kTriadChunksPerItem; q++) {
          if (it.phase == 0) gen_triad_chunk(g, b, c, n, stream_key(job.key, 1), stream_key(job.key, 2), vec, q);
          else triad_chunk(g, a, b, c, 3.0f, n, vec, q);
        }
      }
    } else if (job.kind == SG_KIND_GEMM) {
      const uint32_t m = (uint32_t)job.p0, n = (uint32_t)job.p1, k = job.p2;
      const GemmLayoutHD L = gemm_layout_hd(m, n, k);
      uint16_t* A = (uint16_t*)(base + L.A);
      uint16_t* Bt = (uint16_t*)(base + L.B);
      float* C = (float*)(base + L.C);
      if (digest) {
        digest_chunk(g, (const uint32_t*)C, (uint64_t)m * n, B.keep + it.job, it.chunk);
      } else if (it.phase == 0) {
        const uint64_t ca = cdiv((uint64_t)m * k, kBf16Chunk), c1 = ca + cdiv((uint64_t)n * k, kBf16Chunk);
        for (uint64_t q = it.chunk * kBf16ChunksPerItem; q < c1 && q < (it.chunk + 1) * kBf16ChunksPerItem; q++) {
          if (q < ca) gen_bf16_chunk(g, A, (uint64_t)m * k, stream_key(job.key, 1), q);
          else gen_bf16_chunk(g, Bt, (uint64_t)n * k, stream_key(job.key, 2), q - ca);
        }
      } else if (gemm_bn_small(n) == 128) {
        ok = gemm_chunk<128>(g, A, Bt, C, m, n, k, it.chunk, sa, tmem, smem_u32(&mbar[gi]), mphase, &s_abort,
                             &vote[gi]);
      } else {
        ok = gemm_chunk<64>(g, A, Bt, C, m, n, k, it.chunk, sa, tmem, smem_u32(&mbar[gi]), mphase, &s_abort,
                            &vote[gi]);
      }
    } else {
      const uint64_t rows = job.p0, cap = job.p1;
      const SpmvLayoutHD L = spmv_layout_hd(rows, cap);
      uint64_t* scan = (uint64_t*)(base + L.scan);
      const uint64_t lk = stream_key(job.key, 1);
      uint8_t* lens = (uint8_t*)(base + L.y);   // row lengths, in y until the SpMV writes it
      if (it.phase == 0 && it.chunk < L.nchunks) {
        if (g.t() < 64) {
          const uint64_t t = B.tables[64ull * job.p2 + g.t()];
          T[gi][g.t()] = t;
          T32[gi][g.t()] = table_u32(t);
        }
        g.sync();
      }
      if (digest) {
        digest_chunk(g, (const uint32_t*)(base + L.y), rows, B.keep + it.job, it.chunk);
      } else if (it.phase == 0) {
        if (it.chunk < L.nchunks) spmv_chunk_sum(g, T[gi], T32[gi], lk, rows, lens, scan, it.chunk, red[gi]);
        else {
          const uint64_t f1 = cdiv(cap > 4 * rows ? cap : 4 * rows, kFillChunk);
          const uint64_t f0 = (it.chunk - L.nchunks) * kFillChunksPerItem;
          for (uint64_t q = f0; q < f1 && q < f0 + kFillChunksPerItem; q++)
            spmv_fill_chunk(g, (int32_t*)(base + L.col), (float*)(base + L.val), (float*)(base + L.x), cap, rows,
                            stream_key(job.key, 2), stream_key(job.key, 3), stream_key(job.key, 4), q);
        }
      } else if (it.phase == 1) {
        spmv_scan(g, scan, L.nchunks, red[gi], &carry[gi]);
      } else if (it.phase == 2) {
        if (L.ptr64)
          spmv_row_ptr_chunk<SubGroup, int64_t>(g, lens, rows, scan, L.nchunks, (int64_t*)(base + L.row_ptr),
                                                cap, B.err, it.chunk, red[gi]);
        else
          spmv_row_ptr_chunk<SubGroup, int32_t>(g, lens, rows, scan, L.nchunks, (int32_t*)(base + L.row_ptr),
                                                cap, B.err, it.chunk, red[gi]);
      } else {
        const uint64_t c1 = cdiv(rows, kSpmvRowsChunk);
        for (uint64_t c = it.chunk * kSpmvChunksPerItem; c < c1 && c < (it.chunk + 1) * kSpmvChunksPerItem; c++) {
          if (L.ptr64)
            spmv_chunk<SubGroup, int64_t, XLoadL2>(g, (const int64_t*)(base + L.row_ptr), (const int32_t*)(base + L.col),
                                          (const float*)(base + L.val), XLoadL2{(const float*)(base + L.x)},
                                          (float*)(base + L.y), rows, 1, c);
          else
            spmv_chunk<SubGroup, int32_t, XLoadL2>(g, (const int32_t*)(base + L.row_ptr), (const int32_t*)(base + L.col),
                                          (const float*)(base + L.val), XLoadL2{(const float*)(base + L.x)},
                                          (float*)(base + L.y), rows, 1, c);
        }
      }
    }
    if (!ok) {
      if (g.t() == 0) atomicOr(B.err, ERR_ITEM);
      break;
    }
    // completion: the worker that finishes a phase enqueues the next one; the
    // one that finishes a job frees its memory for the jobs waiting on it
    g.sync();
    if (g.t() == 0) {
      __threadfence();
      s_last[gi] = atomicSub(B.left + it.job, 1u) == 1u;
    }
    g.sync();
    if (s_last[gi]) {
      __threadfence();
      if (it.phase + 1 < nph) {
        if (g.t() < 32) push_phase_warp(B, it.job, it.phase + 1);
      } else if (B.online) {
        if (g.t() == 0) {                             // hand the job to the engine warp
          const uint64_t r = atomicAdd(&B.ctr[3], 1ull);
          st_gpu(B.comp + r, it.job);
          __threadfence();
          atomicExch(B.comp_seq + r, (uint32_t)(r + 1));
          atomicAdd(&B.ctr[2], 1ull);
        }
      } else {
        for (uint64_t e = B.succ_ptr[it.job] + g.t(); e < B.succ_ptr[it.job + 1]; e += kChunkThreads) {
          const uint32_t s2 = B.succ[e];
          if (atomicSub(B.dep + s2, 1u) == 1u) push_phase(B, s2, 0);
        }
        if (g.t() == 0) atomicAdd(&B.ctr[2], 1ull);
      }
    }
    g.sync();
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kBatchTmemCols)
                 : "memory");
  }
}

}  // namespace
}  // namespace sg

using namespace sg;

namespace {

bool batch_kernel_attributes() {
  bool ok = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) ==
            cudaSuccess;
  // the smallest shared-memory split that holds the staging buffers: the
  // rest is L1 for the chunk bodies (10,000 tiny jobs: 9.2 ms, against
  // 10.7 ms with the largest split)
  ok &= cudaFuncSetAttribute(k_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxL1) == cudaSuccess;
  return ok;
}

// one block (four workers) per SM: a kernel that allocates TMEM gets one
int batch_grid(uint64_t total) {
  int grid = num_sms();
  if ((uint64_t)grid * kGroups > total && total > 0) grid = (int)((total + kGroups - 1) / kGroups);
  return grid;
}

// the job checks both builds make
int batch_job_ok(const sg_job& jb, const uint64_t* tables_dev) {
  if (jb.kind > SG_KIND_GEMM) return SG_ERR_INVALID;
  if (jb.kind == SG_KIND_GEMM && (jb.p2 == 0 || jb.p2 % 8 || jb.p0 == 0 || jb.p1 == 0)) return SG_ERR_INVALID;
  if (jb.kind == SG_KIND_SPMV && (!tables_dev || jb.p0 == 0 || jb.p0 > 0xFFFFFFFFull)) return SG_ERR_INVALID;
  if (jb.kind == SG_KIND_TRIAD && jb.p0 == 0) return SG_ERR_INVALID;
  return SG_OK;
}

}  // namespace

struct sg_batch {
  char* dev = nullptr;           // one allocation: every device array below
  BatchDev d{};
  uint32_t n = 0, granted = 0;
  int grid = 0;
  // admitting on the device
  bool online = false;
  uint64_t budget = 0, granule = 256;
  uint32_t policy = 0;
  // launch-time initial state, kept on the device
  uint32_t* dep0 = nullptr;
  uint32_t* left0 = nullptr;
  uint64_t init_items = 0;
  Item* items0 = nullptr;
};

extern "C" int sg_batch_build(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                              const uint64_t* tables_dev, const sg_record* plan, uint64_t* keep_dev,
                              sg_batch** out) {
  if (!out || !dev_pool || (!jobs && n) || (!plan && n)) return SG_ERR_INVALID;
  *out = nullptr;
  PlanDeps pd;
  if (!plan_deps(jobs, n, plan, pool_bytes, &pd)) return SG_ERR_INVALID;
  const bool keep = keep_dev != nullptr;
  std::vector<uint8_t> granted(n, 0);
  uint64_t total = 0;
  for (uint32_t j : pd.order) {
    const sg_job& jb = jobs[j];
    if (batch_job_ok(jb, tables_dev) != SG_OK) return SG_ERR_INVALID;
    granted[j] = 1;
    for (uint32_t ph = 0; ph < job_phases(jb, keep); ph++) total += phase_chunks(jb, ph);
  }
  // initial state: predecessor counts; phase-0 chunks of jobs with none
  std::vector<uint32_t> dep0(n, 0), left0(n, 0);
  std::vector<Item> items0;
  for (uint32_t j = 0; j < n; j++) dep0[j] = (uint32_t)(pd.pred_ptr[j + 1] - pd.pred_ptr[j]);
  for (uint32_t j : pd.order) {
    if (dep0[j] != 0) continue;
    const uint64_t cnt = phase_chunks(jobs[j], 0);
    left0[j] = (uint32_t)cnt;
    for (uint64_t c = 0; c < cnt; c++) items0.push_back(Item{j, 0u, c});
  }
  if (total > 0xFFFFFFF0ull) return SG_ERR_CAPACITY;
  auto a256 = [](uint64_t x) { return (x + 255) / 256 * 256; };
  const uint64_t nn = n ? n : 1, tt = total ? total : 1;
  uint64_t o = 0;
  const uint64_t o_jobs = o; o += a256(sizeof(sg_job) * nn);
  const uint64_t o_off = o; o += a256(8 * nn);
  const uint64_t o_sp = o; o += a256(8 * (nn + 1));
  const uint64_t o_s = o; o += a256(4 * (pd.succ.size() + 1));
  const uint64_t o_dep = o; o += a256(4 * nn);
  const uint64_t o_left = o; o += a256(4 * nn);
  const uint64_t o_dep0 = o; o += a256(4 * nn);
  const uint64_t o_left0 = o; o += a256(4 * nn);
  const uint64_t o_items = o; o += a256(sizeof(Item) * tt);
  const uint64_t o_items0 = o; o += a256(sizeof(Item) * (items0.size() + 1));
  const uint64_t o_seq = o; o += a256(4 * tt);
  const uint64_t o_ctr = o; o += 256;
  const uint64_t o_err = o; o += 256;
  sg_batch* b = new sg_batch();
  if (cudaMalloc(&b->dev, o) != cudaSuccess) {
    delete b;
    return SG_ERR_CUDA;
  }
  char* d = b->dev;
  std::vector<uint64_t> off(nn, 0);
  for (uint32_t j = 0; j < n; j++) off[j] = plan[j].offset;
  bool okc = true;
  okc &= cudaMemcpy(d + o_jobs, jobs, sizeof(sg_job) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(d + o_off, off.data(), 8 * n, cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(d + o_sp, pd.succ_ptr.data(), 8 * (n + 1), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!pd.succ.empty())
    okc &= cudaMemcpy(d + o_s, pd.succ.data(), 4 * pd.succ.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(d + o_dep0, dep0.data(), 4 * n, cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(d + o_left0, left0.data(), 4 * n, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!items0.empty())
    okc &= cudaMemcpy(d + o_items0, items0.data(), sizeof(Item) * items0.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  okc &= batch_kernel_attributes();
  if (!okc) {
    cudaFree(b->dev);
    delete b;
    return SG_ERR_CUDA;
  }
  b->n = n;
  b->granted = (uint32_t)pd.order.size();
  b->grid = batch_grid(total);
  BatchDev& B = b->d;
  B.jobs = (const sg_job*)(d + o_jobs);
  B.offset = (uint64_t*)(d + o_off);
  B.pool = (char*)dev_pool;
  B.tables = tables_dev;
  B.keep = keep_dev;
  B.succ_ptr = (const uint64_t*)(d + o_sp);
  B.succ = (const uint32_t*)(d + o_s);
  B.dep = (uint32_t*)(d + o_dep);
  B.left = (uint32_t*)(d + o_left);
  B.items = (Item*)(d + o_items);
  B.seq = (uint32_t*)(d + o_seq);
  B.ctr = (unsigned long long*)(d + o_ctr);
  B.err = (uint32_t*)(d + o_err);
  B.total = total;
  b->dep0 = (uint32_t*)(d + o_dep0);
  b->left0 = (uint32_t*)(d + o_left0);
  b->items0 = (Item*)(d + o_items0);
  b->init_items = items0.size();
  *out = b;
  return SG_OK;
}

extern "C" int sg_batch_build_online(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                                     const uint64_t* tables_dev, uint32_t policy, uint64_t* keep_dev,
                                     sg_batch** out) {
  if (!out || !dev_pool || (!jobs && n) || policy > SG_POLICY_PRIO_FIRST_FIT) return SG_ERR_INVALID;
  *out = nullptr;
  const uint64_t granule = 256;
  const uint64_t budget = pool_bytes / granule * granule;
  if (budget / granule > kKeyNeedMask) return SG_ERR_INVALID;
  const bool keep = keep_dev != nullptr;
  uint64_t total = 0;
  for (uint32_t j = 0; j < n; j++) {
    const sg_job& jb = jobs[j];
    if (batch_job_ok(jb, tables_dev) != SG_OK) return SG_ERR_INVALID;
    if ((jb.need + granule - 1) / granule * granule > budget) return SG_ERR_TOO_LARGE;   // would never run
    if (jb.prio < -32768 || jb.prio > 32767) return SG_ERR_INVALID;
    for (uint32_t ph = 0; ph < job_phases(jb, keep); ph++) total += phase_chunks(jb, ph);
  }
  if (total > 0xFFFFFFF0ull) return SG_ERR_CAPACITY;
  auto a256 = [](uint64_t x) { return (x + 255) / 256 * 256; };
  const uint64_t nn = n ? n : 1, tt = total ? total : 1;
  uint64_t o = 0;
  const uint64_t o_jobs = o; o += a256(sizeof(sg_job) * nn);
  const uint64_t o_off = o; o += a256(8 * nn);
  const uint64_t o_left = o; o += a256(4 * nn);
  const uint64_t o_items = o; o += a256(sizeof(Item) * tt);
  const uint64_t o_seq = o; o += a256(4 * tt);
  const uint64_t o_ctr = o; o += 256;
  const uint64_t o_err = o; o += 256;
  const uint64_t o_comp = o; o += a256(4 * nn);
  const uint64_t o_cseq = o; o += a256(4 * nn);
  const uint64_t o_glist = o; o += a256(4 * nn);
  const uint64_t o_eng = o; o += a256(batch_engine_bytes((uint32_t)nn));
  sg_batch* b = new sg_batch();
  if (cudaMalloc(&b->dev, o) != cudaSuccess) {
    delete b;
    return SG_ERR_CUDA;
  }
  char* d = b->dev;
  bool okc = n == 0 || cudaMemcpy(d + o_jobs, jobs, sizeof(sg_job) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= batch_kernel_attributes();
  if (!okc) {
    cudaFree(b->dev);
    delete b;
    return SG_ERR_CUDA;
  }
  b->n = n;
  b->granted = n;
  b->grid = batch_grid(total) + 1;                   // block 0 serves the engine
  if (b->grid > num_sms()) b->grid = num_sms();
  b->online = true;
  b->budget = budget;
  b->granule = granule;
  b->policy = policy;
  BatchDev& B = b->d;
  B.jobs = (const sg_job*)(d + o_jobs);
  B.offset = (uint64_t*)(d + o_off);
  B.pool = (char*)dev_pool;
  B.tables = tables_dev;
  B.keep = keep_dev;
  B.left = (uint32_t*)(d + o_left);
  B.items = (Item*)(d + o_items);
  B.seq = (uint32_t*)(d + o_seq);
  B.ctr = (unsigned long long*)(d + o_ctr);
  B.err = (uint32_t*)(d + o_err);
  B.total = total;
  B.eng = batch_engine_at(d + o_eng, (uint32_t)nn);
  B.comp = (uint32_t*)(d + o_comp);
  B.comp_seq = (uint32_t*)(d + o_cseq);
  B.glist = (uint32_t*)(d + o_glist);
  B.online = 1;
  B.n = (uint32_t)nn;
  *out = b;
  return SG_OK;
}

__global__ void k_batch_seed(uint32_t* seq, uint64_t init, uint64_t total, unsigned long long* ctr, uint32_t* err) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < total; i += stride) seq[i] = i < init ? (uint32_t)(i + 1) : 0u;
  if (tid == 0) {
    ctr[0] = 0;
    ctr[1] = init;
    ctr[2] = 0;
    ctr[3] = 0;
    *err = 0;
  }
}

extern "C" int sg_batch_launch(sg_batch* b, void* stream) {
  if (!b) return SG_ERR_INVALID;
  if (b->d.total == 0) return SG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t n = b->n;
  if (b->online) {
    if (batch_engine_start(b->d.eng, b->d.jobs, n, b->budget, b->granule, b->policy, st) != SG_OK ||
        cudaMemsetAsync(b->d.comp_seq, 0, 4ull * n, st) != cudaSuccess)
      return SG_ERR_CUDA;
  } else if (cudaMemcpyAsync(b->d.dep, b->dep0, 4ull * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
             cudaMemcpyAsync(b->d.left, b->left0, 4ull * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    return SG_ERR_CUDA;
  }
  if (b->init_items &&
      cudaMemcpyAsync(b->d.items, b->items0, sizeof(Item) * b->init_items, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return SG_ERR_CUDA;
  if (b->d.keep && cudaMemsetAsync(b->d.keep, 0, 8ull * n, st) != cudaSuccess) return SG_ERR_CUDA;
  k_batch_seed<<<256, 256, 0, st>>>(b->d.seq, b->init_items, b->d.total, b->d.ctr, b->d.err);
  if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
  void* args[] = {(void*)&b->d};
  const cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)k_batch, dim3(b->grid), dim3(kBatchThreads), args, kBatchSmem, st);
  return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

extern "C" int sg_batch_status(sg_batch* b, uint64_t* jobs_done, uint32_t* err_flags) {
  if (!b) return SG_ERR_INVALID;
  unsigned long long c[3] = {0, 0, 0};
  uint32_t e = 0;
  if (cudaMemcpy(c, b->d.ctr, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&e, b->d.err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SG_ERR_CUDA;
  if (jobs_done) *jobs_done = c[2];
  if (err_flags) *err_flags = e;
  return (c[2] == b->granted && e == 0) ? SG_OK : SG_ERR_DEVICE;
}

extern "C" int sg_batch_records(sg_batch* b, sg_record* out) {
  if (!b || !out || !b->online) return SG_ERR_INVALID;
  if (b->n && cudaMemcpy(out, b->d.eng.rec, sizeof(sg_record) * b->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SG_ERR_CUDA;
  return SG_OK;
}

extern "C" int sg_batch_info(const sg_batch* b, uint64_t* jobs, uint64_t* chunks, uint64_t* blocks) {
  if (!b) return SG_ERR_INVALID;
  if (jobs) *jobs = b->granted;
  if (chunks) *chunks = b->d.total;
  if (blocks) *blocks = (uint64_t)b->grid * kGroups;   // workers
  return SG_OK;
}

extern "C" int sg_batch_destroy(sg_batch* b) {
  if (!b) return SG_ERR_INVALID;
  if (b->dev) cudaFree(b->dev);
  delete b;
  return SG_OK;
}
