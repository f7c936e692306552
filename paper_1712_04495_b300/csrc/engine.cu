// Host runtime of the co-scheduler and the engine's kernels.
//
// The engine state (Sec. III-B shared data) is device memory allocated once
// in sg_init. Every life-cycle call of Sec. IV becomes a one-warp control
// kernel that takes the device lock, runs the operation and its policy pass
// (Sec. V), and publishes the resulting grants through host-mapped memory:
// a per-ticket record whose status word is written last, and a ring of
// granted tickets -- the in-process stand-in for the paper's signal to a
// waiting client. Jobs launched by the library release their ticket from
// the last block of their final kernel, so wake-on-release needs no host
// round trip.
#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "engine.cuh"
#include "jobs.h"
#include "phases.h"

using namespace sg;

static_assert(kKindTriad == SG_KIND_TRIAD && kKindSpmv == SG_KIND_SPMV && kKindGemm == SG_KIND_GEMM,
              "runner kinds follow the ABI's job kinds");

namespace {

// the runner's queue of a job kind (unknown kinds go with the triads; their
// launch fails and their memory is given back)
inline int kind_of(const sg_job& j) { return j.kind < kKinds ? (int)j.kind : kKindTriad; }

// ------------------------------------------------------------- kernels
__global__ void k_eng_reset(Eng E, uint64_t budget, uint64_t granule, uint32_t policy, uint32_t flags,
                            uint32_t cap, uint64_t qt_len) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < cap; i += stride) {
    E.status[i] = ST_PENDING;
    E.blk_done[i] = 0;
  }
  for (uint64_t i = tid; i < E.qcap; i += stride) E.qa[i] = kNone;
  for (uint64_t i = tid; i < qt_len; i += stride) E.qt[i] = kInf;
  if (tid == 0) {
    EngHdr* h = E.hdr;
    h->budget = budget;
    h->granule = granule;
    h->used = 0;
    h->seq = 0;
    h->peak_used = 0;
    h->frag_waits = 0;
    h->passes = 0;
    h->policy = policy;
    h->flags = flags;
    h->cap = cap;
    h->lock = 0;
    h->err = 0;
    h->n_ext = budget > 0 ? 1 : 0;
    h->q_len = 0;
    h->ring_tail = 0;
    h->n_done = 0;
    h->q_begin = 0;
    h->q_end = 0;
    E.ext_off[0] = 0;
    E.ext_len[0] = budget;
    h->max_ext = budget;
  }
}

// Declare tickets [first, first + count): their needs come from `jobs`
// (ticket i = job i) or, for a single ticket, from (need, prio).
__global__ void k_declare(Eng shared, uint32_t first, uint32_t count, const sg_job* jobs, uint64_t need,
                          int32_t prio, uint32_t exclusive) {
  if (threadIdx.x >= 32) return;
  const Eng E = eng_live(shared);
  for (uint32_t t = first; t < first + count; t++) {
    if (!eng_lock(E)) return;
    Sess s = sess_load(E);
    uint64_t raw = jobs ? jobs[t].need : need;
    int32_t pr = jobs ? (int32_t)jobs[t].prio : prio;
    uint64_t g = exclusive ? s.budget : round_need(raw, s.granule);
    if (lane_id() == 0) {
      st_gpu(E.need_g + t, g);
      st_gpu(E.need_raw + t, exclusive ? s.budget : raw);
      st_gpu(E.prio + t, pr);
      st_gpu(E.blk_done + t, 0u);
    }
    __syncwarp();
    op_declare(E, s, t, globaltimer_ns(), -1, nullptr, nullptr, nullptr);
    sess_store(E, s);
    eng_unlock(E);
  }
}

__global__ void k_release(Eng E, uint32_t t, uint64_t bytes) {
  if (threadIdx.x >= 32) return;
  eng_release_locked(E, t, bytes);
}

__global__ void k_cancel(Eng shared, uint32_t t) {
  if (threadIdx.x >= 32) return;
  const Eng E = eng_live(shared);
  if (!eng_lock(E)) return;
  Sess s = sess_load(E);
  op_cancel(E, s, t, globaltimer_ns(), nullptr, nullptr);
  sess_store(E, s);
  eng_unlock(E);
}

// Replay: the whole event loop of a trace on one warp, logical clock.
// Events at equal time: completions, then arrivals, then timeouts, then by
// ticket id (the same total order as the oracle).
__global__ void k_replay(Eng state, const sg_job* __restrict__ jobs, uint32_t n, uint32_t exclusive,
                         uint64_t* dur, uint64_t* tmo, EvHeap H, uint64_t* stats) {
  if (threadIdx.x >= 32) return;
  replay_run(state, jobs, n, exclusive, dur, tmo, H, stats);
}

// ------------------------------------------------------- device layout
struct DevLayout {
  uint64_t hdr, need_g, need_raw, prio, status, blk_done, qa, qt, qpos, ext_off, ext_len, rec, extra, total;
  uint32_t qcap;
  uint64_t qt_len;
};

uint32_t queue_positions(uint32_t n) {
  uint32_t q = 32;
  while (q < n) q <<= 1;
  return q;
}

// entries of the 32-ary min-tree over qcap leaves (levels down to <= 32 nodes)
uint64_t tree_entries(uint32_t qcap) {
  uint64_t total = 0, size = qcap;
  for (;;) {
    total += size;
    if (size <= 32) break;
    size >>= 5;
  }
  return total;
}

// positions: queue positions (a power of two >= positions); a replay queues
// each job at most once (positions = n), a live context recycles tickets
// and compacts its positions (positions = 2 * cap)
DevLayout dev_layout(uint32_t cap, bool with_rec, uint64_t extra_bytes, uint64_t positions) {
  auto a256 = [](uint64_t x) { return (x + 255) / 256 * 256; };
  DevLayout L;
  L.qcap = queue_positions((uint32_t)positions);
  L.qt_len = tree_entries(L.qcap);
  uint64_t o = 0;
  L.hdr = o; o += a256(sizeof(EngHdr));
  L.need_g = o; o += a256(8ull * cap);
  L.need_raw = o; o += a256(8ull * cap);
  L.prio = o; o += a256(4ull * cap);
  L.status = o; o += a256(4ull * cap);
  L.blk_done = o; o += a256(4ull * cap);
  L.qa = o; o += a256(4ull * L.qcap);
  L.qt = o; o += a256(8ull * L.qt_len);
  L.qpos = o; o += a256(4ull * cap);
  L.ext_off = o; o += a256(8ull * (cap + 2));
  L.ext_len = o; o += a256(8ull * (cap + 2));
  L.rec = o; if (with_rec) o += a256(sizeof(sg_record) * (uint64_t)cap);
  L.extra = o; o += a256(extra_bytes);
  L.total = o;
  return L;
}

Eng eng_from(char* base, const DevLayout& L) {
  Eng E;
  memset(&E, 0, sizeof E);
  E.hdr = (EngHdr*)(base + L.hdr);
  E.need_g = (uint64_t*)(base + L.need_g);
  E.need_raw = (uint64_t*)(base + L.need_raw);
  E.prio = (int32_t*)(base + L.prio);
  E.status = (uint32_t*)(base + L.status);
  E.blk_done = (uint32_t*)(base + L.blk_done);
  E.qa = (uint32_t*)(base + L.qa);
  E.qt = (uint64_t*)(base + L.qt);
  E.qpos = (uint32_t*)(base + L.qpos);
  E.qcap = L.qcap;
  E.ext_off = (uint64_t*)(base + L.ext_off);
  E.ext_len = (uint64_t*)(base + L.ext_len);
  E.rec = (sg_record*)(base + L.rec);
  return E;
}

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

inline void cpu_relax() {
#if defined(__x86_64__)
  __builtin_ia32_pause();
#endif
}

uint64_t nearest_rank(std::vector<uint64_t>& v, double p) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  double r = p * (double)v.size();
  uint64_t k = (uint64_t)r;
  if ((double)k < r) k++;
  if (k < 1) k = 1;
  return v[k - 1];
}

}  // namespace

// ================================================================ context
struct sg_ctx {
  int device = 0;
  char* pool = nullptr;
  uint64_t pool_bytes = 0, budget = 0, granule = 256;
  uint32_t policy = 0, flags = 0, cap = 0, n_slots = 0;
  char* dev = nullptr;           // engine state
  DevLayout L{};
  Eng eng{};
  char* mapped = nullptr;        // host-mapped publication block
  volatile sg_record* h_rec = nullptr;
  volatile uint32_t* h_ring = nullptr;
  volatile uint32_t* h_hdr = nullptr;
  sg_job* d_jobs = nullptr;      // [cap] job records for sg_run_trace
  uint64_t* d_keep = nullptr;    // [cap] output digests
  uint32_t* d_err = nullptr;     // generator error flags
  std::mutex mu;
  uint32_t next_ticket = 0;
  std::vector<uint8_t> rel_enq;  // a full release is already enqueued
  std::vector<uint64_t> held_raw;  // declared bytes a ticket holds after the partial releases enqueued
  std::vector<uint32_t> free_tickets;   // finished tickets that sg_declare may reuse
  std::vector<uint8_t> in_free;
  cudaStream_t ctrl = nullptr;
  uint32_t n_hp = 4;             // high-priority slots [n_slots, n_slots + n_hp): GEMM jobs
  uint32_t run_flags = 0;        // SG_RUNF_*
  uint32_t phase_jobs = 64;      // starts of one kind per SpMV / GEMM phase (phases.h)
  std::vector<cudaStream_t> slots;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> slot_ev;
};

#define CK(x)                                 \
  do {                                        \
    if ((x) != cudaSuccess) return SG_ERR_CUDA; \
  } while (0)

static void ctx_free(sg_ctx* c) {
  if (!c) return;
  tex_windows_remove(c);
  for (auto s : c->slots) if (s) cudaStreamDestroy(s);
  for (auto e : c->slot_ev) if (e) cudaEventDestroy(e);
  if (c->ctrl) cudaStreamDestroy(c->ctrl);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->dev) cudaFree(c->dev);
  if (c->mapped) cudaFreeHost(c->mapped);
  delete c;
}

static int ctx_reset_locked(sg_ctx* c) {
  for (auto s : c->slots) CK(cudaStreamSynchronize(s));
  CK(cudaStreamSynchronize(c->ctrl));
  k_eng_reset<<<64, 256, 0, c->ctrl>>>(c->eng, c->budget, c->granule, c->policy, c->flags, c->cap,
                                       c->L.qt_len);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(c->d_err, 0, 4, c->ctrl));
  CK(cudaStreamSynchronize(c->ctrl));
  for (uint32_t i = 0; i < c->cap; i++) {
    c->h_rec[i].status = SG_ST_PENDING;
    c->h_rec[i].grant_seq = -1;
  }
  c->h_hdr[0] = 0;
  c->h_hdr[1] = 0;
  c->h_hdr[2] = 0;
  c->next_ticket = 0;
  std::fill(c->rel_enq.begin(), c->rel_enq.end(), 0);
  c->free_tickets.clear();
  std::fill(c->in_free.begin(), c->in_free.end(), 0);
  return SG_OK;
}

extern "C" int sg_init(sg_ctx** out, void* dev_pool, uint64_t pool_bytes, const sg_config* cfg) {
  if (!out) return SG_ERR_INVALID;
  *out = nullptr;
  sg_config d{};
  if (cfg) d = *cfg;
  if (d.policy > SG_POLICY_PRIO_FIRST_FIT) return SG_ERR_INVALID;
  uint64_t granule = d.granule ? d.granule : 256;
  if (granule < 256 || (granule & (granule - 1))) return SG_ERR_INVALID;
  if (!dev_pool || ((uintptr_t)dev_pool % 256) || pool_bytes < granule) return SG_ERR_INVALID;
  if (pool_bytes / granule > kKeyNeedMask) return SG_ERR_INVALID;   // queue keys hold 47-bit needs
  uint32_t cap = d.max_tickets ? d.max_tickets : (1u << 17);
  if (cap > (1u << 24)) return SG_ERR_INVALID;
  if (d.n_streams > 1024 || d.n_gemm_streams > 1024) return SG_ERR_INVALID;
  if (d.run_flags & ~SG_RUNF_OVERLAP) return SG_ERR_INVALID;
  sg_ctx* c = new sg_ctx();
  c->pool = (char*)dev_pool;
  c->pool_bytes = pool_bytes;
  c->granule = granule;
  c->budget = pool_bytes / granule * granule;
  c->policy = d.policy;
  c->flags = d.flags;
  c->cap = cap;
  // Few slots by default: each job kernel alone fills the GPU, and more
  // concurrent memory-bound jobs only contend for L2 (on the mixed trace,
  // 2-4 slots beat 8 or more by 15%)
  c->n_slots = d.n_streams ? d.n_streams : 4;
  c->n_hp = d.n_gemm_streams ? d.n_gemm_streams : 4;
  c->run_flags = d.run_flags;
  c->phase_jobs = d.phase_jobs ? d.phase_jobs : 64;
  c->rel_enq.assign(cap, 0);
  c->held_raw.assign(cap, 0);
  c->in_free.assign(cap, 0);
  int rc = SG_ERR_CUDA;
  do {
    if (cudaGetDevice(&c->device) != cudaSuccess) break;
    uint64_t extra = 64ull * cap + 8ull * cap + 256;  // jobs, keep, err
    c->L = dev_layout(cap, true, extra, 2ull * cap);
    if (cudaMalloc(&c->dev, c->L.total) != cudaSuccess) break;
    c->eng = eng_from(c->dev, c->L);
    c->d_jobs = (sg_job*)(c->dev + c->L.extra);
    c->d_keep = (uint64_t*)(c->dev + c->L.extra + 64ull * cap);
    c->d_err = (uint32_t*)(c->dev + c->L.extra + 72ull * cap);
    uint64_t mbytes = sizeof(sg_record) * (uint64_t)cap + 4ull * cap + 256;
    if (cudaHostAlloc((void**)&c->mapped, mbytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess)
      break;
    memset(c->mapped, 0, mbytes);
    c->h_rec = (volatile sg_record*)c->mapped;
    c->h_ring = (volatile uint32_t*)(c->mapped + sizeof(sg_record) * (uint64_t)cap);
    c->h_hdr = (volatile uint32_t*)(c->mapped + sizeof(sg_record) * (uint64_t)cap + 4ull * cap);
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, c->mapped, 0) != cudaSuccess) break;
    char* dm = (char*)dp;
    c->eng.pub_rec = (sg_record*)dm;
    c->eng.pub_ring = (uint32_t*)(dm + sizeof(sg_record) * (uint64_t)cap);
    c->eng.pub_hdr = (uint32_t*)(dm + sizeof(sg_record) * (uint64_t)cap + 4ull * cap);
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) break;
    if (cudaStreamCreateWithPriority(&c->ctrl, cudaStreamNonBlocking, hi) != cudaSuccess) break;
    // GEMM jobs get streams one step above the others: their persistent
    // CTAs (one per SM) are then placed ahead of pending memory-bound blocks
    const int gemm_prio = hi < lo ? hi + 1 : hi;
    const uint32_t total = c->n_slots + c->n_hp;
    c->slots.assign(total, nullptr);
    c->slot_ev.assign(total, nullptr);
    bool ok = true;
    for (uint32_t i = 0; i < total && ok; i++) {
      ok = cudaStreamCreateWithPriority(&c->slots[i], cudaStreamNonBlocking, i < c->n_slots ? lo : gemm_prio) ==
               cudaSuccess &&
           cudaEventCreateWithFlags(&c->slot_ev[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) break;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) break;
    rc = ctx_reset_locked(c);
  } while (0);
  if (rc != SG_OK) {
    ctx_free(c);
    return rc;
  }
  tex_windows_add(c, c->pool, c->pool_bytes);
  *out = c;
  return SG_OK;
}

extern "C" int sg_reset(sg_ctx* c) {
  if (!c) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  return ctx_reset_locked(c);
}

extern "C" uint32_t sg_device_error(sg_ctx* c) { return c ? c->h_hdr[1] : 0u; }

extern "C" int sg_state(sg_ctx* c, sg_state_summary* out) {
  if (!c || !out) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  for (auto s : c->slots) CK(cudaStreamSynchronize(s));
  CK(cudaStreamSynchronize(c->ctrl));
  EngHdr h;
  CK(cudaMemcpy(&h, c->eng.hdr, sizeof h, cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof *out);
  out->budget = h.budget;
  out->used = h.used;
  out->peak_used = h.peak_used;
  out->max_free_extent = h.max_ext;
  out->grants = h.seq;
  out->passes = h.passes;
  out->frag_waits = h.frag_waits;
  out->policy = h.policy;
  out->free_extents = h.n_ext;
  out->waiting = h.q_len;
  out->done = h.n_done;
  out->error_flags = h.err;
  return SG_OK;
}

// Tickets whose life is over: the full release has run on the device (it
// was requested by sg_release or is done by the job itself), or the request
// timed out. The device keeps no reference to them; they may be reused.
static void collect_finished(sg_ctx* c) {
  for (uint32_t t = 0; t < c->next_ticket; t++) {
    if (c->in_free[t]) continue;
    const uint32_t st = (uint32_t)c->h_rec[t].status;
    if ((st == SG_ST_DONE && c->rel_enq[t]) || st == SG_ST_TIMEOUT) {
      c->in_free[t] = 1;
      c->free_tickets.push_back(t);
    }
  }
}

extern "C" int sg_declare(sg_ctx* c, uint64_t need, int32_t priority, sg_ticket* out) {
  if (!c || !out) return SG_ERR_INVALID;
  if (priority < -32768 || priority > 32767) return SG_ERR_INVALID;
  uint64_t g = (need + c->granule - 1) / c->granule * c->granule;
  if (g > c->budget) return SG_ERR_TOO_LARGE;
  std::lock_guard<std::mutex> lk(c->mu);
  uint32_t t;
  if (c->next_ticket < c->cap) {
    t = c->next_ticket++;
  } else {
    if (c->free_tickets.empty()) collect_finished(c);
    if (c->free_tickets.empty()) return SG_ERR_CAPACITY;
    t = c->free_tickets.back();
    c->free_tickets.pop_back();
    c->in_free[t] = 0;
    c->rel_enq[t] = 0;
  }
  c->h_rec[t].status = SG_ST_PENDING;
  c->held_raw[t] = need;
  k_declare<<<1, 32, 0, c->ctrl>>>(c->eng, t, 1, nullptr, need, priority, 0);
  if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
  *out = t;
  return SG_OK;
}

static int grant_of(sg_ctx* c, sg_ticket t, sg_grant* out) {
  uint32_t st = (uint32_t)c->h_rec[t].status;
  if (st == SG_ST_RUNNING) {
    if (out) {
      out->offset = c->h_rec[t].offset;
      out->ptr = c->pool + out->offset;
      out->grant_time_ns = c->h_rec[t].grant_t;
    }
    return SG_OK;
  }
  if (st == SG_ST_PENDING || st == SG_ST_QUEUED) return SG_NOT_READY;
  if (st == SG_ST_TIMEOUT) return SG_ERR_TIMEOUT;
  return SG_ERR_INVALID;
}

extern "C" int sg_try(sg_ctx* c, sg_ticket t, sg_grant* out) {
  if (!c || t >= c->cap) return SG_ERR_INVALID;
  if (c->h_hdr[1]) return SG_ERR_DEVICE;
  return grant_of(c, t, out);
}

// Withdraw a waiting request (re-runs the notification pass) and report the
// ticket's state afterwards: SG_ERR_TIMEOUT if it was withdrawn, SG_OK (with
// *out) if it had been granted first.
static int cancel_locked(sg_ctx* c, sg_ticket t, sg_grant* out) {
  k_cancel<<<1, 32, 0, c->ctrl>>>(c->eng, t);
  if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
  if (cudaStreamSynchronize(c->ctrl) != cudaSuccess) return SG_ERR_CUDA;
  int rc = grant_of(c, t, out);
  return rc == SG_NOT_READY ? SG_ERR_DEVICE : rc;
}

extern "C" int sg_wait(sg_ctx* c, sg_ticket t, uint64_t timeout_ns, sg_grant* out) {
  if (!c || t >= c->cap) return SG_ERR_INVALID;
  uint64_t t0 = now_ns();
  for (;;) {
    int rc = grant_of(c, t, out);
    if (rc != SG_NOT_READY) return rc;
    if (c->h_hdr[1]) return SG_ERR_DEVICE;
    if (now_ns() - t0 >= timeout_ns) break;
    for (int i = 0; i < 64; i++) cpu_relax();
  }
  // expired: withdraw the request
  std::lock_guard<std::mutex> lk(c->mu);
  return cancel_locked(c, t, out);
}

extern "C" int sg_cancel(sg_ctx* c, sg_ticket t, sg_grant* out) {
  if (!c || t >= c->cap) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (t >= c->next_ticket) return SG_ERR_INVALID;
  const int rc = grant_of(c, t, out);
  if (rc != SG_NOT_READY) return rc;                  // granted, withdrawn or finished already
  return cancel_locked(c, t, out);
}

namespace {

// Every job of a batch declared at logical time t = 0, in index order: the
// queue holds job j at position j with its key, and one policy pass (the
// batch kernel's first) then grants exactly what per-arrival passes would
// (nothing is released at t = 0, so each arrival's pass grants it iff it
// fits after the earlier grants, and first fit sees the same order).
__global__ void k_declare_all(Eng E, const sg_job* __restrict__ jobs, uint32_t n, uint32_t policy,
                              uint64_t granule) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  Sess ks{};
  ks.policy = policy;
  ks.granule = granule;
  const uint64_t now = globaltimer_ns();
  for (uint64_t j = tid; j < n; j += stride) {
    const sg_job& jb = jobs[j];
    const uint64_t g = round_need(jb.need, granule);
    E.need_g[j] = g;
    E.need_raw[j] = jb.need;
    E.prio[j] = jb.prio;
    E.blk_done[j] = 0;
    E.status[j] = ST_QUEUED;
    sg_record r;
    r.status = ST_QUEUED; r.slot = -1; r.grant_seq = -1; r.grant_t = 0; r.offset = 0; r.done_t = 0;
    r.arrival_t = now;
    E.rec[j] = r;
    E.qa[j] = (uint32_t)j;
    E.qpos[j] = (uint32_t)j;
    E.qt[j] = q_key(ks, g, jb.prio);
  }
  if (tid == 0) {
    E.hdr->q_len = n;
    E.hdr->q_begin = 0;
    E.hdr->q_end = n;
  }
}

// one level of the queue's min-tree from the level below
__global__ void k_tree_level(uint64_t* qt, uint64_t child_off, uint64_t child_size, uint64_t parent_off,
                             uint64_t parent_size) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < parent_size; i += stride) {
    uint64_t m = kInf;
    for (uint64_t c = 32 * i; c < 32 * i + 32 && c < child_size; c++) {
      const uint64_t v = qt[child_off + c];
      m = v < m ? v : m;
    }
    qt[parent_off + i] = m;
  }
}

}  // namespace

namespace sg {
// Engine state of a batch that admits on the device (batch.cu): n tickets,
// n queue positions, the device log and a device grant ring of n entries.
uint64_t batch_engine_bytes(uint32_t n) { return dev_layout(n, true, 4ull * n, n).total; }

Eng batch_engine_at(char* base, uint32_t n) {
  const DevLayout L = dev_layout(n, true, 4ull * n, n);
  Eng E = eng_from(base, L);
  E.dev_ring = (uint32_t*)(base + L.extra);
  return E;
}

// reset to one free extent of `budget` bytes and declare all n jobs at t = 0
int batch_engine_start(const Eng& E, const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
                       uint32_t policy, cudaStream_t st) {
  const DevLayout L = dev_layout(n, true, 4ull * n, n);
  k_eng_reset<<<64, 256, 0, st>>>(E, budget, granule, policy, 0, n, L.qt_len);
  if (n) k_declare_all<<<256, 256, 0, st>>>(E, jobs_dev, n, policy, granule);
  uint64_t off = 0, size = L.qcap;
  while (size > 32) {                    // the tree's levels, leaves first
    const uint64_t parent = size >> 5;
    k_tree_level<<<(unsigned)((parent + 255) / 256), 256, 0, st>>>(E.qt, off, size, off + size, parent);
    off += size;
    size = parent;
  }
  return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

cudaStream_t ctx_control_stream(sg_ctx* c) { return c->ctrl; }
char* ctx_pool_base(sg_ctx* c) { return c->pool; }
uint64_t ctx_pool_bytes(sg_ctx* c) { return c->pool_bytes; }
uint64_t ctx_granule(sg_ctx* c) { return c->granule; }
}  // namespace sg

extern "C" int sg_poll_grants(sg_ctx* c, uint32_t* cursor, sg_ticket* out, uint32_t max, uint32_t* n_out) {
  if (!c || !cursor || (!out && max) || !n_out) return SG_ERR_INVALID;
  const uint32_t tail = c->h_hdr[0];
  if (tail - *cursor > c->cap) return SG_ERR_CAPACITY;   // the ring wrapped over unread grants
  uint32_t n = 0;
  while (*cursor != tail && n < max) out[n++] = (sg_ticket)c->h_ring[(*cursor)++ % c->cap];
  *n_out = n;
  return c->h_hdr[1] ? SG_ERR_DEVICE : SG_OK;
}

extern "C" int sg_release(sg_ctx* c, sg_ticket t, uint64_t bytes, void* stream) {
  if (!c || t >= c->cap) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if ((uint32_t)c->h_rec[t].status != SG_ST_RUNNING || c->rel_enq[t]) return SG_ERR_INVALID;
  // the device frees everything for 0 or for at least what is held; a
  // later release of the same ticket is then refused here, before it could
  // reach the device
  if (bytes == 0 || bytes >= c->held_raw[t]) c->rel_enq[t] = 1;
  else c->held_raw[t] -= bytes;
  k_release<<<1, 32, 0, (cudaStream_t)stream>>>(c->eng, t, bytes);
  return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

extern "C" int sg_launch(sg_ctx* c, sg_ticket t, const sg_job* job, const uint64_t* tables_dev,
                         void* stream) {
  if (!c || !job || t >= c->cap) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if ((uint32_t)c->h_rec[t].status != SG_ST_RUNNING || c->rel_enq[t]) return SG_ERR_INVALID;
  RelHook h;
  h.eng = c->eng;
  h.ticket = t;
  h.active = 1;
  char* base = c->pool + c->h_rec[t].offset;
  int rc = launch_job(*job, base, tables_dev, h, nullptr, c->d_err, (cudaStream_t)stream, nullptr);
  if (rc == SG_OK) c->rel_enq[t] = 1;
  return rc;
}

extern "C" int sg_shutdown(sg_ctx* c) {
  if (!c) return SG_ERR_INVALID;
  int rc = SG_OK;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto s : c->slots) if (cudaStreamSynchronize(s) != cudaSuccess) rc = SG_ERR_CUDA;
    if (cudaStreamSynchronize(c->ctrl) != cudaSuccess) rc = SG_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) rc = SG_ERR_CUDA;
    for (uint32_t t = 0; t < c->next_ticket && rc == SG_OK; t++) {
      uint32_t st = (uint32_t)c->h_rec[t].status;
      if (st == SG_ST_RUNNING && !c->rel_enq[t]) k_release<<<1, 32, 0, c->ctrl>>>(c->eng, t, 0);
      else if (st == SG_ST_QUEUED || st == SG_ST_PENDING) k_cancel<<<1, 32, 0, c->ctrl>>>(c->eng, t);
    }
    if (cudaStreamSynchronize(c->ctrl) != cudaSuccess) rc = SG_ERR_CUDA;
  }
  ctx_free(c);
  return rc;
}

// ================================================================ runner
extern "C" int sg_run_trace(sg_ctx* c, const sg_job* jobs, uint32_t n, const uint64_t* tables_dev,
                            uint32_t mode, sg_record* log, uint64_t* keep, sg_run_stats* stats) {
  if (!c || (!jobs && n)) return SG_ERR_INVALID;
  if (n > c->cap) return SG_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  const bool host_io = mode & SG_RUN_HOST_IO;
  const bool timed = (mode & SG_RUN_TIMED) && !(mode & SG_RUN_SATURATED);
  const bool excl = mode & SG_RUN_EXCLUSIVE;
  const bool want_keep = (mode & SG_RUN_KEEP) && keep;
  int rc = ctx_reset_locked(c);
  if (rc != SG_OK) return rc;
  // profiler range over the whole trace (no cost without a profiler)
  struct Range {
    Range() { nvtxRangePushA("sg_run_trace"); }
    ~Range() { nvtxRangePop(); }
  } range;
  std::vector<sg_job> hj(n);
  if (n) {
    if (host_io) {
      memcpy(hj.data(), jobs, sizeof(sg_job) * n);
      CK(cudaMemcpyAsync(c->d_jobs, jobs, sizeof(sg_job) * n, cudaMemcpyHostToDevice, c->ctrl));
    } else {
      CK(cudaMemcpyAsync(c->d_jobs, jobs, sizeof(sg_job) * n, cudaMemcpyDeviceToDevice, c->ctrl));
      CK(cudaMemcpyAsync(hj.data(), jobs, sizeof(sg_job) * n, cudaMemcpyDeviceToHost, c->ctrl));
    }
    if (want_keep) CK(cudaMemsetAsync(c->d_keep, 0, 8ull * n, c->ctrl));
  }
  CK(cudaStreamSynchronize(c->ctrl));
  uint64_t launches = 0;
  const uint32_t n_all = (uint32_t)c->slots.size();
  std::vector<int32_t> slot_ticket(n_all, -1);
  std::vector<uint8_t> slot_used(n_all, 0);
  // admitted jobs not yet started, per kind, in grant order
  std::vector<uint32_t> pend[3];
  size_t pend_pos[3] = {0, 0, 0};
  for (auto& q : pend) q.reserve(n);
  uint32_t ring_head = 0, failed = 0, bad_grants = 0;
  CK(cudaEventRecord(c->ev0, c->ctrl));
  uint32_t declared = 0;
  const uint64_t t0 = now_ns();
  if (!timed && n) {
    k_declare<<<1, 32, 0, c->ctrl>>>(c->eng, 0, n, c->d_jobs, 0, 0, excl ? 1u : 0u);
    CK(cudaGetLastError());
    launches++;
    declared = n;
  }
  uint64_t last_progress = now_ns();
  uint32_t last_done = 0, started = 0;
  uint32_t rr = 0, rr_hp = 0;
  RunGate gate;
  gate.apart = !(c->run_flags & SG_RUNF_OVERLAP) && !excl;
  gate.one_long = gate.apart;
  gate.quota = c->phase_jobs;
  std::vector<uint8_t> is_long(n, 0);
  for (uint32_t j = 0; j < n; j++) is_long[j] = hj[j].duration_ns >= kLongJobNs;
  while (true) {
    if (timed && declared < n) {
      uint64_t el = now_ns() - t0;
      uint32_t k = declared;
      while (k < n && hj[k].arrival_ns <= el) k++;
      if (k > declared) {
        k_declare<<<1, 32, 0, c->ctrl>>>(c->eng, declared, k - declared, c->d_jobs, 0, 0, excl ? 1u : 0u);
        CK(cudaGetLastError());
        launches++;
        declared = k;
      }
    }
    uint32_t tail = c->h_hdr[0];
    while (ring_head < tail) {
      uint32_t t = (uint32_t)c->h_ring[(ring_head++) % c->cap];
      pend[kind_of(hj[t])].push_back(t);
    }
    // which kinds may start now (SpMV and GEMM apart unless SG_RUNF_OVERLAP)
    bool waiting[kKinds];
    int64_t head_seq[kKinds];
    uint32_t running[kKinds] = {0, 0, 0}, long_running = 0;
    for (int k = 0; k < kKinds; k++) {
      waiting[k] = pend_pos[k] < pend[k].size();
      head_seq[k] = waiting[k] ? c->h_rec[pend[k][pend_pos[k]]].grant_seq : INT64_MAX;
    }
    if (gate.apart) {
      for (uint32_t s = 0; s < n_all; s++) {
        const int32_t tk = slot_ticket[s];
        if (tk >= 0 && (uint32_t)c->h_rec[tk].status < SG_ST_DONE) {
          running[kind_of(hj[tk])]++;
          long_running += is_long[tk];
        }
      }
    }
    bool may[kKinds];
    gate.gate(waiting, head_seq, running, may);
    // launch admitted jobs on slots whose last job has released its memory
    // (or were never used); GEMM jobs take the high-priority slots when
    // there are any. Within a slot pool the earliest grant of the kinds that
    // may start goes first.
    for (int pool = 0; pool < 2; pool++) {
      const uint32_t first = pool ? c->n_slots : 0, cnt = pool ? c->n_hp : c->n_slots;
      if (cnt == 0) continue;
      uint32_t& cursor = pool ? rr_hp : rr;
      const bool serves[kKinds] = {!pool, !pool, pool == 1 || c->n_hp == 0};
      while (true) {
        const int kind = pick_kind(serves, may, waiting, head_seq);
        if (kind < 0) break;
        if (!gate.may_start(is_long[pend[kind][pend_pos[kind]]], long_running)) {
          may[kind] = false;   // this kind's next job waits for the long job running
          continue;
        }
        int slot = -1;
        for (uint32_t k = 0; k < cnt; k++) {
          uint32_t s = first + (cursor + k) % cnt;
          int32_t tk = slot_ticket[s];
          if (tk < 0 || (uint32_t)c->h_rec[tk].status >= SG_ST_DONE) { slot = (int)s; break; }
        }
        if (slot < 0) break;
        cursor = (uint32_t)slot - first + 1;
        const uint32_t t = pend[kind][pend_pos[kind]++];
        started++;
        gate.started(kind, may);
        long_running += is_long[t];
        waiting[kind] = pend_pos[kind] < pend[kind].size();
        head_seq[kind] = waiting[kind] ? c->h_rec[pend[kind][pend_pos[kind]]].grant_seq : INT64_MAX;
        RelHook h;
        h.eng = c->eng;
        h.ticket = t;
        h.active = 1;
        // a grant outside the pool is never run on (the engine flags its own
        // inconsistencies; this keeps a job from writing outside the pool)
        const uint64_t off = c->h_rec[t].offset;
        const uint64_t need_g = (hj[t].need + c->granule - 1) / c->granule * c->granule;
        int lrc = SG_ERR_DEVICE;
        if (off <= c->budget && need_g <= c->budget - off)
          lrc = launch_job(hj[t], c->pool + off, tables_dev, h, want_keep ? c->d_keep + t : nullptr, c->d_err,
                           c->slots[slot], &launches);
        else
          bad_grants++;
        if (lrc != SG_OK) {
          // the job cannot run: give its memory back so no waiter is lost
          cudaGetLastError();
          k_release<<<1, 32, 0, c->slots[slot]>>>(c->eng, t, 0);
          launches++;
          failed++;
        }
        c->rel_enq[t] = 1;
        slot_ticket[slot] = (int32_t)t;
        slot_used[slot] = 1;
      }
    }
    uint32_t done = c->h_hdr[2];
    if (done >= n && declared >= n) break;
    if (c->h_hdr[1]) break;
    uint64_t tn = now_ns();
    if (done != last_done || ring_head != started) {
      last_done = done;
      last_progress = tn;
    } else if (tn - last_progress > 120ull * 1000000000ull) {
      break;  // no progress for two minutes: stop waiting, report below
    }
    for (int i = 0; i < 16; i++) cpu_relax();
  }
  for (uint32_t s = 0; s < n_all; s++) {
    if (!slot_used[s]) continue;
    CK(cudaEventRecord(c->slot_ev[s], c->slots[s]));
    CK(cudaStreamWaitEvent(c->ctrl, c->slot_ev[s], 0));
  }
  CK(cudaEventRecord(c->ev1, c->ctrl));
  CK(cudaStreamSynchronize(c->ctrl));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  uint32_t err = c->h_hdr[1];
  uint32_t derr = 0;
  CK(cudaMemcpy(&derr, c->d_err, 4, cudaMemcpyDeviceToHost));
  if (log && n) {
    CK(cudaMemcpyAsync(log, c->eng.rec, sizeof(sg_record) * n,
                       host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->ctrl));
  }
  if (want_keep && n) {
    CK(cudaMemcpyAsync(keep, c->d_keep, 8ull * n,
                       host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->ctrl));
  }
  CK(cudaStreamSynchronize(c->ctrl));
  uint32_t n_done = 0, n_bad = 0;
  uint64_t first = ~0ull, last = 0;
  std::vector<uint64_t> waits, turns;
  waits.reserve(n);
  turns.reserve(n);
  for (uint32_t j = 0; j < n; j++) {
    uint32_t st = (uint32_t)c->h_rec[j].status;
    if (st != SG_ST_DONE) { n_bad++; continue; }
    n_done++;
    uint64_t a = c->h_rec[j].arrival_t, g = c->h_rec[j].grant_t, d = c->h_rec[j].done_t;
    first = std::min(first, a);
    last = std::max(last, d);
    waits.push_back(g - a);
    turns.push_back(d - a);
  }
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->elapsed_ns = (uint64_t)((double)ms * 1e6);
    stats->makespan_ns = n_done ? last - first : 0;
    stats->wait_p50_ns = nearest_rank(waits, 0.50);
    stats->wait_p99_ns = nearest_rank(waits, 0.99);
    stats->turnaround_p50_ns = nearest_rank(turns, 0.50);
    stats->turnaround_p99_ns = nearest_rank(turns, 0.99);
    EngHdr hh;
    CK(cudaMemcpy(&hh, c->eng.hdr, sizeof hh, cudaMemcpyDeviceToHost));
    stats->peak_used = hh.peak_used;
    stats->frag_waits = hh.frag_waits;
    stats->passes = hh.passes;
    stats->launches = launches;
    stats->jobs_done = n_done;
    stats->jobs_failed = n_bad + failed;
  }
  if (err || derr || bad_grants) return SG_ERR_DEVICE;
  if (n_done + failed < n && n_bad > 0) return failed ? SG_ERR_INVALID : SG_ERR_DEVICE;
  return failed ? SG_ERR_INVALID : SG_OK;
}

// ================================================================ replay
extern "C" uint64_t sg_replay_workspace_bytes(uint32_t n) {
  uint64_t cap = n ? n : 1;
  uint64_t extra = 16ull * cap + 16ull * (2 * cap + 1);   // dur, tmo, heap t/k
  return dev_layout((uint32_t)cap, false, extra, cap).total;
}

extern "C" int sg_replay(const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
                         uint32_t policy, uint32_t flags, uint32_t exclusive, sg_record* log_dev,
                         void* workspace_dev, uint64_t* stats_dev, void* stream) {
  if (n == 0) return SG_OK;
  if (!jobs_dev || !log_dev || !workspace_dev || policy > SG_POLICY_PRIO_FIRST_FIT) return SG_ERR_INVALID;
  if (granule == 0) granule = 256;
  if (granule & (granule - 1)) return SG_ERR_INVALID;
  if (budget / granule > kKeyNeedMask) return SG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t cap = n;
  uint64_t extra = 16ull * cap + 16ull * (2ull * cap + 1);
  DevLayout L = dev_layout(cap, false, extra, cap);
  char* base = (char*)workspace_dev;
  Eng E = eng_from(base, L);
  E.rec = log_dev;
  uint64_t* dur = (uint64_t*)(base + L.extra);
  uint64_t* tmo = dur + cap;
  EvHeap H;
  H.t = tmo + cap;
  H.k = H.t + (2ull * cap + 1);
  H.n = 0;
  H.cap = 2 * cap + 1;
  uint64_t b = budget / granule * granule;
  k_eng_reset<<<8, 256, 0, st>>>(E, b, granule, policy, flags, cap, L.qt_len);
  k_replay<<<1, 32, 0, st>>>(E, jobs_dev, n, exclusive, dur, tmo, H, stats_dev);
  return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

extern "C" const char* sg_strerror(int code) {
  switch (code) {
    case SG_OK: return "ok";
    case SG_NOT_READY: return "not ready: request queued";
    case SG_ERR_TIMEOUT: return "timeout: request withdrawn";
    case SG_ERR_TOO_LARGE: return "need exceeds the pool";
    case SG_ERR_INVALID: return "invalid argument or ticket state";
    case SG_ERR_CUDA: return "CUDA error";
    case SG_ERR_UNKNOWN: return "unknown error";
    case SG_ERR_CAPACITY: return "ticket table full";
    case SG_ERR_DEVICE: return "device engine error";
    default: return "unrecognised code";
  }
}

// ======================================================= replay, no allocation
// The same replay as sg_replay, with its workspace in a fixed array that is
// part of this library's device image instead of caller-provided memory.
namespace {

constexpr uint32_t kNoAllocMaxJobs = 16384;
constexpr uint64_t kNoAllocBytes = 2048ull * 1024;   // >= sg_replay_workspace_bytes(16384)

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) unsigned char g_replay_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 128;
static_assert(kNoAllocMaxJobs == SG_REPLAY_NOALLOC_MAX_JOBS, "the header states the limit");

// The array's device address, looked up once per device and context: a
// context torn down and made again (cudaDeviceReset) loads the module anew,
// and the address is looked up again for the new context.
struct ScratchAddr {
  void* ctx = nullptr;
  void* ptr = nullptr;
};
std::mutex g_scratch_mu;
ScratchAddr g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

// Device address of the array on the current device. In host code the
// array's name is only a stand-in for it. The lookup is a set-up step: it is
// refused (SG_ERR_INVALID) while `stream` is being captured into a graph.
int scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SG_ERR_INVALID;
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (!get || get(&ctx) != CUDA_SUCCESS || !ctx) return SG_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  ScratchAddr& a = g_scratch[dev];
  if (a.ptr && a.ctx == (void*)ctx) {
    *out = a.ptr;
    return SG_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return SG_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return SG_ERR_INVALID;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_replay_scratch) != cudaSuccess || !p) return SG_ERR_CUDA;
  a.ctx = (void*)ctx;
  a.ptr = p;
  *out = p;
  return SG_OK;
}

}  // namespace

extern "C" int sg_replay_noalloc(const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
                                 uint32_t policy, uint32_t flags, uint32_t exclusive, sg_record* log_dev,
                                 uint64_t* stats_dev, void* stream) {
  if (n > kNoAllocMaxJobs || sg_replay_workspace_bytes(n) > kNoAllocBytes) return SG_ERR_TOO_LARGE;
  if (n == 0) return SG_OK;
  if (!jobs_dev || !log_dev) return SG_ERR_INVALID;
  void* ws = nullptr;
  int rc = scratch_address((cudaStream_t)stream, &ws);
  if (rc != SG_OK) return rc;
  // the replay kernels initialise every part of the workspace they read, so
  // the previous call's contents need no clearing
  return sg_replay(jobs_dev, n, budget, granule, policy, flags, exclusive, log_dev, ws, stats_dev, stream);
}
