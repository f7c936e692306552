// The device engine's source (engine.cuh) run on the CPU: 32 host threads
// act as the one warp that owns the state (warp_shim.h). Test harness only.
// The build routes every engine state access through the shim's accessors
// (the replay's owned-state path included).
// Exposes the engine's life-cycle steps on host memory, the replay loop, and
// an invariant check of the whole state after any step.
#include <algorithm>
#include <thread>
#include <vector>

#include "engine.cuh"

thread_local ShimDim3 threadIdx;
ShimDim3 gridDim{1, 1, 1};

namespace sg {
WarpSim* g_warp = nullptr;
thread_local uint32_t t_lane = 0;
thread_local std::vector<PendingStore> t_pending;
std::atomic<uint64_t> g_clock{1};
}  // namespace sg

using namespace sg;

namespace {

template <typename F>
void run_warp(F f) {
  static WarpSim w;
  static bool init = false;
  if (!init) {
    pthread_barrier_init(&w.bar, nullptr, 32);
    init = true;
  }
  g_warp = &w;
  std::vector<std::thread> th;
  for (uint32_t l = 0; l < 32; l++)
    th.emplace_back([&, l] {
      t_lane = l;
      threadIdx.x = l;
      f();
      publish_pending();                     // the kernel ends
    });
  for (auto& t : th) t.join();
}

uint32_t positions_for(uint32_t n) {
  uint32_t q = 32;
  while (q < n) q <<= 1;
  return q;
}

uint64_t tree_len(uint32_t qcap) {
  uint64_t total = 0, size = qcap;
  for (;;) {
    total += size;
    if (size <= 32) break;
    size >>= 5;
  }
  return total;
}

struct Host {
  uint32_t cap;
  uint64_t qt_len;
  EngHdr hdr;
  std::vector<uint64_t> need_g, need_raw, qt, ext_off, ext_len;
  std::vector<int32_t> prio;
  std::vector<uint32_t> status, blk_done, qa, qpos;
  std::vector<sg_record> rec;
  Eng E;
};

void reset(Host* h, uint64_t budget, uint64_t granule, uint32_t policy, uint32_t flags) {
  memset(&h->hdr, 0, sizeof h->hdr);
  h->hdr.budget = budget / granule * granule;
  h->hdr.granule = granule;
  h->hdr.policy = policy;
  h->hdr.flags = flags;
  h->hdr.cap = h->cap;
  h->hdr.n_ext = h->hdr.budget > 0 ? 1 : 0;
  h->hdr.max_ext = h->hdr.budget;
  std::fill(h->status.begin(), h->status.end(), (uint32_t)ST_PENDING);
  std::fill(h->qa.begin(), h->qa.end(), kNone);
  std::fill(h->qt.begin(), h->qt.end(), kInf);
  h->ext_off[0] = 0;
  h->ext_len[0] = h->hdr.budget;
}

Host* make_host(uint32_t cap, uint32_t positions) {
  Host* h = new Host;
  h->cap = cap;
  const uint32_t qcap = positions_for(positions);
  h->qt_len = tree_len(qcap);
  h->need_g.assign(cap, 0);
  h->need_raw.assign(cap, 0);
  h->prio.assign(cap, 0);
  h->status.assign(cap, ST_PENDING);
  h->blk_done.assign(cap, 0);
  h->qa.assign(qcap, kNone);
  h->qt.assign(h->qt_len, kInf);
  h->qpos.assign(cap, 0);
  h->ext_off.assign(cap + 2, 0);
  h->ext_len.assign(cap + 2, 0);
  h->rec.assign(cap, sg_record{});
  Eng& E = h->E;
  memset(&E, 0, sizeof E);
  E.hdr = &h->hdr;
  E.need_g = h->need_g.data();
  E.need_raw = h->need_raw.data();
  E.prio = h->prio.data();
  E.status = h->status.data();
  E.blk_done = h->blk_done.data();
  E.qa = h->qa.data();
  E.qt = h->qt.data();
  E.qpos = h->qpos.data();
  E.qcap = qcap;
  E.ext_off = h->ext_off.data();
  E.ext_len = h->ext_len.data();
  E.rec = h->rec.data();
  return h;
}

uint64_t key_of(const Host* h, uint32_t j) {
  const uint32_t pol = h->hdr.policy;
  if (pol != SG_POLICY_PRIO_FIFO && pol != SG_POLICY_PRIO_FIRST_FIT) return h->need_g[j];
  return ((uint64_t)(uint32_t)(h->prio[j] + 32768) << 47) | (h->need_g[j] / h->hdr.granule);
}

}  // namespace

extern "C" {

void* eh_create(uint32_t cap, uint64_t budget, uint64_t granule, uint32_t policy, uint32_t flags) {
  Host* h = make_host(cap, 2 * cap);
  reset(h, budget, granule, policy, flags);
  return h;
}

void eh_destroy(void* p) { delete (Host*)p; }

// Live steps, each one locked session like the library's control kernels.
void eh_declare(void* p, uint32_t t, uint64_t need, int32_t prio) {
  Host* h = (Host*)p;
  const Eng E = eng_live(h->E);
  run_warp([&] {
    if (!eng_lock(E)) return;
    Sess s = sess_load(E);
    if (lane_id() == 0) {
      st_gpu(E.need_g + t, round_need(need, s.granule));
      st_gpu(E.need_raw + t, need);
      st_gpu(E.prio + t, prio);
      st_gpu(E.blk_done + t, 0u);
    }
    __syncwarp();
    op_declare(E, s, t, globaltimer_ns(), -1, nullptr, nullptr, nullptr);
    sess_store(E, s);
    eng_unlock(E);
  });
}

void eh_release(void* p, uint32_t t, uint64_t bytes) {
  Host* h = (Host*)p;
  run_warp([&] { eng_release_locked(h->E, t, bytes); });
}

void eh_cancel(void* p, uint32_t t) {
  Host* h = (Host*)p;
  const Eng E = eng_live(h->E);
  run_warp([&] {
    if (!eng_lock(E)) return;
    Sess s = sess_load(E);
    op_cancel(E, s, t, globaltimer_ns(), nullptr, nullptr);
    sess_store(E, s);
    eng_unlock(E);
  });
}

uint32_t eh_status(void* p, uint32_t t, sg_record* out) {
  Host* h = (Host*)p;
  if (out) *out = h->rec[t];
  return h->status[t];
}

// used, n_ext, q_len, max_ext, err, passes, frag_waits, peak_used, seq
void eh_header(void* p, uint64_t* out) {
  const EngHdr& e = ((Host*)p)->hdr;
  const uint64_t v[9] = {e.used, e.n_ext, e.q_len, e.max_ext, e.err, e.passes, e.frag_waits, e.peak_used, e.seq};
  memcpy(out, v, sizeof v);
}

// Invariants of the whole state; returns the violated ones as bits:
// 1 extents (order, merge, range), 2 extents and grants do not tile the pool,
// 4 used bytes, 8 largest extent, 16 queue membership, 32 queue-tree leaves,
// 64 queue-tree inner nodes, 128 error flag raised.
uint32_t eh_check(void* p) {
  Host* h = (Host*)p;
  const EngHdr& e = h->hdr;
  uint32_t bad = 0;
  std::vector<std::pair<uint64_t, uint64_t>> parts;
  uint64_t mx = 0;
  if (e.n_ext > h->cap + 1) return 1;
  for (uint32_t i = 0; i < e.n_ext; i++) {
    const uint64_t o = h->ext_off[i], l = h->ext_len[i];
    if (l == 0 || o + l > e.budget || (i > 0 && h->ext_off[i - 1] + h->ext_len[i - 1] >= o)) bad |= 1;
    mx = std::max(mx, l);
    parts.push_back({o, l});
  }
  if (mx != e.max_ext) bad |= 8;
  uint64_t used = 0;
  uint32_t queued = 0;
  for (uint32_t j = 0; j < h->cap; j++) {
    if (h->status[j] == ST_RUNNING) {
      used += h->need_g[j];
      parts.push_back({h->rec[j].offset, h->need_g[j]});
    }
    if (h->status[j] == ST_QUEUED) {
      queued++;
      const uint32_t q = h->qpos[j];
      if (q < e.q_begin || q >= e.q_end || q >= h->E.qcap || h->qa[q] != j) bad |= 16;
    }
  }
  if (used != e.used) bad |= 4;
  std::sort(parts.begin(), parts.end());
  uint64_t at = 0;
  for (auto& x : parts) {
    if (x.first != at) bad |= 2;
    at = x.first + x.second;
  }
  if (at != e.budget) bad |= 2;
  if (queued != e.q_len) bad |= 16;
  for (uint32_t q = 0; q < h->E.qcap; q++) {
    const uint32_t j = h->qa[q];
    const bool live = j != kNone && j < h->cap && h->status[j] == ST_QUEUED && h->qpos[j] == q;
    if (h->qt[q] != (live ? key_of(h, j) : kInf)) bad |= 32;
  }
  uint64_t off = 0, size = h->E.qcap;
  while (size > 32) {
    for (uint64_t i = 0; i < size / 32; i++) {
      uint64_t m = kInf;
      for (uint64_t c = 0; c < 32; c++) m = std::min(m, h->qt[off + 32 * i + c]);
      if (h->qt[off + size + i] != m) bad |= 64;
    }
    off += size;
    size >>= 5;
  }
  if (e.err) bad |= 128;
  return bad;
}

// The replay of a trace (the library's replay loop, owned state).
int eh_replay(const sg_job* jobs, uint32_t n, uint64_t budget, uint64_t granule, uint32_t policy, uint32_t flags,
              uint32_t exclusive, sg_record* out, uint64_t* stats) {
  Host* h = make_host(n, n);
  reset(h, budget, granule, policy, flags);
  std::vector<uint64_t> dur(n), tmo(n), ht(2ull * n + 1), hk(2ull * n + 1);
  EvHeap H;
  H.t = ht.data();
  H.k = hk.data();
  H.n = 0;
  H.cap = 2 * n + 1;
  const Eng E = h->E;
  run_warp([&] {
    EvHeap local = H;
    replay_run(E, jobs, n, exclusive, dur.data(), tmo.data(), local, stats);
  });
  memcpy(out, h->rec.data(), sizeof(sg_record) * n);
  const uint32_t bad = h->hdr.err;
  delete h;
  return (int)bad;
}

}  // extern "C"
