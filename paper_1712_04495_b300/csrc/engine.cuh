// Device-resident admission and notification engine (arXiv 1712.04495).
//
// The shared state of Sec. III-B -- total memory, total used, per-client
// grants and the queue of waiting clients -- lives in device memory. One
// warp at a time owns it (a device spin lock with a bounded wait) and runs
// the life-cycle operations of Sec. IV on it:
//   declare  = pre-allocation: queue the request, run the admission pass;
//   release  = post-free: free the extent, run the notification pass;
//   cancel   = a blocking pre-allocation whose timeout expired.
// The notification passes are the four policies of Sec. V.
//
// Every operation is executed by all 32 lanes of a warp in lock step: scalar
// state sits in lane-uniform registers, and array scans and shifts are
// spread over the lanes (ballot for "first index that ...", chunked copies
// for shifts). The result equals the sequential definition step for step,
// which is what makes replay logs bit-exact against the CPU oracle.
//
// Placement: the pool is a list of free extents sorted by offset and kept
// coalesced; a request (rounded up to the granule) goes to the lowest
// address extent that holds it. A request is served only if it fits the
// byte count (budget - used) and can be placed.
//
// State accesses: a live engine is shared by kernels on many SMs and every
// access is a strong GPU-scope load or store (ld/st .relaxed.gpu) made under
// the lock's acquire and release fences. A replay owns its state in one warp for
// the whole kernel, so it uses plain (L1-cached) accesses; `Eng::owned` says
// which, and kernels set it in a local copy so the choice is made at compile
// time.
#pragma once
#include "common.cuh"

namespace sg {

enum : uint32_t { ST_PENDING = 0, ST_QUEUED = 1, ST_RUNNING = 2, ST_DONE = 3, ST_TIMEOUT = 4,
                  ST_TOO_LARGE = 5 };
enum : uint32_t { ERR_LOCK = 1u, ERR_STATE = 2u, ERR_ORDER = 4u, ERR_HEAP = 8u, ERR_NNZ = 16u,
                  ERR_CAP = 32u, ERR_ITEM = 64u };
static_assert(ERR_LOCK == SG_DEVERR_WAIT && ERR_STATE == SG_DEVERR_STATE && ERR_ORDER == SG_DEVERR_ORDER &&
                  ERR_HEAP == SG_DEVERR_EVENTS && ERR_NNZ == SG_DEVERR_NNZ && ERR_CAP == SG_DEVERR_CAPACITY &&
                  ERR_ITEM == SG_DEVERR_ITEM,
              "device error bits match the ABI's SG_DEVERR_*");

struct EngHdr {            // scalar state, device memory
  uint64_t budget, granule, used, seq, peak_used, frag_waits, passes;
  uint32_t policy, flags, cap, lock, err, n_ext, q_len, ring_tail, n_done, q_begin, q_end, pad;
  uint64_t max_ext;        // length of the largest free extent
};

struct Eng {               // array pointers (kernel parameter, by value)
  EngHdr* hdr;
  uint64_t* need_g;        // [cap] granule-rounded held / requested bytes
  uint64_t* need_raw;      // [cap] declared bytes
  int32_t* prio;           // [cap]
  uint32_t* status;        // [cap]
  uint32_t* blk_done;      // [cap] finished blocks of a ticket's final kernel
  uint32_t* qa;            // [qcap] FIFO / first fit: ticket at each queue position, or kNone
  uint64_t* qt;            // 32-ary min-tree over the positions' needs (levels stored back to back)
  uint32_t* qpos;          // [cap] queue position of a waiting ticket
  uint32_t qcap;           // positions: a power of two >= max(cap, 32)
  uint64_t* ext_off;       // [cap + 2] free extents, sorted, coalesced
  uint64_t* ext_len;       // [cap + 2]
  sg_record* rec;          // [cap] per-ticket log (device)
  sg_record* pub_rec;      // [cap] host-mapped copy of the log, or null
  uint32_t* pub_ring;      // [cap] host-mapped ring of granted tickets, or null
  uint32_t* pub_hdr;       // host-mapped: [0] ring tail, [1] error flags, [2] done count
  uint32_t* dev_ring;      // [cap] device copy of the grant ring (a batch admitting on the device), or null
  uint32_t owned;          // 1: one warp owns the state for the whole kernel (replay)
};

__device__ __forceinline__ Eng eng_live(Eng E) { E.owned = 0; return E; }
__device__ __forceinline__ Eng eng_owned(Eng E) { E.owned = 1; return E; }

template <typename T>
__device__ __forceinline__ T eld(const Eng& E, const T* p) { return E.owned ? *p : ld_gpu(p); }
template <typename T>
__device__ __forceinline__ void est(const Eng& E, T* p, T v) {
  if (E.owned) *p = v;
  else st_gpu(p, v);
}

// granule-rounded request; a request of 0 bytes still takes a granule
__device__ __forceinline__ uint64_t round_need(uint64_t need, uint64_t granule) {
  uint64_t g = (need + granule - 1) / granule * granule;
  return g == 0 ? granule : g;
}

// Lane-uniform register copy of the scalar state for one locked session.
struct Sess {
  uint64_t budget, granule, used, seq, peak, frag, passes, max_ext;
  uint32_t policy, flags, cap, n_ext, q_len, ring_tail, n_done, err, q_begin, q_end;
};

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint64_t kInf = ~0ull;

// Replay only: min-heap of pending completion / timeout events.
struct EvHeap {
  uint64_t* t;             // [cap] event time
  uint64_t* k;             // [cap] (type << 32) | ticket
  uint32_t n, cap;
};

__device__ __forceinline__ Sess sess_load(const Eng& E) {
  Sess s;
  const EngHdr* h = E.hdr;
  s.budget = eld(E, &h->budget);
  s.granule = eld(E, &h->granule);
  s.used = eld(E, &h->used);
  s.seq = eld(E, &h->seq);
  s.peak = eld(E, &h->peak_used);
  s.frag = eld(E, &h->frag_waits);
  s.passes = eld(E, &h->passes);
  s.policy = eld(E, &h->policy);
  s.flags = eld(E, &h->flags);
  s.cap = eld(E, &h->cap);
  s.n_ext = eld(E, &h->n_ext);
  s.q_len = eld(E, &h->q_len);
  s.ring_tail = eld(E, &h->ring_tail);
  s.n_done = eld(E, &h->n_done);
  s.q_begin = eld(E, &h->q_begin);
  s.q_end = eld(E, &h->q_end);
  s.max_ext = eld(E, &h->max_ext);
  s.err = 0;
  return s;
}

__device__ __forceinline__ void sess_store(const Eng& E, const Sess& s) {
  __syncwarp();
  if (lane_id() == 0) {
    EngHdr* h = E.hdr;
    est(E, &h->used, s.used);
    est(E, &h->seq, s.seq);
    est(E, &h->peak_used, s.peak);
    est(E, &h->frag_waits, s.frag);
    est(E, &h->passes, s.passes);
    est(E, &h->n_ext, s.n_ext);
    est(E, &h->q_len, s.q_len);
    est(E, &h->ring_tail, s.ring_tail);
    est(E, &h->n_done, s.n_done);
    est(E, &h->q_begin, s.q_begin);
    est(E, &h->q_end, s.q_end);
    est(E, &h->max_ext, s.max_ext);
    if (s.err) {
      atomicOr(&h->err, s.err);
      if (E.pub_hdr) atomicOr_system(&E.pub_hdr[1], s.err);
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------------ lock
// Spin on the engine lock with a bounded wait (globaltimer); on expiry the
// caller gets false and the error flag is raised. Warp-uniform result.
//
// Every lane reads and writes the state, not only lane 0 that takes the
// lock, so every lane must be ordered after the acquisition and before the
// release. A shuffle carries a value between lanes but orders no memory, so
// after lane 0's acquiring fence the warp meets at a __syncwarp (a barrier
// that orders memory among its lanes) and each lane then runs its own
// acquire fence before its first load of the state. Unlocking mirrors it:
// each lane fences its own stores, the warp meets, and only then does lane 0
// store the free lock word.
__device__ __forceinline__ bool eng_lock(const Eng& E, uint64_t limit_ns = 2000000000ull) {
  int ok = 0;
  if (lane_id() == 0) {
    uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
      if (atomicCAS(&E.hdr->lock, 0u, 1u) == 0u) { ok = 1; break; }
      if (globaltimer_ns() - t0 > limit_ns) break;
      // short naps: a holder keeps the lock for microseconds, and a waiter
      // that sleeps longer than that lets the declaring kernel, which takes
      // the lock again at once, win it over a job's release again and again
      __nanosleep(ns);
      if (ns < 128) ns <<= 1;
    }
    if (!ok) {
      atomicOr(&E.hdr->err, ERR_LOCK);
      if (E.pub_hdr) atomicOr_system(&E.pub_hdr[1], ERR_LOCK);
    }
    fence_gpu();
  }
  ok = __shfl_sync(SG_FULL, ok, 0);
  __syncwarp();
  fence_gpu();
  return ok != 0;
}

__device__ __forceinline__ void eng_unlock(const Eng& E) {
  fence_gpu();
  __syncwarp();
  if (lane_id() == 0) {
    fence_gpu();
    atomicExch(&E.hdr->lock, 0u);
  }
  __syncwarp();
}

// -------------------------------------------------------- warp primitives
// first index i in [from, len) with pred(i), or -1 (warp-uniform)
template <typename Pred>
__device__ __forceinline__ int64_t warp_find_first(uint32_t from, uint32_t len, Pred pred) {
  for (uint32_t base = from; base < len; base += 32) {
    uint32_t i = base + lane_id();
    bool p = (i < len) && pred(i);
    unsigned m = __ballot_sync(SG_FULL, p);
    if (m) return (int64_t)base + (__ffs(m) - 1);
  }
  return -1;
}

// remove element at index i from an array of length len (shift left)
template <typename T>
__device__ __forceinline__ void warp_remove_at(const Eng& E, T* a, uint32_t i, uint32_t len) {
  for (uint32_t base = i; base + 1 < len; base += 32) {
    uint32_t k = base + lane_id();
    T v{};
    bool act = k + 1 < len;
    if (act) v = eld(E, a + k + 1);
    __syncwarp();
    if (act) est(E, a + k, v);
    __syncwarp();
  }
}

// insert v at index i of an array of length len (shift right)
template <typename T>
__device__ __forceinline__ void warp_insert_at(const Eng& E, T* a, uint32_t i, uint32_t len, T v) {
  // move a[i .. len-1] to a[i+1 .. len], top chunk first
  for (int64_t top = (int64_t)len; top > (int64_t)i; top -= 32) {
    int64_t k = top - (int64_t)lane_id();   // destination index
    bool act = k > (int64_t)i;
    T x{};
    if (act) x = eld(E, a + k - 1);
    __syncwarp();
    if (act) est(E, a + k, x);
    __syncwarp();
  }
  if (lane_id() == 0) est(E, a + i, v);
  __syncwarp();
}

// --------------------------------------------------------------- extents
__device__ __forceinline__ int64_t ext_find(const Eng& E, const Sess& s, uint64_t g) {
  const uint64_t* len = E.ext_len;
  return warp_find_first(0, s.n_ext, [&](uint32_t i) { return eld(E, len + i) >= g; });
}

// largest free extent (warp-wide maximum over the list)
__device__ __forceinline__ uint64_t ext_max(const Eng& E, const Sess& s) {
  uint64_t m = 0;
  for (uint32_t base = 0; base < s.n_ext; base += 32) {
    const uint32_t i = base + lane_id();
    const uint64_t v = i < s.n_ext ? eld(E, E.ext_len + i) : 0;
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(SG_FULL, m, o);
    m = w > m ? w : m;
  }
  return m;
}

// take g bytes from the front of extent e
__device__ __forceinline__ uint64_t ext_take(const Eng& E, Sess& s, uint32_t e, uint64_t g) {
  uint64_t off = eld(E, E.ext_off + e);
  uint64_t len = eld(E, E.ext_len + e);
  __syncwarp();
  if (len == g) {
    warp_remove_at(E, E.ext_off, e, s.n_ext);
    warp_remove_at(E, E.ext_len, e, s.n_ext);
    s.n_ext -= 1;
  } else {
    if (lane_id() == 0) {
      est(E, E.ext_off + e, off + g);
      est(E, E.ext_len + e, len - g);
    }
    __syncwarp();
  }
  if (len == s.max_ext) s.max_ext = ext_max(E, s);   // the largest one shrank
  return off;
}

// return [off, off+g) to the free list, merging with neighbours
__device__ __forceinline__ void ext_give(const Eng& E, Sess& s, uint64_t off, uint64_t g) {
  const uint64_t* eo = E.ext_off;
  int64_t p = warp_find_first(0, s.n_ext, [&](uint32_t i) { return eld(E, eo + i) > off; });
  uint32_t ip = p < 0 ? s.n_ext : (uint32_t)p;
  bool left = false, right = false;
  uint64_t ll = 0, rl = 0;
  if (ip > 0) {
    uint64_t lo = eld(E, E.ext_off + ip - 1);
    ll = eld(E, E.ext_len + ip - 1);
    left = lo + ll == off;
  }
  if (ip < s.n_ext) {
    uint64_t ro = eld(E, E.ext_off + ip);
    rl = eld(E, E.ext_len + ip);
    right = off + g == ro;
  }
  __syncwarp();
  uint64_t merged = g;
  if (left && right) {
    merged = ll + g + rl;
    if (lane_id() == 0) est(E, E.ext_len + ip - 1, merged);
    __syncwarp();
    warp_remove_at(E, E.ext_off, ip, s.n_ext);
    warp_remove_at(E, E.ext_len, ip, s.n_ext);
    s.n_ext -= 1;
  } else if (left) {
    merged = ll + g;
    if (lane_id() == 0) est(E, E.ext_len + ip - 1, merged);
    __syncwarp();
  } else if (right) {
    merged = rl + g;
    if (lane_id() == 0) { est(E, E.ext_off + ip, off); est(E, E.ext_len + ip, merged); }
    __syncwarp();
  } else {
    warp_insert_at(E, E.ext_off, ip, s.n_ext, off);
    warp_insert_at(E, E.ext_len, ip, s.n_ext, g);
    s.n_ext += 1;
  }
  if (merged > s.max_ext) s.max_ext = merged;
}

// ----------------------------------------------------------- publication
static_assert(sizeof(sg_record) == 48, "sg_record is 6 x 8 bytes");

__device__ __forceinline__ sg_record rec_load(const Eng& E, uint32_t j) {
  const uint64_t* p = reinterpret_cast<const uint64_t*>(E.rec + j);
  uint64_t w[6];
#pragma unroll
  for (int i = 0; i < 6; i++) w[i] = eld(E, p + i);
  sg_record r;
  memcpy(&r, w, sizeof r);
  return r;
}

__device__ __forceinline__ void rec_store(const Eng& E, uint32_t j, const sg_record& r) {
  uint64_t w[6];
  memcpy(w, &r, sizeof r);
  uint64_t* p = reinterpret_cast<uint64_t*>(E.rec + j);
#pragma unroll
  for (int i = 0; i < 6; i++) est(E, p + i, w[i]);
}

// Host-mapped publication (real runs). The host reads a record's fields
// once it sees a flag: the record's status, the grant ring's tail or the
// count of finished tickets. So each publication writes the fields first,
// then one system fence, then its flags.

// The host copy of a record's fields other than its status (lane 0, no fence).
__device__ __forceinline__ void publish_fields(const Eng& E, uint32_t j, const sg_record& r) {
  volatile sg_record* pr = E.pub_rec + j;
  pr->slot = r.slot;
  pr->grant_seq = r.grant_seq;
  pr->grant_t = r.grant_t;
  pr->offset = r.offset;
  pr->done_t = r.done_t;
  pr->arrival_t = r.arrival_t;
}

// A ticket's record: the device log and the host copy, status last.
__device__ __forceinline__ void publish_record(const Eng& E, uint32_t j, const sg_record& r) {
  __syncwarp();
  if (lane_id() == 0) {
    rec_store(E, j, r);
    if (E.pub_rec) {
      publish_fields(E, j, r);
      __threadfence_system();
      ((volatile sg_record*)(E.pub_rec + j))->status = r.status;
    }
  }
  __syncwarp();
}

// A grant: the record and the grant-ring entry, then one system fence, then
// the two flags a host reads them by (the record's status, the ring tail).
__device__ __forceinline__ void publish_grant(const Eng& E, Sess& s, uint32_t j, const sg_record& r) {
  __syncwarp();
  if (lane_id() == 0) {
    rec_store(E, j, r);
    if (E.dev_ring) est(E, E.dev_ring + s.ring_tail % s.cap, j);
    if (E.pub_rec || E.pub_ring) {
      if (E.pub_rec) publish_fields(E, j, r);
      if (E.pub_ring) ((volatile uint32_t*)E.pub_ring)[s.ring_tail % s.cap] = j;
      __threadfence_system();
      if (E.pub_rec) ((volatile sg_record*)(E.pub_rec + j))->status = r.status;
      if (E.pub_ring) ((volatile uint32_t*)E.pub_hdr)[0] = s.ring_tail + 1;
    }
  }
  __syncwarp();
  s.ring_tail += 1;
}

// A finished ticket: the record, one system fence, then its status and the
// count of finished tickets.
__device__ __forceinline__ void publish_finished(const Eng& E, const Sess& s, uint32_t j, const sg_record& r) {
  __syncwarp();
  if (lane_id() == 0) {
    rec_store(E, j, r);
    if (E.pub_rec || E.pub_hdr) {
      if (E.pub_rec) publish_fields(E, j, r);
      __threadfence_system();
      if (E.pub_rec) ((volatile sg_record*)(E.pub_rec + j))->status = r.status;
      if (E.pub_hdr) ((volatile uint32_t*)E.pub_hdr)[2] = s.n_done;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------- events
enum : uint32_t { EV_COMPLETE = 0, EV_ARRIVE = 1, EV_TIMEOUT = 2 };

__device__ __forceinline__ bool ev_less(uint64_t ta, uint64_t ka, uint64_t tb, uint64_t kb) {
  return ta < tb || (ta == tb && ka < kb);
}

// A 4-ary min-heap on (time, key), kept by lane 0. Entries move into a hole
// and the moving entry stays in registers, so no step reloads what it has
// just stored (a load right behind a store to the same line waits for it).
// Keys are unique (they carry the ticket), so the pop order is the same for
// any correct heap.
__device__ __forceinline__ void heap_push(EvHeap& H, uint64_t t, uint64_t k, Sess& s) {
  if (lane_id() == 0) {
    if (H.n >= H.cap) {
      s.err |= ERR_HEAP;
    } else {
      uint32_t i = H.n++;
      while (i > 0) {
        const uint32_t p = (i - 1) / 4;
        const uint64_t pt = H.t[p], pk = H.k[p];
        if (!ev_less(t, k, pt, pk)) break;
        H.t[i] = pt;
        H.k[i] = pk;
        i = p;
      }
      H.t[i] = t;
      H.k[i] = k;
    }
  }
  H.n = __shfl_sync(SG_FULL, H.n, 0);
  s.err = __shfl_sync(SG_FULL, s.err, 0);
  __syncwarp();
}

__device__ __forceinline__ void heap_pop(EvHeap& H) {
  __syncwarp();                                   // every lane has read the top before lane 0 moves it
  if (lane_id() == 0) {
    const uint32_t n = --H.n;
    const uint64_t xt = H.t[n], xk = H.k[n];      // the last entry sinks from the root
    uint32_t i = 0;
    for (;;) {
      const uint32_t c0 = 4 * i + 1;
      if (c0 >= n) break;
      uint64_t ct[4], ck[4];
#pragma unroll
      for (uint32_t c = 0; c < 4; c++) {
        ct[c] = c0 + c < n ? H.t[c0 + c] : ~0ull;
        ck[c] = c0 + c < n ? H.k[c0 + c] : ~0ull;
      }
      uint32_t m = 0;
#pragma unroll
      for (uint32_t c = 1; c < 4; c++)
        if (c0 + c < n && ev_less(ct[c], ck[c], ct[m], ck[m])) m = c;
      if (!ev_less(ct[m], ck[m], xt, xk)) break;
      H.t[i] = ct[m];
      H.k[i] = ck[m];
      i = c0 + m;
    }
    H.t[i] = xt;
    H.k[i] = xk;
  }
  H.n = __shfl_sync(SG_FULL, H.n, 0);
  __syncwarp();
}

// ------------------------------------------------------------ admission
// Serve ticket j at time t if it count-fits and can be placed.
// heap != null (replay): push its completion at t + dur[j].
__device__ __forceinline__ bool try_grant(const Eng& E, Sess& s, uint32_t j, uint64_t t,
                                          EvHeap* heap, const uint64_t* dur) {
  uint64_t g = eld(E, E.need_g + j);
  if (g > s.budget - s.used) return false;              // count test (Sec. III-B)
  if (g > s.max_ext) return false;                      // fits the count, no extent holds it
  int64_t e = ext_find(E, s, g);
  if (e < 0) { s.err |= ERR_STATE; return false; }      // the largest extent would hold it
  uint64_t off = ext_take(E, s, (uint32_t)e, g);
  s.used += g;
  if (s.used > s.peak) s.peak = s.used;
  sg_record r = rec_load(E, j);
  r.status = ST_RUNNING;
  r.grant_seq = (int64_t)s.seq;
  r.grant_t = t;
  r.offset = off;
  s.seq += 1;
  if (lane_id() == 0) {
    est(E, E.status + j, (uint32_t)ST_RUNNING);
    est(E, E.blk_done + j, 0u);
  }
  publish_grant(E, s, j, r);
  if (heap) heap_push(*heap, t + dur[j], ((uint64_t)EV_COMPLETE << 32) | j, s);
  return true;
}

__device__ __forceinline__ bool is_prio_policy(const Sess& s) {
  return s.policy == SG_POLICY_PRIO_FIFO || s.policy == SG_POLICY_PRIO_FIRST_FIT;
}

// ---------------------------------------------------------------- queue
// Every queued ticket gets the next queue position once, in arrival order,
// and keeps it; a served or withdrawn ticket leaves a hole. Each position
// holds a key, and a 32-ary tree of minimum keys over the positions answers
// "first waiter at or after position i whose key is at most K" with one
// warp-wide load per level.
//
// FIFO and first fit: the key is the granule-rounded need, so the search is
// exactly the sequential scan of the policy (entries above the free bytes
// fail the count test and are skipped, as in Sec. V).
//
// Priority policies: the key is the priority class above the need in
// granules. Serving order is (priority, arrival), and within one class it is
// arrival order, i.e. position order. The smallest key in the tree gives the
// highest class present, and the bound (class, need <= F) selects the waiters
// of that class that fit F, in their service order.
constexpr uint32_t kKeyShift = 47;                       // need in granules < 2^47
constexpr uint64_t kKeyNeedMask = (1ull << kKeyShift) - 1;

__device__ __forceinline__ uint64_t q_key(const Sess& s, uint64_t g, int32_t prio) {
  if (!is_prio_policy(s)) return g;
  return ((uint64_t)(uint32_t)(prio + 32768) << kKeyShift) | (g / s.granule);
}

// Key bound: waiters of class `cls` (priority policies) whose need is at most
// `bytes`; `bytes` = kInf means any need.
__device__ __forceinline__ uint64_t q_bound(const Sess& s, uint64_t cls, uint64_t bytes) {
  if (!is_prio_policy(s)) return bytes == kInf ? kInf - 1 : bytes;
  uint64_t gr = bytes == kInf ? kKeyNeedMask : bytes / s.granule;
  if (gr > kKeyNeedMask) gr = kKeyNeedMask;
  return (cls << kKeyShift) | gr;
}
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    uint64_t w = __shfl_xor_sync(SG_FULL, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ void qt_set(const Eng& E, uint64_t pos, uint64_t v) {
  uint64_t off = 0, size = E.qcap, idx = pos;
  if (lane_id() == 0) est(E, E.qt + idx, v);
  __syncwarp();
  while (size > 32) {
    const uint64_t block = idx & ~31ull;
    const uint64_t m = warp_min_u64(eld(E, E.qt + off + block + lane_id()));
    const uint64_t parent = idx >> 5;
    off += size;
    size >>= 5;
    if (lane_id() == 0) est(E, E.qt + off + parent, m);
    __syncwarp();
    idx = parent;
  }
}

// first position >= from whose need is <= thr, or -1 (warp-uniform)
__device__ __forceinline__ int64_t qt_find(const Eng& E, uint64_t from, uint64_t thr) {
  uint64_t off = 0, size = E.qcap, pos = from;
  uint32_t level = 0;
  for (;;) {
    if (pos >= size) return -1;
    const uint64_t block = pos & ~31ull, idx = block + lane_id();
    const bool ok = idx >= pos && idx < size && eld(E, E.qt + off + idx) <= thr;
    const unsigned m = __ballot_sync(SG_FULL, ok);
    if (m) { pos = block + (__ffs(m) - 1); break; }
    if (size <= 32) return -1;
    pos = (pos >> 5) + 1;
    off += size;
    size >>= 5;
    level++;
  }
  while (level > 0) {                     // descend to the first qualifying leaf
    size <<= 5;
    off -= size;
    level--;
    const uint64_t block = pos << 5, idx = block + lane_id();
    const bool ok = idx < size && eld(E, E.qt + off + idx) <= thr;
    const unsigned m = __ballot_sync(SG_FULL, ok);
    pos = block + (__ffs(m) - 1);         // the parent's minimum guarantees a child
  }
  return (int64_t)pos;
}

// smallest key in the queue (kInf if empty): the tree's top level
__device__ __forceinline__ uint64_t qt_min(const Eng& E) {
  uint64_t off = 0, size = E.qcap;
  while (size > 32) {
    off += size;
    size >>= 5;
  }
  return warp_min_u64(lane_id() < size ? eld(E, E.qt + off + lane_id()) : kInf);
}

// priority class of the first waiter in service order (queue not empty)
__device__ __forceinline__ uint64_t q_top_class(const Eng& E) { return qt_min(E) >> kKeyShift; }

__device__ __forceinline__ void qt_remove(const Eng& E, Sess& s, uint32_t pos) {
  if (lane_id() == 0) est(E, E.qa + pos, kNone);
  __syncwarp();
  qt_set(E, pos, kInf);
  s.q_len -= 1;
}

// Positions run out when many tickets have come and gone: move the waiting
// tickets, in order, to positions 0, 1, ... Removed positions already hold
// kInf, so only the moved entries touch the tree. A live context has at
// least twice as many positions as tickets, so this leaves at least half
// free and its cost is spread over that many insertions.
__device__ __forceinline__ void q_compact(const Eng& E, Sess& s) {
  const uint32_t lane = lane_id();
  uint32_t k = 0;
  for (uint32_t base = s.q_begin; base < s.q_end; base += 32) {
    const uint32_t p = base + lane;
    const uint32_t t = p < s.q_end ? eld(E, E.qa + p) : kNone;
    const uint64_t key = t != kNone ? eld(E, E.qt + p) : kInf;
    unsigned live = __ballot_sync(SG_FULL, t != kNone);
    __syncwarp();
    while (live) {
      const int src_lane = __ffs(live) - 1;
      live &= live - 1;
      const uint32_t from = __shfl_sync(SG_FULL, p, src_lane);
      const uint32_t tk = __shfl_sync(SG_FULL, t, src_lane);
      const uint64_t ky = __shfl_sync(SG_FULL, key, src_lane);
      const uint32_t to = k++;
      if (to == from) continue;            // already in place (warp-uniform)
      if (lane == 0) {
        est(E, E.qa + from, kNone);
        est(E, E.qa + to, tk);
        est(E, E.qpos + tk, to);
      }
      __syncwarp();
      qt_set(E, from, kInf);
      qt_set(E, to, ky);
    }
  }
  s.q_begin = 0;
  s.q_end = k;
}

__device__ __forceinline__ void q_insert(const Eng& E, Sess& s, uint32_t j) {
  if (s.q_end >= E.qcap) q_compact(E, s);
  if (s.q_end >= E.qcap) {                // every position holds a waiting ticket
    s.err |= ERR_CAP;
    return;
  }
  const uint32_t pos = s.q_end++;
  if (lane_id() == 0) {
    est(E, E.qa + pos, j);
    est(E, E.qpos + j, pos);
  }
  __syncwarp();
  qt_set(E, pos, q_key(s, eld(E, E.need_g + j), eld(E, E.prio + j)));
  s.q_len += 1;
  if (lane_id() == 0) est(E, E.status + j, (uint32_t)ST_QUEUED);
  __syncwarp();
}

// One notification pass (Sec. V) over the waiting queue at time t.
__device__ __forceinline__ void policy_pass(const Eng& E, Sess& s, uint64_t t, EvHeap* heap,
                                            const uint64_t* dur) {
  s.passes += 1;
  if (s.policy == SG_POLICY_FIFO) {
    // Policy 1: serve the head while it fits; stop at the first that does not
    while (s.q_len > 0) {
      const int64_t h = qt_find(E, s.q_begin, kInf - 1);
      if (h < 0) break;
      s.q_begin = (uint32_t)h;
      if (!try_grant(E, s, eld(E, E.qa + h), t, heap, dur)) break;
      qt_remove(E, s, (uint32_t)h);
    }
  } else if (s.policy == SG_POLICY_FIRST_FIT) {
    // Policy 2 (MMU): every waiter that fits, in queue order. Free bytes only
    // shrink within a pass, so waiters above the free count are skipped.
    // Waiters above the largest free extent cannot be placed either, so the
    // search skips them too and every waiter it finds is served.
    uint64_t i = s.q_begin;
    while (s.q_len > 0) {
      const uint64_t freeb = s.budget - s.used;
      const int64_t c = qt_find(E, i, freeb < s.max_ext ? freeb : s.max_ext);
      if (c < 0) break;
      if (try_grant(E, s, eld(E, E.qa + c), t, heap, dur)) qt_remove(E, s, (uint32_t)c);
      i = (uint64_t)c + 1;
    }
  } else if (s.policy == SG_POLICY_PRIO_FIFO) {
    // Policy 3: FIFO over the queue sorted by (priority, arrival): serve the
    // first waiter of the highest class present while it fits
    while (s.q_len > 0) {
      const int64_t h = qt_find(E, s.q_begin, q_bound(s, q_top_class(E), kInf));
      if (h < 0) { s.err |= ERR_STATE; break; }          // the class is present
      if (!try_grant(E, s, eld(E, E.qa + h), t, heap, dur)) break;
      qt_remove(E, s, (uint32_t)h);
    }
  } else {
    // Policy 4: first fit inside the highest-priority class present; the next
    // class is considered only once this one is emptied
    while (s.q_len > 0) {
      const uint64_t cls = q_top_class(E);
      uint64_t i = s.q_begin;
      for (;;) {
        const uint64_t freeb = s.budget - s.used;
        const int64_t c = qt_find(E, i, q_bound(s, cls, freeb < s.max_ext ? freeb : s.max_ext));
        if (c < 0) break;
        if (try_grant(E, s, eld(E, E.qa + c), t, heap, dur)) qt_remove(E, s, (uint32_t)c);
        i = (uint64_t)c + 1;
      }
      if (s.q_len > 0 && q_top_class(E) == cls) break;
    }
  }
  // A pass ends blocked by fragmentation when a waiter the policy would serve
  // next fits the free byte count but no free extent holds it: the head under
  // FIFO and Priority FIFO, any waiter under first fit, any waiter of the top
  // class under Priority MMU.
  if (s.q_len > 0) {
    const uint64_t freeb = s.budget - s.used;
    const uint64_t* ng = E.need_g;
    bool blocked = false;
    if (s.policy == SG_POLICY_FIFO || s.policy == SG_POLICY_PRIO_FIFO) {
      const uint64_t cls = s.policy == SG_POLICY_FIFO ? 0 : q_top_class(E);
      const int64_t h = qt_find(E, s.q_begin, q_bound(s, cls, kInf));
      blocked = h >= 0 && eld(E, ng + eld(E, E.qa + h)) <= freeb;
    } else if (s.max_ext >= freeb) {
      // first fit (within the top class under Priority MMU) has just searched
      // with bound min(freeb, max_ext) = freeb and found nobody: no waiter
      // fits the byte count
      blocked = false;
    } else if (s.policy == SG_POLICY_FIRST_FIT) {
      blocked = qt_find(E, s.q_begin, freeb) >= 0;
    } else {
      blocked = qt_find(E, s.q_begin, q_bound(s, q_top_class(E), freeb)) >= 0;
    }
    if (blocked) s.frag += 1;
  }
}

// ----------------------------------------------------- life-cycle steps
// Pre-allocation request of ticket j at time t (need_g / need_raw / prio
// already stored). Returns the ticket's status after the call.
__device__ __forceinline__ void op_declare(const Eng& E, Sess& s, uint32_t j, uint64_t t,
                                           int32_t slot, EvHeap* heap, const uint64_t* dur,
                                           const uint64_t* timeout) {
  sg_record r;
  r.status = ST_PENDING; r.slot = slot; r.grant_seq = -1; r.grant_t = 0; r.offset = 0;
  r.done_t = 0; r.arrival_t = t;
  uint64_t g = eld(E, E.need_g + j);
  if (g > s.budget) {
    // larger than the whole pool: refused at once, never queued
    r.status = ST_TOO_LARGE;
    if (lane_id() == 0) est(E, E.status + j, (uint32_t)ST_TOO_LARGE);
    s.n_done += 1;
    publish_finished(E, s, j, r);
    return;
  }
  if (lane_id() == 0) rec_store(E, j, r);
  __syncwarp();
  if ((s.flags & SG_FLAG_FIFO_BYPASS) && s.policy == SG_POLICY_FIFO) {
    if (try_grant(E, s, j, t, heap, dur)) return;
  }
  q_insert(E, s, j);
  r.status = ST_QUEUED;
  if (lane_id() == 0) rec_store(E, j, r);
  __syncwarp();
  if (heap && timeout && timeout[j] != ~0ull) {
    uint64_t tt = t + timeout[j];
    if (tt < t) tt = ~0ull;
    heap_push(*heap, tt, ((uint64_t)EV_TIMEOUT << 32) | j, s);
  }
  policy_pass(E, s, t, heap, dur);
  // the host's copy says QUEUED only if the pass left j waiting (a grant in
  // the pass published it as RUNNING)
  if (E.pub_rec && eld(E, E.status + j) == ST_QUEUED) publish_record(E, j, r);
}

// Post-free of `bytes` declared bytes of ticket j (0 or >= held: all).
// Returns false (and flags ERR_STATE) if j holds no memory.
__device__ __forceinline__ bool op_release(const Eng& E, Sess& s, uint32_t j, uint64_t bytes,
                                           uint64_t t, EvHeap* heap, const uint64_t* dur) {
  uint32_t st = eld(E, E.status + j);
  if (st != ST_RUNNING) { s.err |= ERR_STATE; return false; }
  uint64_t g = eld(E, E.need_g + j);
  uint64_t raw = eld(E, E.need_raw + j);
  sg_record r = rec_load(E, j);
  uint64_t freed_off, freed;
  bool all = bytes == 0 || bytes >= raw;
  if (all) {
    freed_off = r.offset;
    freed = g;
    r.status = ST_DONE;
    r.done_t = t;
    if (lane_id() == 0) est(E, E.status + j, (uint32_t)ST_DONE);
    s.n_done += 1;
  } else {
    // shrink: keep the granule-rounded remainder at the front of the extent
    uint64_t keep_raw = raw - bytes;
    uint64_t keep = (keep_raw + s.granule - 1) / s.granule * s.granule;
    freed_off = r.offset + keep;
    freed = g - keep;
    if (lane_id() == 0) { est(E, E.need_g + j, keep); est(E, E.need_raw + j, keep_raw); }
  }
  __syncwarp();
  if (freed > 0) {
    ext_give(E, s, freed_off, freed);
    s.used -= freed;
  }
  if (all) publish_finished(E, s, j, r);
  else publish_record(E, j, r);
  policy_pass(E, s, t, heap, dur);
  return true;
}

// Withdraw a waiting ticket (timeout). Returns its status after the call.
__device__ __forceinline__ uint32_t op_cancel(const Eng& E, Sess& s, uint32_t j, uint64_t t,
                                              EvHeap* heap, const uint64_t* dur) {
  uint32_t st = eld(E, E.status + j);
  if (st != ST_QUEUED) return st;
  const uint32_t pos = eld(E, E.qpos + j);
  if (pos < s.q_end && eld(E, E.qa + pos) == j) qt_remove(E, s, pos);
  sg_record r = rec_load(E, j);
  r.status = ST_TIMEOUT;
  r.done_t = t;
  if (lane_id() == 0) est(E, E.status + j, (uint32_t)ST_TIMEOUT);
  s.n_done += 1;
  publish_finished(E, s, j, r);
  // removing the head can unblock FIFO: notify
  policy_pass(E, s, t, heap, dur);
  return ST_TIMEOUT;
}

// Replay of a trace by one warp on a logical clock: the whole event loop
// (arrivals in index order, completions at grant + declared duration,
// timeouts), one policy pass per event. Events at equal time: completions,
// then arrivals, then timeouts, then by ticket.
__device__ __forceinline__ void replay_run(const Eng& state, const sg_job* __restrict__ jobs, uint32_t n,
                                           uint32_t exclusive, uint64_t* dur, uint64_t* tmo, EvHeap& H,
                                           uint64_t* stats) {
  const Eng E = eng_owned(state);   // this warp is the only user of the state
  const uint32_t lane = lane_id();
  const EngHdr* h0 = E.hdr;
  const uint64_t budget = h0->budget, granule = h0->granule;
  uint32_t bad = 0;
  for (uint32_t j = lane; j < n; j += 32) {
    const sg_job& jb = jobs[j];
    uint64_t g = exclusive ? budget : round_need(jb.need, granule);
    E.need_g[j] = g;
    E.need_raw[j] = exclusive ? budget : jb.need;
    E.prio[j] = jb.prio;
    E.status[j] = ST_PENDING;
    dur[j] = jb.duration_ns;
    tmo[j] = jb.timeout_ns;
    sg_record r;
    r.status = ST_PENDING; r.slot = -1; r.grant_seq = -1; r.grant_t = 0; r.offset = 0;
    r.done_t = 0; r.arrival_t = jb.arrival_ns;
    E.rec[j] = r;
    if (j > 0 && jobs[j - 1].arrival_ns > jb.arrival_ns) bad = 1;
  }
  __syncwarp();
  Sess s = sess_load(E);
  if (__any_sync(SG_FULL, bad)) s.err |= ERR_ORDER;
  uint32_t na = 0;
  while (s.err == 0) {
    bool has_a = na < n;
    bool has_e = H.n > 0;
    if (!has_a && !has_e) break;
    uint64_t et = 0, ek = 0, at = 0, ak = 0;
    if (has_e) { et = H.t[0]; ek = H.k[0]; }
    if (has_a) { at = jobs[na].arrival_ns; ak = ((uint64_t)EV_ARRIVE << 32) | na; }
    bool take_e = has_e && (!has_a || ev_less(et, ek, at, ak));
    if (take_e) {
      heap_pop(H);
      uint32_t type = (uint32_t)(ek >> 32), j = (uint32_t)ek;
      if (type == EV_COMPLETE) op_release(E, s, j, 0, et, &H, dur);
      else op_cancel(E, s, j, et, &H, dur);
    } else {
      op_declare(E, s, na, at, -1, &H, dur, tmo);
      na++;
    }
  }
  sess_store(E, s);
  if (stats && lane == 0) {
    stats[0] = s.peak;
    stats[1] = s.frag;
    stats[2] = s.passes;
    stats[3] = s.err | ld_gpu(&E.hdr->err);
  }
}

// Locked release from a job kernel's last block (warp 0 of it).
__device__ __forceinline__ void eng_release_locked(const Eng& shared, uint32_t j, uint64_t bytes) {
  const Eng E = eng_live(shared);
  if (!eng_lock(E)) return;
  Sess s = sess_load(E);
  op_release(E, s, j, bytes, globaltimer_ns(), nullptr, nullptr);
  sess_store(E, s);
  eng_unlock(E);
}

// Release hook carried by a job's final kernel: the last block to finish
// releases the ticket (post-free on the device, no host round trip).
struct RelHook {
  Eng eng;
  uint32_t ticket;
  uint32_t active;
};

__device__ __forceinline__ void job_epilogue(const RelHook& h) {
  if (!h.active) return;
  __shared__ uint32_t s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    uint32_t nblk = gridDim.x * gridDim.y * gridDim.z;
    uint32_t prev = atomicAdd(h.eng.blk_done + h.ticket, 1u);
    s_last = (prev + 1 == nblk);
  }
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    __threadfence();
    eng_release_locked(h.eng, h.ticket, 0);
  }
}

}  // namespace sg
