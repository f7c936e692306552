// Scheduler state shared by client processes through host shared memory:
// the distributed control of arXiv 1712.04495, Sec. III-A ("Shared
// Memory"), with the shared data of Sec. III-B, the pre-allocation and
// post-free of Sec. IV and the notification policies of Sec. V.
//
// Every client process maps one POSIX shared-memory segment and makes its
// own admission decisions on it; there is no server. The segment holds:
//   - the budget (the GPU memory under the scheduler's control), the bytes
//     in use and, per ticket, the owner process and the bytes it holds (the
//     paper's itemised used memory);
//   - the queue of waiting requests with their priorities;
//   - the free-extent list of the pool (address-ordered first fit with
//     coalescing, granule-rounded requests), so a grant is an offset in one
//     device pool, as in the device engine.
//
// Synchronisation (Sec. III-A): a file lock (an open-file-description
// lock on the segment's first byte) serialises the updates. The kernel
// drops it when its holder dies, so a client that ends inside an update
// does not block the others (abandonment). A waiting client sleeps on a
// futex word in its own ticket and the process that grants the ticket
// wakes exactly that word; the paper sends a user signal instead.
//
// Robustness (Sec. III-A, the four features):
//   - checkpointing: a client that ends (close) writes a backup copy of the
//     segment with a checksum;
//   - integrity check and recovery: a client that starts (open), and any
//     client that takes the lock after a holder died in the middle of an
//     update (the dirty mark is still set), checks the structure. A corrupt
//     state is rebuilt from the ticket table when that table is itself
//     consistent; otherwise the backup is restored; if there is no valid
//     backup, the state is initialised afresh;
//   - sanity check: a client that ends, or that has been blocked waiting,
//     reclaims the memory and withdraws the requests of processes that have
//     exited;
//   - abandonment: the file lock above.
//
// Host code only: the library wraps it with the pool's CUDA IPC mapping.
#pragma once
#include <fcntl.h>
#include <linux/futex.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <sys/syscall.h>
#include <time.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/schedgpu.h"
#include "proc.h"

namespace sg {
namespace shm {

constexpr uint64_t kMagic = 0x5347534d30314131ull;
constexpr uint32_t kVersion = 1;
constexpr uint32_t kMaxCap = 1u << 16;      // slot index: the ticket's low 16 bits
constexpr uint32_t kFree = 0xffffffffu;     // status of an unused ticket slot

// integrity problems (sg_shm_check)
enum : uint32_t {
  BAD_HEADER = SG_SHM_BAD_HEADER, BAD_TICKETS = SG_SHM_BAD_TICKETS, BAD_USED = SG_SHM_BAD_USED,
  BAD_EXTENTS = SG_SHM_BAD_EXTENTS, BAD_QUEUE = SG_SHM_BAD_QUEUE, BAD_SLOTS = SG_SHM_BAD_SLOTS,
  DIRTY = SG_SHM_DIRTY
};

struct Hdr {
  // fixed at creation
  uint64_t magic;
  uint32_t version, cap;
  uint64_t budget, granule;
  uint32_t policy, flags;
  uint64_t bytes;               // size of the whole segment
  // under the lock
  uint32_t dirty;               // set while the lock holder updates the state
  uint32_t n_ext, q_len, n_free;
  uint64_t used, peak_used, grants, passes, frag_waits, arrivals, generation;
  uint64_t reaped, rebuilt, restored, reset, abandoned, timeouts, backups;
  // the device pool, published by one process (CUDA IPC)
  uint32_t pool_set;
  int32_t pool_pid;
  uint64_t pool_pid_start, pool_offset, pool_bytes, pool_local;
  uint8_t pool_handle[64];
  uint64_t pool_owner;          // the handle that published it
  uint64_t reserved[7];
};

struct Tk {
  std::atomic<uint32_t> status;  // SG_ST_QUEUED, SG_ST_RUNNING or kFree; the futex word
  std::atomic<uint32_t> gen;     // bumped when the slot is reused (ticket = gen << 16 | slot)
  int32_t pid, prio;
  uint64_t pid_start, owner;     // owner: the handle that declared it
  uint64_t need_raw, need_g;
  uint64_t offset, grant_seq, grant_ns;   // written before status turns RUNNING
  uint64_t arrival_seq, arrival_ns;
};
static_assert(std::atomic<uint32_t>::is_always_lock_free, "futex word");
// The segment is a wire format between processes (and the host-side tests
// that damage it on purpose): these offsets are fixed.
static_assert(sizeof(Hdr) == 344 && offsetof(Hdr, dirty) == 48 && offsetof(Hdr, used) == 64, "header layout");
static_assert(sizeof(Tk) == 88 && offsetof(Tk, pid) == 8 && offsetof(Tk, need_g) == 40 && offsetof(Tk, offset) == 48,
              "ticket layout");

inline uint64_t align64(uint64_t x) { return (x + 63) & ~63ull; }

struct Layout {
  uint64_t tk, eo, el, q, fs, bytes;
};

inline Layout layout(uint32_t cap) {
  Layout L;
  uint64_t o = align64(sizeof(Hdr));
  L.tk = o; o += align64(sizeof(Tk) * (uint64_t)cap);
  L.eo = o; o += align64(8ull * (cap + 1));
  L.el = o; o += align64(8ull * (cap + 1));
  L.q = o; o += align64(4ull * cap);
  L.fs = o; o += align64(4ull * cap);
  L.bytes = o;
  return L;
}

// Pointers into one mapping of the segment.
struct View {
  Hdr* h = nullptr;
  Tk* tk = nullptr;
  uint64_t* eo = nullptr;      // free extents: offsets (ascending) ...
  uint64_t* el = nullptr;      // ... and lengths
  uint32_t* q = nullptr;       // waiting slots in service order
  uint32_t* fs = nullptr;      // stack of unused slots
};

inline View view_of(void* base, uint32_t cap) {
  const Layout L = layout(cap);
  char* b = (char*)base;
  View v;
  v.h = (Hdr*)b;
  v.tk = (Tk*)(b + L.tk);
  v.eo = (uint64_t*)(b + L.eo);
  v.el = (uint64_t*)(b + L.el);
  v.q = (uint32_t*)(b + L.q);
  v.fs = (uint32_t*)(b + L.fs);
  return v;
}

inline uint64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

inline uint32_t ticket_of(const View& v, uint32_t slot) {
  return (v.tk[slot].gen.load(std::memory_order_relaxed) << 16) | slot;
}

inline void futex_wake_all(std::atomic<uint32_t>* w) {
  syscall(SYS_futex, (uint32_t*)w, FUTEX_WAKE, INT_MAX, nullptr, nullptr, 0);
}

// Sleep while *w == expected, at most ns. Returns on wake-up, change or timeout.
inline void futex_wait_for(std::atomic<uint32_t>* w, uint32_t expected, uint64_t ns) {
  timespec ts;
  ts.tv_sec = (time_t)(ns / 1000000000ull);
  ts.tv_nsec = (long)(ns % 1000000000ull);
  syscall(SYS_futex, (uint32_t*)w, FUTEX_WAIT, expected, &ts, nullptr, 0);
}

// ------------------------------------------------------------ fresh state
inline void init_state(View v, uint32_t cap, uint64_t budget, uint64_t granule, uint32_t policy,
                       uint32_t flags) {
  Hdr* h = v.h;
  const Layout L = layout(cap);
  memset((void*)h, 0, sizeof(Hdr));
  h->version = kVersion;
  h->cap = cap;
  h->granule = granule;
  h->budget = budget / granule * granule;
  h->policy = policy;
  h->flags = flags;
  h->bytes = L.bytes;
  for (uint32_t i = 0; i < cap; i++) {
    v.tk[i].status.store(kFree, std::memory_order_relaxed);
    v.tk[i].gen.store(0, std::memory_order_relaxed);
    v.fs[i] = cap - 1 - i;                 // slot 0 on top
  }
  h->n_free = cap;
  h->n_ext = h->budget > 0 ? 1 : 0;
  v.eo[0] = 0;
  v.el[0] = h->budget;
  h->magic = kMagic;
}

// ------------------------------------------------------- free extents
// Lowest-address free extent that holds g bytes, or -1.
inline int64_t ext_find(const View& v, uint64_t g) {
  for (uint32_t i = 0; i < v.h->n_ext; i++)
    if (v.el[i] >= g) return i;
  return -1;
}

inline uint64_t ext_take(View v, uint32_t i, uint64_t g) {
  const uint64_t off = v.eo[i];
  v.eo[i] += g;
  v.el[i] -= g;
  if (v.el[i] == 0) {
    const uint32_t n = v.h->n_ext;
    memmove(v.eo + i, v.eo + i + 1, 8ull * (n - i - 1));
    memmove(v.el + i, v.el + i + 1, 8ull * (n - i - 1));
    v.h->n_ext = n - 1;
  }
  return off;
}

// Return [off, off + len) to the free list, merging with its neighbours.
inline void ext_give(View v, uint64_t off, uint64_t len) {
  const uint32_t n = v.h->n_ext;
  uint32_t pos = (uint32_t)(std::upper_bound(v.eo, v.eo + n, off) - v.eo);   // first extent after off
  const bool left = pos > 0 && v.eo[pos - 1] + v.el[pos - 1] == off;
  const bool right = pos < n && off + len == v.eo[pos];
  if (left && right) {
    v.el[pos - 1] += len + v.el[pos];
    memmove(v.eo + pos, v.eo + pos + 1, 8ull * (n - pos - 1));
    memmove(v.el + pos, v.el + pos + 1, 8ull * (n - pos - 1));
    v.h->n_ext = n - 1;
  } else if (left) {
    v.el[pos - 1] += len;
  } else if (right) {
    v.eo[pos] = off;
    v.el[pos] += len;
  } else {
    memmove(v.eo + pos + 1, v.eo + pos, 8ull * (n - pos));
    memmove(v.el + pos + 1, v.el + pos, 8ull * (n - pos));
    v.eo[pos] = off;
    v.el[pos] = len;
    v.h->n_ext = n + 1;
  }
}

// ----------------------------------------------------------- tickets
inline void slot_free(View v, uint32_t s) {
  v.tk[s].status.store(kFree, std::memory_order_release);
  futex_wake_all(&v.tk[s].status);          // a waiter on a withdrawn ticket sees it gone
  v.fs[v.h->n_free++] = s;
}

inline void q_remove_at(View v, uint32_t pos) {
  const uint32_t n = v.h->q_len;
  memmove(v.q + pos, v.q + pos + 1, 4ull * (n - pos - 1));
  v.h->q_len = n - 1;
}

inline int64_t q_find(const View& v, uint32_t s) {
  for (uint32_t i = 0; i < v.h->q_len; i++)
    if (v.q[i] == s) return i;
  return -1;
}

// Serve slot s now if its need fits both the free byte count and one free
// extent (Sec. IV pre-allocation: granted when the memory is available).
inline bool try_grant(View v, uint32_t s, uint64_t t) {
  Hdr* h = v.h;
  Tk& k = v.tk[s];
  if (k.need_g > h->budget - h->used) return false;
  const int64_t e = ext_find(v, k.need_g);
  if (e < 0) return false;
  const uint64_t off = ext_take(v, (uint32_t)e, k.need_g);
  h->used += k.need_g;
  if (h->used > h->peak_used) h->peak_used = h->used;
  __atomic_store_n(&k.offset, off, __ATOMIC_RELAXED);
  __atomic_store_n(&k.grant_seq, h->grants++, __ATOMIC_RELAXED);
  __atomic_store_n(&k.grant_ns, t, __ATOMIC_RELAXED);
  k.status.store(SG_ST_RUNNING, std::memory_order_release);
  futex_wake_all(&k.status);
  return true;
}

inline bool count_fits(const View& v, uint32_t s) { return v.tk[s].need_g <= v.h->budget - v.h->used; }

// Queue position of the first waiter of the highest priority class (the
// smallest priority value), earliest arrival first.
inline uint32_t q_top(const View& v) {
  uint32_t best = 0;
  for (uint32_t i = 1; i < v.h->q_len; i++)
    if (v.tk[v.q[i]].prio < v.tk[v.q[best]].prio) best = i;
  return best;
}

// One notification pass (Sec. V) at time t. The queue is kept in arrival
// order; the priority policies select by (priority, arrival) on the fly.
inline void policy_pass(View v, uint64_t t) {
  Hdr* h = v.h;
  h->passes++;
  if (h->policy == SG_POLICY_FIFO) {
    // Policy 1: serve the head while it fits
    while (h->q_len > 0 && try_grant(v, v.q[0], t)) q_remove_at(v, 0);
  } else if (h->policy == SG_POLICY_FIRST_FIT) {
    // Policy 2 (MMU): every waiter that fits, in queue order
    uint32_t i = 0;
    while (i < h->q_len) {
      if (try_grant(v, v.q[i], t)) q_remove_at(v, i);
      else i++;
    }
  } else if (h->policy == SG_POLICY_PRIO_FIFO) {
    // Policy 3: FIFO over (priority, arrival)
    while (h->q_len > 0) {
      const uint32_t p = q_top(v);
      if (!try_grant(v, v.q[p], t)) break;
      q_remove_at(v, p);
    }
  } else {
    // Policy 4: first fit inside the highest class present; the next class
    // only once this one is emptied
    while (h->q_len > 0) {
      const int32_t cls = v.tk[v.q[q_top(v)]].prio;
      uint32_t i = 0;
      bool left = false;
      while (i < h->q_len) {
        const uint32_t s = v.q[i];
        if (v.tk[s].prio == cls && try_grant(v, s, t)) { q_remove_at(v, i); continue; }
        if (v.tk[s].prio == cls) left = true;
        i++;
      }
      if (left) break;
    }
  }
  // ended blocked by fragmentation: a waiter the policy would serve next
  // fits the free byte count but no free extent holds it
  if (h->q_len > 0) {
    bool blocked = false;
    if (h->policy == SG_POLICY_FIFO) {
      blocked = count_fits(v, v.q[0]);
    } else if (h->policy == SG_POLICY_PRIO_FIFO) {
      blocked = count_fits(v, v.q[q_top(v)]);
    } else {
      const int32_t cls = v.tk[v.q[q_top(v)]].prio;
      for (uint32_t i = 0; i < h->q_len && !blocked; i++) {
        const uint32_t s = v.q[i];
        if (h->policy == SG_POLICY_PRIO_FIRST_FIT && v.tk[s].prio != cls) continue;
        blocked = count_fits(v, s);
      }
    }
    if (blocked) h->frag_waits++;
  }
}

// Pre-allocation request (Sec. IV). SG_OK with *ticket (granted or queued),
// SG_ERR_TOO_LARGE, SG_ERR_CAPACITY.
inline int op_declare(View v, uint64_t need, int32_t prio, int32_t pid, uint64_t pid_start, uint64_t owner,
                      uint64_t t, uint32_t* ticket) {
  Hdr* h = v.h;
  uint64_t g = (need + h->granule - 1) / h->granule * h->granule;
  if (g == 0) g = h->granule;                // a request of 0 bytes still takes a granule
  if (g > h->budget) return SG_ERR_TOO_LARGE;
  if (h->n_free == 0) return SG_ERR_CAPACITY;
  const uint32_t s = v.fs[--h->n_free];
  Tk& k = v.tk[s];
  k.gen.store((k.gen.load(std::memory_order_relaxed) + 1) & 0xffffu, std::memory_order_relaxed);
  k.pid = pid;
  k.prio = prio;
  k.pid_start = pid_start;
  k.owner = owner;
  k.need_raw = need;
  k.need_g = g;
  k.offset = 0;
  k.grant_seq = 0;
  k.grant_ns = 0;
  k.arrival_seq = h->arrivals++;
  k.arrival_ns = t;
  k.status.store(SG_ST_QUEUED, std::memory_order_release);
  *ticket = ticket_of(v, s);
  if ((h->flags & SG_FLAG_FIFO_BYPASS) && h->policy == SG_POLICY_FIFO && try_grant(v, s, t)) return SG_OK;
  v.q[h->q_len++] = s;                       // joins the tail
  policy_pass(v, t);
  return SG_OK;
}

// Post-free (Sec. IV) of `bytes` declared bytes of slot s (0 or >= held:
// all, and the ticket ends). A partial release keeps the granule-rounded
// remainder at the front of the grant.
inline void op_release(View v, uint32_t s, uint64_t bytes, uint64_t t) {
  Hdr* h = v.h;
  Tk& k = v.tk[s];
  uint64_t off, len;
  const bool all = bytes == 0 || bytes >= k.need_raw;
  if (all) {
    off = k.offset;
    len = k.need_g;
  } else {
    const uint64_t keep_raw = k.need_raw - bytes;
    const uint64_t keep = (keep_raw + h->granule - 1) / h->granule * h->granule;
    off = k.offset + keep;
    len = k.need_g - keep;
    k.need_raw = keep_raw;
    k.need_g = keep;
  }
  if (len > 0) {
    ext_give(v, off, len);
    h->used -= len;
  }
  if (all) slot_free(v, s);
  policy_pass(v, t);
}

// Withdraw a waiting request (its wait ran out); removing the head can
// unblock FIFO, so the pass runs again.
inline void op_withdraw(View v, uint32_t s, uint64_t t) {
  const int64_t p = q_find(v, s);
  if (p >= 0) q_remove_at(v, (uint32_t)p);
  slot_free(v, s);
  v.h->timeouts++;
  policy_pass(v, t);
}

// Sanity check: reclaim the memory and withdraw the requests of processes
// that have ended. Returns the tickets reclaimed.
inline uint32_t op_reap(View v, uint64_t t) {
  Hdr* h = v.h;
  std::vector<std::pair<int32_t, bool>> seen;   // pid -> ended
  uint32_t n = 0;
  for (uint32_t s = 0; s < h->cap; s++) {
    const uint32_t st = v.tk[s].status.load(std::memory_order_relaxed);
    if (st != SG_ST_QUEUED && st != SG_ST_RUNNING) continue;
    const int32_t pid = v.tk[s].pid;
    bool ended = false, known = false;
    for (auto& p : seen)
      if (p.first == pid) { ended = p.second; known = true; break; }
    if (!known) {
      ended = process_ended(pid, v.tk[s].pid_start);
      seen.push_back({pid, ended});
    }
    if (!ended) continue;
    if (st == SG_ST_RUNNING) {
      op_release(v, s, 0, t);
    } else {
      const int64_t p = q_find(v, s);
      if (p >= 0) q_remove_at(v, (uint32_t)p);
      slot_free(v, s);
      policy_pass(v, t);
    }
    n++;
  }
  h->reaped += n;
  return n;
}

// ------------------------------------------------- integrity check
// Checks the header against the segment size. Everything else depends on it.
inline bool header_ok(const Hdr* h, uint64_t seg_bytes) {
  if (h->magic != kMagic || h->version != kVersion) return false;
  if (h->cap == 0 || h->cap > kMaxCap || layout(h->cap).bytes != h->bytes || h->bytes != seg_bytes) return false;
  if (h->granule < 256 || (h->granule & (h->granule - 1)) || h->budget % h->granule) return false;
  if (h->policy > SG_POLICY_PRIO_FIRST_FIT) return false;
  return true;
}

// The ticket table on its own: statuses, and the grants lie inside the pool,
// aligned and pairwise disjoint. Fills the held grants sorted by offset.
inline bool tickets_ok(const View& v, std::vector<std::pair<uint64_t, uint64_t>>* held) {
  const Hdr* h = v.h;
  held->clear();
  for (uint32_t s = 0; s < h->cap; s++) {
    const Tk& k = v.tk[s];
    const uint32_t st = k.status.load(std::memory_order_relaxed);
    if (st == kFree) continue;
    if (st != SG_ST_QUEUED && st != SG_ST_RUNNING) return false;
    if (k.gen.load(std::memory_order_relaxed) > 0xffffu) return false;
    if (k.need_g == 0 || k.need_g % h->granule || k.need_g > h->budget) return false;
    if (k.need_raw > k.need_g) return false;
    if (st == SG_ST_RUNNING) {
      if (k.offset % h->granule || k.offset > h->budget - k.need_g) return false;
      held->push_back({k.offset, k.need_g});
    }
  }
  std::sort(held->begin(), held->end());
  for (size_t i = 1; i < held->size(); i++)
    if ((*held)[i - 1].first + (*held)[i - 1].second > (*held)[i].first) return false;
  return true;
}

// Full check; returns BAD_* bits (0 = consistent).
inline uint32_t check_state(const View& v, uint64_t seg_bytes) {
  const Hdr* h = v.h;
  if (!header_ok(h, seg_bytes)) return BAD_HEADER;
  uint32_t bad = 0;
  std::vector<std::pair<uint64_t, uint64_t>> held;
  if (!tickets_ok(v, &held)) return BAD_TICKETS;
  uint64_t used = 0;
  for (auto& p : held) used += p.second;
  if (used != h->used || h->peak_used < h->used) bad |= BAD_USED;
  // free extents: aligned, ascending, coalesced; with the grants they tile the pool
  if (h->n_ext > h->cap + 1) {
    bad |= BAD_EXTENTS;
  } else {
    uint64_t pos = 0;
    size_t gi = 0;
    for (uint32_t e = 0; e < h->n_ext && !(bad & BAD_EXTENTS); e++) {
      if (v.el[e] == 0 || v.eo[e] % h->granule || v.el[e] % h->granule || v.eo[e] > h->budget ||
          v.el[e] > h->budget - v.eo[e]) { bad |= BAD_EXTENTS; break; }
      if (e > 0 && v.eo[e - 1] + v.el[e - 1] >= v.eo[e]) { bad |= BAD_EXTENTS; break; }   // order, merge
      while (gi < held.size() && held[gi].first < v.eo[e]) {
        if (held[gi].first != pos) { bad |= BAD_EXTENTS; break; }
        pos += held[gi].second;
        gi++;
      }
      if (pos != v.eo[e]) { bad |= BAD_EXTENTS; break; }
      pos += v.el[e];
    }
    while (!(bad & BAD_EXTENTS) && gi < held.size()) {
      if (held[gi].first != pos) { bad |= BAD_EXTENTS; break; }
      pos += held[gi].second;
      gi++;
    }
    if (!(bad & BAD_EXTENTS) && pos != h->budget) bad |= BAD_EXTENTS;
  }
  // queue: distinct waiting slots in arrival order, and every waiting slot in it
  uint32_t n_wait = 0, n_free = 0;
  for (uint32_t s = 0; s < h->cap; s++) {
    const uint32_t st = v.tk[s].status.load(std::memory_order_relaxed);
    n_wait += st == SG_ST_QUEUED;
    n_free += st == kFree;
  }
  if (h->q_len != n_wait) {
    bad |= BAD_QUEUE;
  } else {
    for (uint32_t i = 0; i < h->q_len; i++) {
      const uint32_t s = v.q[i];
      if (s >= h->cap || v.tk[s].status.load(std::memory_order_relaxed) != SG_ST_QUEUED ||
          (i > 0 && v.tk[v.q[i - 1]].arrival_seq >= v.tk[s].arrival_seq)) { bad |= BAD_QUEUE; break; }
    }
  }
  // unused-slot stack: exactly the free slots (distinct, since the count matches)
  if (h->n_free != n_free) {
    bad |= BAD_SLOTS;
  } else {
    for (uint32_t i = 0; i < h->n_free; i++) {
      const uint32_t s = v.fs[i];
      if (s >= h->cap || v.tk[s].status.load(std::memory_order_relaxed) != kFree) { bad |= BAD_SLOTS; break; }
    }
  }
  return bad;
}

// Recompute everything derived from the ticket table (used bytes, free
// extents, queue, unused slots). False if the table itself is inconsistent.
inline bool rebuild_from_tickets(View v) {
  Hdr* h = v.h;
  std::vector<std::pair<uint64_t, uint64_t>> held;
  if (!tickets_ok(v, &held)) return false;
  uint64_t used = 0, pos = 0;
  uint32_t n = 0;
  for (auto& p : held) {
    if (p.first > pos) { v.eo[n] = pos; v.el[n] = p.first - pos; n++; }
    pos = p.first + p.second;
    used += p.second;
  }
  if (pos < h->budget) { v.eo[n] = pos; v.el[n] = h->budget - pos; n++; }
  h->n_ext = n;
  h->used = used;
  if (h->peak_used < used) h->peak_used = used;
  std::vector<std::pair<uint64_t, uint32_t>> wait;
  uint32_t nf = 0;
  for (uint32_t s = h->cap; s-- > 0;) {
    const uint32_t st = v.tk[s].status.load(std::memory_order_relaxed);
    if (st == SG_ST_QUEUED) wait.push_back({v.tk[s].arrival_seq, s});
    else if (st == kFree) v.fs[nf++] = s;
  }
  h->n_free = nf;
  std::sort(wait.begin(), wait.end());
  for (size_t i = 1; i < wait.size(); i++)
    if (wait[i].first == wait[i - 1].first) return false;   // arrival order lost
  h->q_len = (uint32_t)wait.size();
  for (size_t i = 0; i < wait.size(); i++) v.q[i] = wait[i].second;
  uint64_t next = 0;
  for (auto& w : wait) next = std::max(next, w.first + 1);
  for (uint32_t s = 0; s < h->cap; s++)
    if (v.tk[s].status.load(std::memory_order_relaxed) == SG_ST_RUNNING) next = std::max(next, v.tk[s].arrival_seq + 1);
  if (h->arrivals < next) h->arrivals = next;
  return true;
}

// 64-bit FNV-1a of the backup image (checkpoint integrity).
inline uint64_t checksum(const void* p, uint64_t n) {
  const unsigned char* b = (const unsigned char*)p;
  uint64_t x = 0xcbf29ce484222325ull;
  for (uint64_t i = 0; i < n; i++) {
    x ^= b[i];
    x *= 0x100000001b3ull;
  }
  return x;
}

}  // namespace shm
}  // namespace sg
