// Client processes sharing the scheduler through host shared memory, the
// distributed control of arXiv 1712.04495, Sec. III-A (the state and its
// operations are in shm_core.h). This file holds the handle: the mapping,
// the file lock with the dirty mark, recovery, the backup copy and the
// pool's CUDA IPC mapping.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "shm_core.h"

using namespace sg::shm;

struct sg_shm {
  std::string name, bak;
  int fd = -1;
  void* base = nullptr;
  uint64_t bytes = 0;
  View v;
  // fixed parameters of the segment (its header may be damaged later)
  uint32_t cap = 0, policy = 0, flags = 0;
  uint64_t budget = 0, granule = 0;
  std::mutex mu;              // threads sharing this handle share its lock
  uint64_t id = 0;            // owner tag of this handle's tickets
  int32_t pid = 0;
  uint64_t pid_start = 0;
  std::atomic<uint64_t> last_reap{0};
  char* pool = nullptr;       // this process's address of the pool
  void* ipc_base = nullptr;   // mapping opened through CUDA IPC (closed at the end)
};

namespace {

constexpr uint64_t kLockLimitNs = 10ull * 1000000000ull;   // a lock not had by then: SG_ERR_UNKNOWN
constexpr uint64_t kFirstReapNs = 2ull * 1000000;          // a blocked client checks the holders ...
constexpr uint64_t kReapPeriodNs = 20ull * 1000000;        // ... and then every 20 ms
constexpr uint32_t kDefaultCap = 4096;

uint64_t sat_add(uint64_t a, uint64_t b) { return a + b < a ? ~0ull : a + b; }

bool ofd_lock(int fd, uint64_t deadline) {
  struct flock fl;
  memset(&fl, 0, sizeof fl);
  fl.l_type = F_WRLCK;
  fl.l_whence = SEEK_SET;
  fl.l_start = 0;
  fl.l_len = 1;
  uint64_t pause = 2000;
  for (uint32_t tries = 0;; tries++) {
    if (fcntl(fd, F_OFD_SETLK, &fl) == 0) return true;
    if (errno != EAGAIN && errno != EACCES && errno != EINTR) return false;
    if (now_ns() >= deadline) return false;
    if (tries < 32) {
      sched_yield();
    } else {
      timespec ts{0, (long)pause};
      nanosleep(&ts, nullptr);
      pause = std::min<uint64_t>(pause * 2, 100000);
    }
  }
}

void ofd_unlock(int fd) {
  struct flock fl;
  memset(&fl, 0, sizeof fl);
  fl.l_type = F_UNLCK;
  fl.l_whence = SEEK_SET;
  fl.l_start = 0;
  fl.l_len = 1;
  fcntl(fd, F_OFD_SETLK, &fl);
}

void wake_every_ticket(const View& v, uint32_t cap) {
  for (uint32_t s = 0; s < cap; s++) futex_wake_all(&v.tk[s].status);
}

// Rewrite the fixed header fields from the handle's copy.
void restore_fixed_header(sg_shm* s) {
  Hdr* h = s->v.h;
  h->magic = kMagic;
  h->version = kVersion;
  h->cap = s->cap;
  h->budget = s->budget;
  h->granule = s->granule;
  h->policy = s->policy;
  h->flags = s->flags;
  h->bytes = s->bytes;
}

struct Counters {
  uint64_t reaped, rebuilt, restored, reset, abandoned, timeouts, backups, generation;
};

Counters counters_of(const Hdr* h) {
  return {h->reaped, h->rebuilt, h->restored, h->reset, h->abandoned, h->timeouts, h->backups, h->generation};
}

void put_counters(Hdr* h, const Counters& c) {
  h->reaped = c.reaped;
  h->rebuilt = c.rebuilt;
  h->restored = c.restored;
  h->reset = c.reset;
  h->abandoned = c.abandoned;
  h->timeouts = c.timeouts;
  h->backups = c.backups;
  h->generation = c.generation;
}

// The backup object: the segment image followed by {checksum, generation}.
bool restore_backup(sg_shm* s) {
  const int fd = shm_open(s->bak.c_str(), O_RDONLY, 0);
  if (fd < 0) return false;
  struct stat st;
  bool ok = fstat(fd, &st) == 0 && (uint64_t)st.st_size == s->bytes + 16;
  std::vector<char> img;
  uint64_t trailer[2] = {0, 0};
  if (ok) {
    img.resize(s->bytes);
    ok = pread(fd, img.data(), s->bytes, 0) == (ssize_t)s->bytes &&
         pread(fd, trailer, 16, (off_t)s->bytes) == 16 && checksum(img.data(), s->bytes) == trailer[0];
  }
  close(fd);
  if (!ok) return false;
  const View b = view_of(img.data(), s->cap);
  if (check_state(b, s->bytes) != 0) return false;
  memcpy(s->base, img.data(), s->bytes);
  return true;
}

void write_backup(sg_shm* s) {
  std::vector<char> img((const char*)s->base, (const char*)s->base + s->bytes);
  ((Hdr*)img.data())->dirty = 0;
  const uint64_t trailer[2] = {checksum(img.data(), s->bytes), s->v.h->generation};
  const int fd = shm_open(s->bak.c_str(), O_RDWR | O_CREAT, 0600);
  if (fd < 0) return;
  if (ftruncate(fd, (off_t)(s->bytes + 16)) == 0 && pwrite(fd, img.data(), s->bytes, 0) == (ssize_t)s->bytes &&
      pwrite(fd, trailer, 16, (off_t)s->bytes) == 16)
    s->v.h->backups++;
  close(fd);
}

// Integrity check and recovery (under the lock). Returns the problems found.
uint32_t verify_and_recover(sg_shm* s, uint32_t found) {
  View v = s->v;
  uint32_t bad = check_state(v, s->bytes);
  if (bad == 0) return found;
  found |= bad;
  const Counters c = counters_of(v.h);
  if (bad & BAD_HEADER) {
    restore_fixed_header(s);
    bad = check_state(v, s->bytes);
    if (bad == 0) return found;
  }
  const uint64_t t = now_ns();
  if (!(bad & BAD_HEADER) && rebuild_from_tickets(v) && check_state(v, s->bytes) == 0) {
    v.h->rebuilt++;
    policy_pass(v, t);
  } else if (restore_backup(s)) {
    put_counters(v.h, c);
    v.h->restored++;
    wake_every_ticket(v, s->cap);
    op_reap(v, t);
    policy_pass(v, t);
  } else {
    init_state(v, s->cap, s->budget, s->granule, s->policy, s->flags);
    put_counters(v.h, c);
    v.h->reset++;
    wake_every_ticket(v, s->cap);
  }
  return found;
}

// Holds the handle's mutex and the segment's file lock. On entry, a dirty
// mark left by a holder that died inside an update triggers the integrity
// check; the mark is then set for this update and cleared on exit.
class Locked {
 public:
  Locked(sg_shm* s, uint64_t deadline) : s_(s), lk_(s->mu) {
    if (!ofd_lock(s->fd, deadline)) return;
    held_ = true;
    Hdr* h = s->v.h;
    if (h->dirty) {
      h->abandoned++;
      found_ = verify_and_recover(s, DIRTY);
    }
    h->dirty = 1;
  }
  ~Locked() {
    if (!held_) return;
    Hdr* h = s_->v.h;
    h->generation++;
    std::atomic_thread_fence(std::memory_order_release);
    h->dirty = 0;
    ofd_unlock(s_->fd);
  }
  bool held() const { return held_; }
  uint32_t found() const { return found_; }

 private:
  sg_shm* s_;
  std::unique_lock<std::mutex> lk_;
  bool held_ = false;
  uint32_t found_ = 0;
};

bool valid_name(const char* name) {
  if (!name || name[0] != '/') return false;
  const size_t n = strlen(name);
  return n >= 2 && n < 200 && !strchr(name + 1, '/');
}

// Slot of a ticket whose generation still matches, else -1.
int64_t slot_of(const sg_shm* s, sg_ticket t) {
  const uint32_t slot = t & 0xffffu;
  if (slot >= s->cap) return -1;
  if (s->v.tk[slot].gen.load(std::memory_order_acquire) != (t >> 16)) return -1;
  return slot;
}

// Lock-free read of a ticket's state (the grant fields are written before
// its status turns RUNNING and do not change while it runs).
int read_grant(sg_shm* s, sg_ticket t, sg_grant* out) {
  const uint32_t slot = t & 0xffffu;
  if (slot >= s->cap) return SG_ERR_INVALID;
  Tk& k = s->v.tk[slot];
  for (int tries = 0; tries < 8; tries++) {
    const uint32_t st = k.status.load(std::memory_order_acquire);
    const uint32_t g = k.gen.load(std::memory_order_acquire);
    if (g != (t >> 16)) return SG_ERR_INVALID;            // ended, slot reused
    if (st == SG_ST_QUEUED) return SG_NOT_READY;
    if (st != SG_ST_RUNNING) return SG_ERR_INVALID;       // ended
    const uint64_t off = __atomic_load_n(&k.offset, __ATOMIC_RELAXED);
    const uint64_t gt = __atomic_load_n(&k.grant_ns, __ATOMIC_RELAXED);
    std::atomic_thread_fence(std::memory_order_acquire);
    if (k.status.load(std::memory_order_relaxed) == SG_ST_RUNNING && k.gen.load(std::memory_order_relaxed) == g) {
      if (out) {
        out->offset = off;
        out->ptr = s->pool ? s->pool + off : nullptr;
        out->grant_time_ns = gt;
      }
      return SG_OK;
    }
  }
  return SG_ERR_UNKNOWN;
}

PFN_cuMemGetAddressRange_v3020 g_range = nullptr;
std::once_flag g_range_once;

bool range_fn() {
  std::call_once(g_range_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 3020, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_range = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(fn);
  });
  return g_range != nullptr;
}

void teardown(sg_shm* s) {
  if (s->base) munmap(s->base, s->bytes);
  if (s->fd >= 0) close(s->fd);
  delete s;
}

}  // namespace

extern "C" int sg_shm_open(const char* name, uint64_t budget, uint32_t policy, const sg_config* cfg,
                           sg_shm** out) {
  if (!out) return SG_ERR_INVALID;
  *out = nullptr;
  if (!valid_name(name)) return SG_ERR_INVALID;
  const uint32_t cap = cfg && cfg->max_tickets ? cfg->max_tickets : kDefaultCap;
  const uint64_t granule = cfg && cfg->granule ? cfg->granule : 256;
  const uint32_t flags = cfg ? cfg->flags : 0;
  if (cap > kMaxCap || granule < 256 || (granule & (granule - 1))) return SG_ERR_INVALID;
  if (budget != 0 && (policy > SG_POLICY_PRIO_FIRST_FIT || budget < granule)) return SG_ERR_INVALID;

  sg_shm* s = new sg_shm;
  s->name = name;
  s->bak = std::string(name) + ".bak";
  s->pid = (int32_t)getpid();
  s->pid_start = sg::process_start(s->pid);
  s->id = ((uint64_t)s->pid << 32) ^ now_ns() ^ (uint64_t)(uintptr_t)s;
  bool created = false;
  s->fd = shm_open(name, O_RDWR | O_CREAT | O_EXCL, 0600);
  if (s->fd >= 0) {
    created = true;
  } else if (errno == EEXIST) {
    s->fd = shm_open(name, O_RDWR, 0);
  }
  if (s->fd < 0) {
    teardown(s);
    return SG_ERR_INVALID;
  }
  if (created && budget == 0) {                  // attaching needs an existing segment
    shm_unlink(name);
    teardown(s);
    return SG_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  if (!ofd_lock(s->fd, now_ns() + kLockLimitNs)) {
    lk.unlock();
    teardown(s);
    return SG_ERR_UNKNOWN;
  }
  int rc = SG_OK;
  struct stat st;
  bool fresh = false;
  if (fstat(s->fd, &st) != 0) {
    rc = SG_ERR_UNKNOWN;
  } else if (st.st_size == 0) {
    // new, or its creator ended before sizing it
    if (budget == 0) {
      rc = SG_ERR_INVALID;
    } else {
      s->bytes = layout(cap).bytes;
      if (ftruncate(s->fd, (off_t)s->bytes) != 0) rc = SG_ERR_UNKNOWN;
      fresh = true;
    }
  } else {
    s->bytes = (uint64_t)st.st_size;
  }
  if (rc == SG_OK) {
    s->base = mmap(nullptr, s->bytes, PROT_READ | PROT_WRITE, MAP_SHARED, s->fd, 0);
    if (s->base == MAP_FAILED) {
      s->base = nullptr;
      rc = SG_ERR_UNKNOWN;
    }
  }
  if (rc == SG_OK) {
    const Hdr* h = (const Hdr*)s->base;
    if (fresh) {
      s->cap = cap;
      s->budget = budget / granule * granule;
      s->granule = granule;
      s->policy = policy;
      s->flags = flags;
      s->v = view_of(s->base, cap);
      init_state(s->v, cap, budget, granule, policy, flags);
    } else if (header_ok(h, s->bytes)) {
      s->cap = h->cap;
      s->budget = h->budget;
      s->granule = h->granule;
      s->policy = h->policy;
      s->flags = h->flags;
      if (budget != 0 && (s->budget != budget / granule * granule || s->policy != policy ||
                          s->granule != granule)) {
        rc = SG_ERR_INVALID;                       // a segment of that name with other parameters
      }
      s->v = view_of(s->base, s->cap);
    } else if (budget != 0 && layout(cap).bytes == s->bytes) {
      // damaged header: the caller's parameters describe the segment
      s->cap = cap;
      s->budget = budget / granule * granule;
      s->granule = granule;
      s->policy = policy;
      s->flags = flags;
      s->v = view_of(s->base, cap);
    } else {
      rc = SG_ERR_UNKNOWN;
    }
  }
  if (rc == SG_OK && !fresh) {
    // a client that starts checks the structure (and recovers it) and
    // reclaims what clients that ended still hold
    Hdr* h = s->v.h;
    if (h->dirty) h->abandoned++;
    h->dirty = 1;
    verify_and_recover(s, 0);
    op_reap(s->v, now_ns());
  }
  if (rc == SG_OK) {
    s->v.h->generation++;
    std::atomic_thread_fence(std::memory_order_release);
    s->v.h->dirty = 0;
  }
  ofd_unlock(s->fd);
  lk.unlock();
  if (rc != SG_OK) {
    teardown(s);
    return rc;
  }
  *out = s;
  return SG_OK;
}

extern "C" int sg_shm_declare(sg_shm* s, uint64_t need, int32_t priority, sg_ticket* out) {
  if (!s || !out) return SG_ERR_INVALID;
  if (priority < -32768 || priority > 32767) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  return op_declare(s->v, need, priority, s->pid, s->pid_start, s->id, now_ns(), out);
}

extern "C" int sg_shm_try(sg_shm* s, sg_ticket t, sg_grant* out) {
  if (!s) return SG_ERR_INVALID;
  return read_grant(s, t, out);
}

extern "C" int sg_shm_wait(sg_shm* s, sg_ticket t, uint64_t timeout_ns, sg_grant* out) {
  if (!s) return SG_ERR_INVALID;
  const uint32_t slot = t & 0xffffu;
  if (slot >= s->cap) return SG_ERR_INVALID;
  const uint64_t t0 = now_ns();
  const uint64_t deadline = sat_add(t0, timeout_ns);
  for (;;) {
    const int rc = read_grant(s, t, out);
    if (rc != SG_NOT_READY) return rc;
    const uint64_t now = now_ns();
    if (now >= deadline) {
      // the wait ran out: withdraw the request (unless it was granted meanwhile)
      Locked L(s, now + kLockLimitNs);
      if (!L.held()) return SG_ERR_UNKNOWN;
      const int64_t sl = slot_of(s, t);
      if (sl < 0) return SG_ERR_INVALID;
      Tk& k = s->v.tk[sl];
      if (k.status.load(std::memory_order_relaxed) == SG_ST_QUEUED) {
        if (k.pid != s->pid) return SG_NOT_READY;   // another process's request: leave it
        op_withdraw(s->v, (uint32_t)sl, now_ns());
        return SG_ERR_TIMEOUT;
      }
      continue;
    }
    // a blocked client checks that the holders are still alive
    const uint64_t last = s->last_reap.load(std::memory_order_relaxed);
    if (now - t0 >= kFirstReapNs && now - last >= kReapPeriodNs) {
      s->last_reap.store(now, std::memory_order_relaxed);
      Locked L(s, now + kLockLimitNs);
      if (L.held()) op_reap(s->v, now_ns());
      continue;
    }
    uint64_t nap = deadline - now;
    const uint64_t next_reap = now - t0 < kFirstReapNs ? t0 + kFirstReapNs - now : kReapPeriodNs;
    if (nap > next_reap) nap = next_reap;
    futex_wait_for(&s->v.tk[slot].status, SG_ST_QUEUED, nap);
  }
}

extern "C" int sg_shm_release(sg_shm* s, sg_ticket t, uint64_t bytes) {
  if (!s) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  const int64_t sl = slot_of(s, t);
  if (sl < 0) return SG_ERR_INVALID;
  Tk& k = s->v.tk[sl];
  if (k.status.load(std::memory_order_relaxed) != SG_ST_RUNNING || k.pid != s->pid) return SG_ERR_INVALID;
  op_release(s->v, (uint32_t)sl, bytes, now_ns());
  return SG_OK;
}

extern "C" int sg_shm_record(sg_shm* s, sg_ticket t, sg_record* out) {
  if (!s || !out) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  const int64_t sl = slot_of(s, t);
  if (sl < 0) return SG_ERR_INVALID;
  const Tk& k = s->v.tk[sl];
  const uint32_t st = k.status.load(std::memory_order_relaxed);
  if (st != SG_ST_QUEUED && st != SG_ST_RUNNING) return SG_ERR_INVALID;
  out->status = (int32_t)st;
  out->slot = -1;
  out->grant_seq = st == SG_ST_RUNNING ? (int64_t)k.grant_seq : -1;
  out->grant_t = st == SG_ST_RUNNING ? k.grant_ns : 0;
  out->offset = st == SG_ST_RUNNING ? k.offset : 0;
  out->done_t = 0;
  out->arrival_t = k.arrival_ns;
  return SG_OK;
}

extern "C" int sg_shm_stats(sg_shm* s, sg_shm_counts* out) {
  if (!s || !out) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  const Hdr* h = s->v.h;
  memset(out, 0, sizeof *out);
  out->budget = h->budget;
  out->granule = h->granule;
  out->used = h->used;
  out->peak_used = h->peak_used;
  out->grants = h->grants;
  out->passes = h->passes;
  out->frag_waits = h->frag_waits;
  out->reaped = h->reaped;
  out->rebuilt = h->rebuilt;
  out->restored = h->restored;
  out->reset = h->reset;
  out->abandoned = h->abandoned;
  out->timeouts = h->timeouts;
  out->backups = h->backups;
  out->generation = h->generation;
  out->policy = h->policy;
  out->max_tickets = h->cap;
  out->waiting = h->q_len;
  uint32_t running = 0;
  for (uint32_t i = 0; i < s->cap; i++) running += s->v.tk[i].status.load(std::memory_order_relaxed) == SG_ST_RUNNING;
  out->running = running;
  out->free_extents = h->n_ext;
  return SG_OK;
}

extern "C" int sg_shm_used_by(sg_shm* s, int32_t pid, uint64_t* bytes) {
  if (!s || !bytes) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  uint64_t b = 0;
  for (uint32_t i = 0; i < s->cap; i++) {
    const Tk& k = s->v.tk[i];
    if (k.status.load(std::memory_order_relaxed) == SG_ST_RUNNING && k.pid == pid) b += k.need_g;
  }
  *bytes = b;
  return SG_OK;
}

extern "C" int sg_shm_check(sg_shm* s, uint32_t* problems) {
  if (!s) return SG_ERR_INVALID;
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  const uint32_t found = verify_and_recover(s, L.found());
  if (problems) *problems = found;
  return SG_OK;
}

extern "C" int sg_shm_set_pool(sg_shm* s, void* dev_pool, uint64_t pool_bytes) {
  if (!s || !dev_pool || pool_bytes < s->budget) return SG_ERR_INVALID;
  if (!range_fn()) return SG_ERR_CUDA;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (g_range(&base, &size, (CUdeviceptr)dev_pool) != CUDA_SUCCESS) return SG_ERR_CUDA;
  if ((char*)dev_pool + pool_bytes > (char*)base + size) return SG_ERR_INVALID;
  cudaIpcMemHandle_t ih;
  if (cudaIpcGetMemHandle(&ih, (void*)base) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  static_assert(sizeof(cudaIpcMemHandle_t) == 64, "CUDA IPC handle size");
  Locked L(s, now_ns() + kLockLimitNs);
  if (!L.held()) return SG_ERR_UNKNOWN;
  Hdr* h = s->v.h;
  memcpy(h->pool_handle, &ih, 64);
  h->pool_offset = (uint64_t)((char*)dev_pool - (char*)base);
  h->pool_bytes = pool_bytes;
  h->pool_local = (uint64_t)(uintptr_t)dev_pool;
  h->pool_pid = s->pid;
  h->pool_pid_start = s->pid_start;
  h->pool_owner = s->id;
  h->pool_set = 1;
  s->pool = (char*)dev_pool;
  return SG_OK;
}

extern "C" int sg_shm_pool(sg_shm* s, void** ptr) {
  if (!s || !ptr) return SG_ERR_INVALID;
  *ptr = nullptr;
  if (s->pool) {
    *ptr = s->pool;
    return SG_OK;
  }
  uint8_t handle[64];
  uint64_t offset = 0, local = 0;
  int32_t owner_pid = 0;
  {
    Locked L(s, now_ns() + kLockLimitNs);
    if (!L.held()) return SG_ERR_UNKNOWN;
    const Hdr* h = s->v.h;
    if (!h->pool_set) return SG_NOT_READY;
    memcpy(handle, h->pool_handle, 64);
    offset = h->pool_offset;
    local = h->pool_local;
    owner_pid = h->pool_pid;
  }
  if (owner_pid == s->pid) {                 // published by another handle of this process
    s->pool = (char*)(uintptr_t)local;
  } else {
    cudaIpcMemHandle_t ih;
    memcpy(&ih, handle, 64);
    void* base = nullptr;
    if (cudaIpcOpenMemHandle(&base, ih, cudaIpcMemLazyEnablePeerAccess) != cudaSuccess) {
      cudaGetLastError();
      return SG_ERR_CUDA;
    }
    s->ipc_base = base;
    s->pool = (char*)base + offset;
  }
  *ptr = s->pool;
  return SG_OK;
}

extern "C" int sg_shm_close(sg_shm* s) {
  if (!s) return SG_ERR_INVALID;
  {
    Locked L(s, now_ns() + kLockLimitNs);
    if (L.held()) {
      // the client ends: its requests are withdrawn and its memory freed,
      // then the holders are checked and the state is backed up
      View v = s->v;
      const uint64_t t = now_ns();
      for (uint32_t i = 0; i < s->cap; i++) {
        Tk& k = v.tk[i];
        const uint32_t st = k.status.load(std::memory_order_relaxed);
        if (k.owner != s->id || (st != SG_ST_QUEUED && st != SG_ST_RUNNING)) continue;
        if (st == SG_ST_RUNNING) {
          op_release(v, i, 0, t);
        } else {
          const int64_t p = q_find(v, i);
          if (p >= 0) q_remove_at(v, (uint32_t)p);
          slot_free(v, i);
          policy_pass(v, t);
        }
      }
      if (v.h->pool_set && v.h->pool_owner == s->id) v.h->pool_set = 0;
      op_reap(v, t);
      write_backup(s);
    }
  }
  if (s->ipc_base) cudaIpcCloseMemHandle(s->ipc_base);
  teardown(s);
  return SG_OK;
}

extern "C" int sg_shm_unlink(const char* name) {
  if (!valid_name(name)) return SG_ERR_INVALID;
  const std::string bak = std::string(name) + ".bak";
  const int a = shm_unlink(name);
  shm_unlink(bak.c_str());
  return a == 0 ? SG_OK : SG_ERR_INVALID;
}
