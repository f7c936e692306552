// Client side of the scheduler server (arXiv 1712.04495, Sec. IV life cycle
// for a separate process): declare a need, wait for the grant (pushed by the
// server), run work on the grant through this process's mapping of the
// pool, release. The wire protocol is in server_core.h.
#include <poll.h>
#include <sys/socket.h>
#include <sys/un.h>
#include <time.h>
#include <unistd.h>

#include <chrono>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "server_core.h"

namespace {

struct TicketState {
  int rc;              // SG_NOT_READY (waiting), SG_OK (granted), SG_ERR_TIMEOUT
  uint64_t offset, grant_ns;
};

constexpr uint64_t kReplyWaitNs = 30ull * 1000000000ull;   // a server that does not answer

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sg_client {
  int fd = -1;
  std::mutex mu;
  uint64_t pool_bytes = 0, granule = 0, pool_off = 0;
  int handle_rc = SG_ERR_UNKNOWN;
  uint8_t handle[64] = {};
  char* mapped = nullptr;           // this process's mapping of the pool's allocation
  std::unordered_map<uint32_t, TicketState> st;

  // one message within timeout_ns: 1, 0 on timeout, -1 if the server is gone
  int recv_one(uint64_t timeout_ns, sg::WireMsg* m) {
    pollfd p{fd, POLLIN, 0};
    timespec ts{(time_t)(timeout_ns / 1000000000ull), (long)(timeout_ns % 1000000000ull)};
    for (;;) {
      const int r = ppoll(&p, 1, &ts, nullptr);
      if (r < 0 && errno == EINTR) continue;
      if (r == 0) return 0;
      if (r < 0) return -1;
      const ssize_t n = recv(fd, m, sizeof *m, 0);
      if (n == (ssize_t)sizeof *m) return 1;
      if (n < 0 && errno == EINTR) continue;
      return -1;
    }
  }

  // GRANT / TIMEOUT arrive at any time; returns true if `m` was one of them
  bool absorb(const sg::WireMsg& m) {
    if (m.op == sg::MSG_GRANT) {
      st[m.ticket] = TicketState{SG_OK, m.a, m.b};
      return true;
    }
    if (m.op == sg::MSG_TIMEOUT) {
      st[m.ticket] = TicketState{SG_ERR_TIMEOUT, 0, 0};
      return true;
    }
    return false;
  }

  // send a request and wait for its reply (absorbing notifications meanwhile)
  int request(const sg::WireMsg& q, uint32_t reply_op, sg::WireMsg* r) {
    if (send(fd, &q, sizeof q, MSG_NOSIGNAL) != (ssize_t)sizeof q) return SG_ERR_UNKNOWN;
    const uint64_t t0 = now_ns();
    for (;;) {
      const uint64_t el = now_ns() - t0;
      if (el >= kReplyWaitNs) return SG_ERR_UNKNOWN;
      const int got = recv_one(kReplyWaitNs - el, r);
      if (got <= 0) return SG_ERR_UNKNOWN;
      if (absorb(*r)) continue;
      if (r->op == reply_op) return SG_OK;
      if (r->op == sg::MSG_ERROR) return r->rc ? r->rc : SG_ERR_INVALID;
    }
  }

  void drain() {
    sg::WireMsg m;
    while (recv_one(0, &m) == 1) absorb(m);
  }

  int fill(uint32_t t, sg_grant* g) {
    auto it = st.find(t);
    if (it == st.end()) return SG_ERR_INVALID;
    if (it->second.rc == SG_OK && g) {
      g->offset = it->second.offset;
      g->ptr = mapped ? mapped + pool_off + it->second.offset : nullptr;
      g->grant_time_ns = it->second.grant_ns;
    }
    return it->second.rc;
  }
};

extern "C" int sg_client_connect(const char* socket_path, sg_client** out) {
  if (!socket_path || !out) return SG_ERR_INVALID;
  *out = nullptr;
  sockaddr_un addr{};
  if (strlen(socket_path) >= sizeof addr.sun_path) return SG_ERR_INVALID;
  const int fd = socket(AF_UNIX, SOCK_SEQPACKET | SOCK_CLOEXEC, 0);
  if (fd < 0) return SG_ERR_UNKNOWN;
  addr.sun_family = AF_UNIX;
  strcpy(addr.sun_path, socket_path);
  if (connect(fd, (sockaddr*)&addr, sizeof addr) != 0) {
    close(fd);
    return SG_ERR_UNKNOWN;
  }
  sg_client* c = new sg_client();
  c->fd = fd;
  sg::WireMsg q{}, r{};
  q.op = sg::MSG_HELLO;
  q.prio = (int32_t)sg::kWireVersion;
  q.a = (uint64_t)getpid();
  const int rc = c->request(q, sg::MSG_HELLO_OK, &r);
  if (rc != SG_OK || r.prio != (int32_t)sg::kWireVersion) {
    close(fd);
    delete c;
    return rc != SG_OK ? rc : SG_ERR_INVALID;
  }
  c->pool_bytes = r.a;
  c->granule = r.b;
  c->pool_off = r.c;
  c->handle_rc = r.rc;
  memcpy(c->handle, r.payload, 64);
  *out = c;
  return SG_OK;
}

extern "C" int sg_client_info(sg_client* c, uint64_t* pool_bytes, uint64_t* granule) {
  if (!c) return SG_ERR_INVALID;
  if (pool_bytes) *pool_bytes = c->pool_bytes;
  if (granule) *granule = c->granule;
  return SG_OK;
}

extern "C" int sg_client_pool(sg_client* c, void** dev_ptr) {
  if (!c || !dev_ptr) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  if (!c->mapped) {
    if (c->handle_rc != SG_OK) return c->handle_rc;
    cudaIpcMemHandle_t h;
    memcpy(&h, c->handle, 64);
    void* p = nullptr;
    if (cudaIpcOpenMemHandle(&p, h, cudaIpcMemLazyEnablePeerAccess) != cudaSuccess) return SG_ERR_CUDA;
    c->mapped = (char*)p;
  }
  *dev_ptr = c->mapped + c->pool_off;
  return SG_OK;
}

extern "C" int sg_client_declare(sg_client* c, uint64_t need, int32_t priority, uint64_t timeout_ns,
                                 sg_ticket* out) {
  if (!c || !out) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  sg::WireMsg q{}, r{};
  q.op = sg::MSG_DECLARE;
  q.prio = priority;
  q.a = need;
  q.b = timeout_ns;
  int rc = c->request(q, sg::MSG_DECLARED, &r);
  if (rc != SG_OK) return rc;
  if (r.rc != SG_OK) return r.rc;
  if (!c->st.count(r.ticket)) c->st[r.ticket] = TicketState{SG_NOT_READY, 0, 0};   // unless already granted
  *out = r.ticket;
  return SG_OK;
}

extern "C" int sg_client_try(sg_client* c, sg_ticket t, sg_grant* out) {
  if (!c) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  c->drain();
  return c->fill(t, out);
}

extern "C" int sg_client_wait(sg_client* c, sg_ticket t, uint64_t max_block_ns, sg_grant* out) {
  if (!c) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  const uint64_t t0 = now_ns();
  for (;;) {
    const int rc = c->fill(t, out);
    if (rc != SG_NOT_READY) return rc;
    const uint64_t el = now_ns() - t0;
    if (el >= max_block_ns) return SG_NOT_READY;
    sg::WireMsg m;
    const int got = c->recv_one(max_block_ns - el, &m);
    if (got < 0) return SG_ERR_UNKNOWN;
    if (got > 0) c->absorb(m);
  }
}

extern "C" int sg_client_release(sg_client* c, sg_ticket t, uint64_t bytes) {
  if (!c) return SG_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  sg::WireMsg q{}, r{};
  q.op = sg::MSG_RELEASE;
  q.ticket = t;
  q.a = bytes;
  int rc = c->request(q, sg::MSG_RELEASED, &r);
  if (rc != SG_OK) return rc;
  if (r.rc == SG_OK && bytes == 0) c->st.erase(t);
  return r.rc;
}

extern "C" int sg_client_close(sg_client* c) {
  if (!c) return SG_ERR_INVALID;
  if (c->mapped) cudaIpcCloseMemHandle(c->mapped);
  if (c->fd >= 0) close(c->fd);
  delete c;
  return SG_OK;
}
