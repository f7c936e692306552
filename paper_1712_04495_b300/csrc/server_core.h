// Scheduler server for client processes (arXiv 1712.04495, Sec. III-IV).
//
// In the paper every application process links the scheduler library and
// the processes share the scheduler state (shared memory, a file lock, a
// signal to wake a waiting client, a check that clients are still alive).
// Here one server process owns the pool and the device-resident engine.
// Client processes talk to it over a UNIX socket:
//   HELLO    -> HELLO_OK  (pool size, granule, the pool's CUDA IPC handle)
//   DECLARE  -> DECLARED  (ticket); later GRANT (offset) or TIMEOUT
//   RELEASE  -> RELEASED
// GRANT is pushed to the owner as soon as the engine's grant ring shows the
// ticket; it replaces the paper's signal. A request declared with a finite
// timeout is withdrawn when it expires (TIMEOUT), as a blocking
// pre-allocation that runs out does.
//
// Dead clients (Sec. III-B sanity check): the server learns a client's pid
// from the socket (SO_PEERCRED). When the connection closes, the client's
// tickets stay held until that process has exited. Its kernels may still
// run until then. After that, queued requests are withdrawn and granted
// memory is released, which notifies the waiters. A process that closes its
// connection but keeps running keeps its grants until it exits
// (abandonment).
//
// The engine is reached through ServerEngine, so this file has no CUDA
// dependency: the library instantiates it over the device engine.
#pragma once
#include <errno.h>
#include <fcntl.h>
#include <poll.h>
#include <signal.h>
#include <sys/epoll.h>
#include <sys/socket.h>
#include <sys/un.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/schedgpu.h"
#include "proc.h"

namespace sg {

enum : uint32_t {
  MSG_HELLO = 1, MSG_HELLO_OK = 2, MSG_DECLARE = 3, MSG_DECLARED = 4, MSG_GRANT = 5, MSG_TIMEOUT = 6,
  MSG_RELEASE = 7, MSG_RELEASED = 8, MSG_ERROR = 9
};

constexpr uint32_t kWireVersion = 1;

// One message = one SOCK_SEQPACKET datagram, host byte order (same host).
struct WireMsg {
  uint32_t op;
  uint32_t ticket;
  int32_t prio;
  int32_t rc;          // result code of a reply (SG_*)
  uint64_t a, b, c;    // operands, by op (see the protocol table above)
  uint8_t payload[64]; // HELLO_OK: CUDA IPC handle of the pool's allocation
};
static_assert(sizeof(WireMsg) == 104, "wire message layout");

// What the server needs from an admission engine.
struct ServerEngine {
  virtual ~ServerEngine() {}
  // queue a request; *t receives its ticket
  virtual int declare(uint64_t need, int32_t prio, uint32_t* t) = 0;
  // SG_OK (granted: *offset, *grant_ns), SG_NOT_READY, SG_ERR_TIMEOUT, ...
  virtual int state(uint32_t t, uint64_t* offset, uint64_t* grant_ns) = 0;
  // withdraw a waiting request; returns the state afterwards (as state())
  virtual int cancel(uint32_t t, uint64_t* offset, uint64_t* grant_ns) = 0;
  virtual int release(uint32_t t, uint64_t bytes) = 0;
  // tickets granted since *cursor (advanced), at most max
  virtual int poll(uint32_t* cursor, uint32_t* out, uint32_t max, uint32_t* n) = 0;
  virtual uint64_t pool_bytes() = 0;
  virtual uint64_t granule() = 0;
  // IPC handle of the allocation holding the pool and the pool's offset in it
  virtual int pool_handle(uint8_t handle[64], uint64_t* offset) = 0;
  // called first on the service thread (e.g. to make a device current)
  virtual void on_thread_start() {}
};

struct ServerCounters {
  uint64_t clients_accepted, clients_reaped, declares, grants, timeouts, releases, protocol_errors;
  uint32_t clients_open, tickets_open;
};

inline uint64_t server_now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

class Server {
 public:
  Server(ServerEngine* eng, std::string path) : eng_(eng), path_(std::move(path)) {}
  ~Server() { stop(); }

  // bind, listen and start the service thread: 0, or -errno
  int start() {
    if (path_.size() >= sizeof(sockaddr_un::sun_path)) return -ENAMETOOLONG;
    lfd_ = socket(AF_UNIX, SOCK_SEQPACKET | SOCK_CLOEXEC | SOCK_NONBLOCK, 0);
    if (lfd_ < 0) return -errno;
    sockaddr_un addr{};
    addr.sun_family = AF_UNIX;
    memcpy(addr.sun_path, path_.c_str(), path_.size() + 1);
    unlink(path_.c_str());
    if (bind(lfd_, (sockaddr*)&addr, sizeof addr) != 0 || listen(lfd_, 64) != 0) {
      const int e = errno;
      close(lfd_);
      lfd_ = -1;
      return -e;
    }
    epfd_ = epoll_create1(EPOLL_CLOEXEC);
    if (epfd_ < 0) {
      const int e = errno;
      close(lfd_);
      lfd_ = -1;
      unlink(path_.c_str());
      return -e;
    }
    epoll_event ev{};
    ev.events = EPOLLIN;
    ev.data.fd = lfd_;
    epoll_ctl(epfd_, EPOLL_CTL_ADD, lfd_, &ev);
    run_ = true;
    thr_ = std::thread([this] { loop(); });
    return 0;
  }

  void stop() {
    if (run_.exchange(false) && thr_.joinable()) thr_.join();
    for (auto& kv : clients_) close(kv.first);
    clients_.clear();
    if (lfd_ >= 0) { close(lfd_); lfd_ = -1; unlink(path_.c_str()); }
    if (epfd_ >= 0) { close(epfd_); epfd_ = -1; }
  }

  ServerCounters counters() {
    std::lock_guard<std::mutex> g(stat_mu_);
    return cnt_;
  }

 private:
  struct Client {
    pid_t pid = 0;
    bool hello = false;
    bool closed = false;            // connection gone; tickets held until the process exits
    std::vector<uint32_t> tickets;  // outstanding
  };
  struct Ticket {
    int fd;                         // owner's connection
    uint64_t deadline;              // ~0: none
    bool granted;
    uint64_t held;                  // declared bytes not yet released
  };

  static constexpr uint64_t kNone = ~0ull;

  bool send_msg(int fd, const WireMsg& m) {
    for (;;) {
      ssize_t r = send(fd, &m, sizeof m, MSG_NOSIGNAL | MSG_DONTWAIT);
      if (r == (ssize_t)sizeof m) return true;
      if (r < 0 && errno == EINTR) continue;
      if (r < 0 && (errno == EAGAIN || errno == EWOULDBLOCK)) {
        // the client does not read: wait briefly, then give up on it (the
        // caller drops the connection; other clients are not held up long)
        pollfd p{fd, POLLOUT, 0};
        if (poll(&p, 1, 100) == 1) continue;
      }
      return false;
    }
  }

  void bump(uint64_t ServerCounters::*f) {
    std::lock_guard<std::mutex> g(stat_mu_);
    cnt_.*f += 1;
  }

  void publish_open_counts() {
    std::lock_guard<std::mutex> g(stat_mu_);
    uint32_t open = 0;
    for (auto& kv : clients_) open += kv.second.closed ? 0 : 1;
    cnt_.clients_open = open;
    cnt_.tickets_open = (uint32_t)tickets_.size();
  }

  void forget_ticket(uint32_t t) {
    auto it = tickets_.find(t);
    if (it == tickets_.end()) return;
    if (!it->second.granted) n_waiting_--;
    auto c = clients_.find(it->second.fd);
    if (c != clients_.end()) {
      auto& v = c->second.tickets;
      for (size_t i = 0; i < v.size(); i++)
        if (v[i] == t) { v[i] = v.back(); v.pop_back(); break; }
    }
    tickets_.erase(it);
  }

  void hang_up(int fd) {
    epoll_ctl(epfd_, EPOLL_CTL_DEL, fd, nullptr);
    auto it = clients_.find(fd);
    if (it == clients_.end()) return;
    it->second.closed = true;
    // the descriptor stays open until the client is reaped, so its number
    // cannot be reused by a new connection meanwhile
  }

  // a reply that cannot be delivered drops the connection
  void reply(int fd, const WireMsg& r) {
    if (!send_msg(fd, r)) hang_up(fd);
  }

  void on_message(int fd, Client& cl, const WireMsg& m) {
    WireMsg r{};
    r.ticket = m.ticket;
    if (m.op == MSG_HELLO) {
      r.op = MSG_HELLO_OK;
      r.a = eng_->pool_bytes();
      r.b = eng_->granule();
      r.rc = eng_->pool_handle(r.payload, &r.c);
      r.prio = (int32_t)kWireVersion;
      cl.hello = true;
      reply(fd, r);
      return;
    }
    if (!cl.hello) {
      bump(&ServerCounters::protocol_errors);
      r.op = MSG_ERROR;
      r.rc = SG_ERR_INVALID;
      reply(fd, r);
      return;
    }
    if (m.op == MSG_DECLARE) {
      uint32_t t = 0;
      r.op = MSG_DECLARED;
      r.rc = eng_->declare(m.a, m.prio, &t);
      r.ticket = t;
      if (r.rc == 0) {
        bump(&ServerCounters::declares);
        const uint64_t now = server_now_ns();
        const uint64_t dl = m.b == kNone ? kNone : (now + m.b < now ? kNone : now + m.b);
        tickets_[t] = Ticket{fd, dl, false, m.a};
        n_waiting_++;
        if (dl < next_deadline_) next_deadline_ = dl;
        cl.tickets.push_back(t);
        publish_open_counts();
      }
      reply(fd, r);
      return;
    }
    if (m.op == MSG_RELEASE) {
      r.op = MSG_RELEASED;
      auto it = tickets_.find(m.ticket);
      if (it == tickets_.end() || it->second.fd != fd || !it->second.granted) {
        r.rc = SG_ERR_INVALID;   // not this client's grant
      } else {
        const bool all = m.a == 0 || m.a >= it->second.held;
        r.rc = eng_->release(m.ticket, all ? 0 : m.a);
        if (r.rc == 0) {
          bump(&ServerCounters::releases);
          if (all) forget_ticket(m.ticket);
          else it->second.held -= m.a;            // a partial release keeps the ticket
          publish_open_counts();
        }
      }
      reply(fd, r);
      return;
    }
    bump(&ServerCounters::protocol_errors);
    r.op = MSG_ERROR;
    r.rc = SG_ERR_INVALID;
    reply(fd, r);
  }

  void accept_all() {
    for (;;) {
      int fd = accept4(lfd_, nullptr, nullptr, SOCK_CLOEXEC | SOCK_NONBLOCK);
      if (fd < 0) return;
      ucred cr{};
      socklen_t len = sizeof cr;
      Client cl;
      if (getsockopt(fd, SOL_SOCKET, SO_PEERCRED, &cr, &len) == 0) cl.pid = cr.pid;
      clients_[fd] = cl;
      epoll_event ev{};
      ev.events = EPOLLIN | EPOLLRDHUP;
      ev.data.fd = fd;
      epoll_ctl(epfd_, EPOLL_CTL_ADD, fd, &ev);
      bump(&ServerCounters::clients_accepted);
      publish_open_counts();
    }
  }

  void read_client(int fd) {
    auto it = clients_.find(fd);
    if (it == clients_.end() || it->second.closed) return;
    for (;;) {
      WireMsg m;
      ssize_t r = recv(fd, &m, sizeof m, MSG_DONTWAIT);
      if (r == (ssize_t)sizeof m) {
        on_message(fd, it->second, m);
        if (it->second.closed) return;
        continue;
      }
      if (r < 0 && (errno == EAGAIN || errno == EWOULDBLOCK)) return;
      if (r < 0 && errno == EINTR) continue;
      if (r > 0) bump(&ServerCounters::protocol_errors);   // wrong size: drop the connection
      hang_up(fd);
      publish_open_counts();
      return;
    }
  }

  // grants found on the engine's ring go to their owners
  void deliver_grants() {
    uint32_t buf[256], n = 0;
    for (;;) {
      if (eng_->poll(&cursor_, buf, 256, &n) != 0 && n == 0) return;
      for (uint32_t i = 0; i < n; i++) {
        auto it = tickets_.find(buf[i]);
        if (it == tickets_.end() || it->second.granted) continue;
        it->second.granted = true;
        n_waiting_--;
        bump(&ServerCounters::grants);
        auto c = clients_.find(it->second.fd);
        if (c == clients_.end() || c->second.closed) continue;   // reaped later
        WireMsg m{};
        m.op = MSG_GRANT;
        m.ticket = buf[i];
        m.rc = eng_->state(buf[i], &m.a, &m.b);
        if (!send_msg(it->second.fd, m)) hang_up(it->second.fd);
      }
      if (n < 256) return;
    }
  }

  void expire(uint64_t now) {
    if (now < next_deadline_) return;
    std::vector<uint32_t> due;
    next_deadline_ = kNone;
    for (auto& kv : tickets_) {
      if (kv.second.granted || kv.second.deadline == kNone) continue;
      if (now >= kv.second.deadline) due.push_back(kv.first);
      else if (kv.second.deadline < next_deadline_) next_deadline_ = kv.second.deadline;
    }
    for (uint32_t t : due) {
      uint64_t off = 0, gt = 0;
      const int rc = eng_->cancel(t, &off, &gt);
      auto it = tickets_.find(t);
      if (it == tickets_.end()) continue;
      const int fd = it->second.fd;
      auto c = clients_.find(fd);
      const bool live = c != clients_.end() && !c->second.closed;
      if (rc == 0) {              // granted just before the deadline
        it->second.granted = true;
        n_waiting_--;
        bump(&ServerCounters::grants);
        if (live) {
          WireMsg m{};
          m.op = MSG_GRANT;
          m.ticket = t;
          m.a = off;
          m.b = gt;
          reply(fd, m);
        }
        continue;
      }
      bump(&ServerCounters::timeouts);
      if (live) {
        WireMsg m{};
        m.op = MSG_TIMEOUT;
        m.ticket = t;
        m.rc = rc;
        reply(fd, m);
      }
      forget_ticket(t);
    }
    publish_open_counts();
  }

  // connections that closed: once the process has exited, withdraw its
  // waiting requests and release its grants, then drop it
  void reap(uint64_t now) {
    if (now - last_reap_ < 2000000ull) return;   // every 2 ms
    last_reap_ = now;
    std::vector<int> gone;
    for (auto& kv : clients_)
      if (kv.second.closed && process_exited(kv.second.pid)) gone.push_back(kv.first);
    for (int fd : gone) {
      auto it = clients_.find(fd);
      std::vector<uint32_t> held = it->second.tickets;
      for (uint32_t t : held) {
        auto tk = tickets_.find(t);
        if (tk == tickets_.end()) continue;
        uint64_t off = 0, gt = 0;
        int rc = tk->second.granted ? SG_OK : eng_->cancel(t, &off, &gt);
        if (rc == SG_OK) eng_->release(t, 0);   // held (or granted during the cancel)
        forget_ticket(t);
      }
      clients_.erase(it);
      close(fd);
      bump(&ServerCounters::clients_reaped);
    }
    if (!gone.empty()) publish_open_counts();
  }

  void loop() {
    eng_->on_thread_start();
    epoll_event evs[64];
    while (run_) {
      // wake at once on socket activity; otherwise poll the grant ring every
      // few microseconds while a request waits, less often when all are held
      const long wait_ns = n_waiting_ ? 2000 : (tickets_.empty() ? 1000000 : 50000);
      timespec ts{0, wait_ns};
      const int n = epoll_pwait2(epfd_, evs, 64, &ts, nullptr);
      for (int i = 0; i < n; i++) {
        const int fd = evs[i].data.fd;
        if (fd == lfd_) accept_all();
        else if (evs[i].events & (EPOLLIN | EPOLLRDHUP | EPOLLHUP | EPOLLERR)) read_client(fd);
      }
      deliver_grants();
      const uint64_t now = server_now_ns();
      expire(now);
      reap(now);
    }
  }

  ServerEngine* eng_;
  std::string path_;
  int lfd_ = -1, epfd_ = -1;
  std::atomic<bool> run_{false};
  std::thread thr_;
  std::unordered_map<int, Client> clients_;
  std::unordered_map<uint32_t, Ticket> tickets_;
  uint32_t cursor_ = 0;
  uint64_t last_reap_ = 0;
  uint64_t next_deadline_ = kNone;   // earliest deadline of a waiting request
  uint32_t n_waiting_ = 0;           // tickets not granted yet
  std::mutex stat_mu_;
  ServerCounters cnt_{};
};

}  // namespace sg
