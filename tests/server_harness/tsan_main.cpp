// Race check of the scheduler server: the server (service thread) over the
// test engine, eight client threads speaking the wire protocol, and the main
// thread reading the counters meanwhile. Built with -fsanitize=thread by the
// test; exits 0 when every request was served and the counters agree.
#include <sys/socket.h>
#include <sys/un.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "fake_engine.h"

namespace {

constexpr int kClients = 8;
constexpr int kRounds = 150;

bool roundtrip(int fd, const sg::WireMsg& q, uint32_t want, sg::WireMsg* r, uint32_t* granted) {
  if (send(fd, &q, sizeof q, MSG_NOSIGNAL) != (ssize_t)sizeof q) return false;
  for (;;) {
    if (recv(fd, r, sizeof *r, 0) != (ssize_t)sizeof *r) return false;
    if (r->op == sg::MSG_GRANT) { if (granted) *granted = r->ticket + 1; continue; }
    if (r->op == want) return true;
    if (r->op != sg::MSG_TIMEOUT) return false;
  }
}

void client(const std::string& path, int id, std::atomic<int>* failures, std::atomic<int>* served) {
  const int fd = socket(AF_UNIX, SOCK_SEQPACKET, 0);
  sockaddr_un a{};
  a.sun_family = AF_UNIX;
  snprintf(a.sun_path, sizeof a.sun_path, "%s", path.c_str());
  if (fd < 0 || connect(fd, (sockaddr*)&a, sizeof a) != 0) { failures->fetch_add(1); return; }
  sg::WireMsg q{}, r{};
  q.op = sg::MSG_HELLO;
  q.prio = (int32_t)sg::kWireVersion;
  if (!roundtrip(fd, q, sg::MSG_HELLO_OK, &r, nullptr)) { failures->fetch_add(1); close(fd); return; }
  for (int i = 0; i < kRounds; i++) {
    q = sg::WireMsg{};
    q.op = sg::MSG_DECLARE;
    q.a = 100 + (uint64_t)((id * 7 + i * 13) % 400);   // bytes of a 1000-byte pool
    q.b = ~0ull;
    uint32_t granted = 0;
    if (!roundtrip(fd, q, sg::MSG_DECLARED, &r, &granted) || r.rc != SG_OK) { failures->fetch_add(1); break; }
    const uint32_t t = r.ticket;
    while (granted != t + 1) {                            // wait for the pushed grant
      if (recv(fd, &r, sizeof r, 0) != (ssize_t)sizeof r) { failures->fetch_add(1); close(fd); return; }
      if (r.op == sg::MSG_GRANT && r.ticket == t) granted = t + 1;
    }
    q = sg::WireMsg{};
    q.op = sg::MSG_RELEASE;
    q.ticket = t;
    if (!roundtrip(fd, q, sg::MSG_RELEASED, &r, nullptr) || r.rc != SG_OK) { failures->fetch_add(1); break; }
    served->fetch_add(1);
  }
  close(fd);
}

}  // namespace

int main(int argc, char** argv) {
  const std::string path = argc > 1 ? argv[1] : "/tmp/sg_tsan.sock";
  harness::CountingFifo eng(1000);
  sg::Server srv(&eng, path);
  if (srv.start() != 0) return 2;
  std::atomic<int> failures{0}, served{0};
  std::atomic<bool> done{false};
  std::thread reader([&] {                                 // counters read while the server runs
    while (!done.load()) {
      const sg::ServerCounters c = srv.counters();
      (void)c;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  });
  std::vector<std::thread> cl;
  for (int i = 0; i < kClients; i++) cl.emplace_back(client, path, i, &failures, &served);
  for (auto& t : cl) t.join();
  done = true;
  reader.join();
  // the connections closed; the clients were threads of this live process,
  // so their (released) tickets need no reaping
  const sg::ServerCounters c = srv.counters();
  srv.stop();
  const int want = kClients * kRounds;
  std::printf("served %d of %d, declares %llu grants %llu releases %llu, failures %d\n", served.load(), want,
              (unsigned long long)c.declares, (unsigned long long)c.grants, (unsigned long long)c.releases,
              failures.load());
  const bool ok = failures.load() == 0 && served.load() == want && c.declares == (uint64_t)want &&
                  c.grants == (uint64_t)want && c.releases == (uint64_t)want && eng.used() == 0;
  return ok ? 0 : 1;
}
