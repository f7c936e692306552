// Test harness: the scheduler server of the library (server_core.h) over a
// byte-counting FIFO engine, so that the multi-process protocol and the
// dead-client handling can be exercised on a machine without a GPU. Test
// infrastructure only; the library serves the device engine.
#include "fake_engine.h"

namespace {

using harness::CountingFifo;

struct Harness {
  CountingFifo eng;
  sg::Server srv;
  Harness(uint64_t pool, const char* path) : eng(pool), srv(&eng, path) {}
};

}  // namespace

extern "C" void* harness_start(const char* path, uint64_t pool) {
  Harness* h = new Harness(pool, path);
  if (h->srv.start() != 0) {
    delete h;
    return nullptr;
  }
  return h;
}

extern "C" int harness_counters(void* p, sg_server_counts* out) {
  const sg::ServerCounters c = static_cast<Harness*>(p)->srv.counters();
  out->clients_accepted = c.clients_accepted;
  out->clients_reaped = c.clients_reaped;
  out->declares = c.declares;
  out->grants = c.grants;
  out->timeouts = c.timeouts;
  out->releases = c.releases;
  out->protocol_errors = c.protocol_errors;
  out->clients_open = c.clients_open;
  out->tickets_open = c.tickets_open;
  return 0;
}

extern "C" uint64_t harness_used(void* p) { return static_cast<Harness*>(p)->eng.used(); }

extern "C" void harness_stop(void* p) {
  Harness* h = static_cast<Harness*>(p);
  h->srv.stop();
  delete h;
}
