// The scheduler server over the device engine: client processes declare,
// wait for, and release memory of one pool that a server process owns
// (arXiv 1712.04495, Sec. III-IV; the protocol and the dead-client handling
// are in server_core.h). Clients map the pool through CUDA IPC and run their
// own kernels on their grants.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "engine.cuh"
#include "jobs.h"
#include "server_core.h"

namespace sg {
namespace {

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

class DeviceEngine final : public ServerEngine {
 public:
  explicit DeviceEngine(sg_ctx* c) : c_(c) {}

  // in the caller's thread (its context is current): the device and the
  // pool's IPC handle, which the service thread only hands out
  int prepare() {
    static_assert(sizeof(cudaIpcMemHandle_t) == 64, "CUDA IPC handle size");
    if (cudaGetDevice(&dev_) != cudaSuccess) return SG_ERR_CUDA;
    handle_rc_ = SG_ERR_CUDA;
    if (!range_fn()) return SG_OK;             // clients then get no pool mapping
    CUdeviceptr base = 0;
    size_t size = 0;
    char* pool = ctx_pool_base(c_);
    if (g_range(&base, &size, (CUdeviceptr)pool) != CUDA_SUCCESS) return SG_OK;
    cudaIpcMemHandle_t h;
    if (cudaIpcGetMemHandle(&h, (void*)base) != cudaSuccess) {
      cudaGetLastError();
      return SG_OK;
    }
    memcpy(handle_, &h, 64);
    offset_ = (uint64_t)(pool - (char*)base);
    handle_rc_ = SG_OK;
    return SG_OK;
  }
  void on_thread_start() override { cudaSetDevice(dev_); }

  int declare(uint64_t need, int32_t prio, uint32_t* t) override {
    sg_ticket tk = 0;
    const int rc = sg_declare(c_, need, prio, &tk);
    *t = tk;
    return rc;
  }
  int state(uint32_t t, uint64_t* offset, uint64_t* grant_ns) override {
    sg_grant g{};
    const int rc = sg_try(c_, t, &g);
    if (rc == SG_OK) { *offset = g.offset; *grant_ns = g.grant_time_ns; }
    return rc;
  }
  int cancel(uint32_t t, uint64_t* offset, uint64_t* grant_ns) override {
    sg_grant g{};
    const int rc = sg_cancel(c_, t, &g);
    if (rc == SG_OK) { *offset = g.offset; *grant_ns = g.grant_time_ns; }
    return rc;
  }
  int release(uint32_t t, uint64_t bytes) override { return sg_release(c_, t, bytes, ctx_control_stream(c_)); }
  int poll(uint32_t* cursor, uint32_t* out, uint32_t max, uint32_t* n) override {
    return sg_poll_grants(c_, cursor, out, max, n);
  }
  uint64_t pool_bytes() override { return ctx_pool_bytes(c_); }
  uint64_t granule() override { return ctx_granule(c_); }
  int pool_handle(uint8_t handle[64], uint64_t* offset) override {
    memcpy(handle, handle_, 64);
    *offset = offset_;
    return handle_rc_;
  }

 private:
  sg_ctx* c_;
  int dev_ = 0;
  int handle_rc_ = SG_ERR_CUDA;
  uint8_t handle_[64] = {};
  uint64_t offset_ = 0;
};

}  // namespace
}  // namespace sg

struct sg_server {
  sg::DeviceEngine eng;
  sg::Server srv;
  sg_server(sg_ctx* c, const char* path) : eng(c), srv(&eng, path) {}
};

extern "C" int sg_server_start(sg_ctx* ctx, const char* socket_path, sg_server** out) {
  if (!ctx || !socket_path || !out) return SG_ERR_INVALID;
  *out = nullptr;
  sg_server* s = new sg_server(ctx, socket_path);
  if (s->eng.prepare() != SG_OK) {
    delete s;
    return SG_ERR_CUDA;
  }
  const int e = s->srv.start();
  if (e != 0) {
    delete s;
    return SG_ERR_INVALID;
  }
  *out = s;
  return SG_OK;
}

extern "C" int sg_server_counters(sg_server* s, sg_server_counts* out) {
  if (!s || !out) return SG_ERR_INVALID;
  const sg::ServerCounters c = s->srv.counters();
  out->clients_accepted = c.clients_accepted;
  out->clients_reaped = c.clients_reaped;
  out->declares = c.declares;
  out->grants = c.grants;
  out->timeouts = c.timeouts;
  out->releases = c.releases;
  out->protocol_errors = c.protocol_errors;
  out->clients_open = c.clients_open;
  out->tickets_open = c.tickets_open;
  return SG_OK;
}

extern "C" int sg_server_stop(sg_server* s) {
  if (!s) return SG_ERR_INVALID;
  s->srv.stop();
  delete s;
  return SG_OK;
}
