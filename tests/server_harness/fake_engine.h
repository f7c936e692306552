// Test double of an admission engine for the scheduler server: strict FIFO
// by byte count, offsets from a running sum, no device. Test
// infrastructure only; the library serves the device engine.
#pragma once
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../paper_1712_04495_b300/csrc/server_core.h"

namespace harness {

class CountingFifo final : public sg::ServerEngine {
 public:
  explicit CountingFifo(uint64_t pool) : pool_(pool) {}
  int declare(uint64_t need, int32_t, uint32_t* t) override {
    std::lock_guard<std::mutex> g(mu_);
    if (need > pool_) return SG_ERR_TOO_LARGE;
    *t = next_++;
    req_[*t] = Req{need, SG_NOT_READY, 0, 0};
    queue_.push_back(*t);
    pass();
    return SG_OK;
  }
  int state(uint32_t t, uint64_t* off, uint64_t* gt) override {
    std::lock_guard<std::mutex> g(mu_);
    auto it = req_.find(t);
    if (it == req_.end()) return SG_ERR_INVALID;
    if (it->second.st == SG_OK) { *off = it->second.off; *gt = it->second.gt; }
    return it->second.st;
  }
  int cancel(uint32_t t, uint64_t* off, uint64_t* gt) override {
    {
      std::lock_guard<std::mutex> g(mu_);
      auto it = req_.find(t);
      if (it == req_.end()) return SG_ERR_INVALID;
      if (it->second.st == SG_NOT_READY) {
        for (size_t i = 0; i < queue_.size(); i++)
          if (queue_[i] == t) { queue_.erase(queue_.begin() + i); break; }
        it->second.st = SG_ERR_TIMEOUT;
        pass();
      }
    }
    return state(t, off, gt);
  }
  int release(uint32_t t, uint64_t bytes) override {
    std::lock_guard<std::mutex> g(mu_);
    auto it = req_.find(t);
    if (it == req_.end() || it->second.st != SG_OK) return SG_ERR_INVALID;
    const uint64_t give = (bytes == 0 || bytes >= it->second.need) ? it->second.need : bytes;
    used_ -= give;
    it->second.need -= give;
    if (it->second.need == 0) it->second.st = SG_ERR_INVALID;   // done
    released_ += 1;
    pass();
    return SG_OK;
  }
  int poll(uint32_t* cursor, uint32_t* out, uint32_t max, uint32_t* n) override {
    std::lock_guard<std::mutex> g(mu_);
    uint32_t k = 0;
    while (*cursor < ring_.size() && k < max) out[k++] = ring_[(*cursor)++];
    *n = k;
    return SG_OK;
  }
  uint64_t pool_bytes() override { return pool_; }
  uint64_t granule() override { return 1; }
  int pool_handle(uint8_t handle[64], uint64_t* offset) override {
    memset(handle, 0, 64);
    *offset = 0;
    return SG_ERR_UNKNOWN;   // no device memory to share
  }
  uint64_t used() {
    std::lock_guard<std::mutex> g(mu_);
    return used_;
  }

 private:
  struct Req { uint64_t need; int st; uint64_t off, gt; };
  void pass() {   // strict FIFO by byte count
    while (!queue_.empty()) {
      Req& r = req_[queue_.front()];
      if (r.need > pool_ - used_) break;
      used_ += r.need;
      r.st = SG_OK;
      r.off = used_ - r.need;
      r.gt = sg::server_now_ns();
      ring_.push_back(queue_.front());
      queue_.pop_front();
    }
  }
  std::mutex mu_;
  uint64_t pool_, used_ = 0, released_ = 0;
  uint32_t next_ = 0;
  std::unordered_map<uint32_t, Req> req_;
  std::deque<uint32_t> queue_;
  std::vector<uint32_t> ring_;
};

}  // namespace harness

