// Memory dependencies of a planned batch (host side).
//
// A plan is the log of sg_replay: every granted job has an offset in the
// pool and a grant order. Two jobs whose extents overlap must not run at
// the same time; in grant order, a job therefore waits for every earlier
// job that last used any byte of its extent. With these edges alone a batch
// can run with no admission at run time and stay memory-safe.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

#include "../../include/schedgpu.h"

namespace sg {

struct PlanDeps {
  std::vector<uint32_t> order;       // granted jobs in grant order
  std::vector<uint64_t> pred_ptr;    // [n + 1] CSR of predecessors per job
  std::vector<uint32_t> pred;
  std::vector<uint64_t> succ_ptr;    // [n + 1] CSR of successors per job
  std::vector<uint32_t> succ;
};

// Last user of each byte range of the pool, as disjoint [start, end) segments.
class LastUser {
 public:
  // jobs whose segments intersect [a, b); then [a, b) belongs to `job`
  void claim(uint64_t a, uint64_t b, uint32_t job, std::vector<uint32_t>* prev) {
    auto it = seg_.upper_bound(a);
    if (it != seg_.begin()) --it;
    std::vector<std::pair<uint64_t, Seg>> keep;
    while (it != seg_.end() && it->first < b) {
      const uint64_t s = it->first, e = it->second.end;
      if (e <= a) { ++it; continue; }
      prev->push_back(it->second.job);
      if (s < a) keep.push_back({s, Seg{a, it->second.job}});
      if (e > b) keep.push_back({b, Seg{e, it->second.job}});
      it = seg_.erase(it);
    }
    for (auto& kv : keep) seg_[kv.first] = kv.second;
    seg_[a] = Seg{b, job};
  }

 private:
  struct Seg {
    uint64_t end;
    uint32_t job;
  };
  std::map<uint64_t, Seg> seg_;
};

// False if a granted extent leaves the pool.
inline bool plan_deps(const sg_job* jobs, uint32_t n, const sg_record* plan, uint64_t pool_bytes,
                      PlanDeps* out) {
  std::vector<std::pair<int64_t, uint32_t>> ord;
  ord.reserve(n);
  for (uint32_t j = 0; j < n; j++) {
    if (plan[j].status != SG_ST_DONE) continue;   // never granted (too large / timeout)
    if (plan[j].offset + jobs[j].need > pool_bytes) return false;
    ord.push_back({plan[j].grant_seq, j});
  }
  std::sort(ord.begin(), ord.end());
  out->order.clear();
  for (auto& o : ord) out->order.push_back(o.second);
  std::vector<std::vector<uint32_t>> preds(n);
  LastUser lu;
  std::vector<uint32_t> prev;
  for (uint32_t j : out->order) {
    const uint64_t off = plan[j].offset;
    const uint64_t need = jobs[j].need ? jobs[j].need : 1;
    prev.clear();
    lu.claim(off, off + need, j, &prev);
    std::sort(prev.begin(), prev.end());
    prev.erase(std::unique(prev.begin(), prev.end()), prev.end());
    preds[j] = prev;
  }
  out->pred_ptr.assign(n + 1, 0);
  out->succ_ptr.assign(n + 1, 0);
  std::vector<uint64_t> nsucc(n, 0);
  for (uint32_t j = 0; j < n; j++) {
    out->pred_ptr[j + 1] = out->pred_ptr[j] + preds[j].size();
    for (uint32_t p : preds[j]) nsucc[p]++;
  }
  for (uint32_t j = 0; j < n; j++) out->succ_ptr[j + 1] = out->succ_ptr[j] + nsucc[j];
  out->pred.clear();
  out->succ.assign(out->succ_ptr[n], 0);
  std::vector<uint64_t> fill(out->succ_ptr.begin(), out->succ_ptr.end() - 1);
  for (uint32_t j = 0; j < n; j++)
    for (uint32_t p : preds[j]) {
      out->pred.push_back(p);
      out->succ[fill[p]++] = j;
    }
  return true;
}

}  // namespace sg
