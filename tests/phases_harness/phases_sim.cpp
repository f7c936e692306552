// Test harness (CPU): the trace runner's start rule (phases.h) driven by a
// discrete simulation of admitted jobs on stream slots. The loop mirrors
// sg_run_trace's: finished jobs leave their slots, the gate decides which
// kinds may start, and each slot pool takes the earliest-admitted job of a
// kind it serves that may start. Returns 0 or the first violated property.
#include <stdint.h>

#include <vector>

#include "phases.h"

using namespace sg;

namespace {

uint64_t next(uint64_t* s) {   // SplitMix64
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// stats[0] = ticks to finish, stats[1] = SpMV/GEMM phases, stats[2] = most
// starts of one kind in one phase while the other kind waited
extern "C" int ph_sim(uint64_t seed, int n_jobs, int n_other, int n_gemm, int apart, int quota, int64_t* stats) {
  uint64_t rng = seed;
  std::vector<int> kind(n_jobs), dur(n_jobs), admit(n_jobs), is_long(n_jobs);
  int t_admit = 0;
  for (int j = 0; j < n_jobs; j++) {            // admitted in index order (grant order)
    const uint64_t r = next(&rng) % 10;
    kind[j] = r < 4 ? kKindTriad : r < 7 ? kKindSpmv : kKindGemm;
    dur[j] = 1 + (int)(next(&rng) % 40);
    is_long[j] = next(&rng) % 5 == 0;   // a long job (declared duration of at least kLongJobNs)
    t_admit += (int)(next(&rng) % 3);
    admit[j] = t_admit;
  }
  RunGate gate;
  gate.apart = apart != 0;
  gate.quota = (uint32_t)quota;
  gate.one_long = apart != 0;
  const int n_all = n_other + n_gemm;
  std::vector<int> slot_job(n_all, -1), end_t(n_all, 0);
  std::vector<int> pend[kKinds];
  size_t pos[kKinds] = {0, 0, 0};
  int admitted = 0, finished = 0, phases = 0, last_phase = -1, run_in_phase = 0, worst = 0;
  std::vector<int> started_at(n_jobs, -1);
  for (int t = 0; t < 100000000; t++) {
    for (int s = 0; s < n_all; s++)
      if (slot_job[s] >= 0 && end_t[s] <= t) { slot_job[s] = -1; finished++; }
    if (finished == n_jobs) {
      if (stats) { stats[0] = t; stats[1] = phases; stats[2] = worst; }
      for (int j = 0; j < n_jobs; j++) if (started_at[j] < admit[j]) return 5;
      return 0;
    }
    while (admitted < n_jobs && admit[admitted] <= t) { pend[kind[admitted]].push_back(admitted); admitted++; }
    bool waiting[kKinds];
    int64_t head[kKinds];
    uint32_t running[kKinds] = {0, 0, 0}, long_running = 0;
    for (int k = 0; k < kKinds; k++) {
      waiting[k] = pos[k] < pend[k].size();
      head[k] = waiting[k] ? pend[k][pos[k]] : INT64_MAX;
    }
    for (int s = 0; s < n_all; s++)
      if (slot_job[s] >= 0) { running[kind[slot_job[s]]]++; long_running += is_long[slot_job[s]]; }
    bool may[kKinds];
    gate.gate(waiting, head, running, may);
    if (gate.apart && gate.phase != last_phase) { phases++; last_phase = gate.phase; run_in_phase = 0; }
    for (int pool = 0; pool < 2; pool++) {
      const int first = pool ? n_other : 0, cnt = pool ? n_gemm : n_other;
      if (cnt == 0) continue;
      const bool serves[kKinds] = {!pool, !pool, pool == 1 || n_gemm == 0};
      while (true) {
        const int k = pick_kind(serves, may, waiting, head);
        if (k < 0) break;
        if (!gate.may_start(is_long[pend[k][pos[k]]], long_running)) {
          may[k] = false;
          continue;
        }
        int slot = -1;
        for (int s = first; s < first + cnt; s++) if (slot_job[s] < 0) { slot = s; break; }
        if (slot < 0) break;
        // property 1: the pick is the earliest-admitted waiting job the pool may start
        for (int k2 = 0; k2 < kKinds; k2++)
          if (serves[k2] && may[k2] && waiting[k2] && head[k2] < head[k]) return 1;
        const int j = pend[k][pos[k]++];
        gate.started(k, may);
        waiting[k] = pos[k] < pend[k].size();
        head[k] = waiting[k] ? pend[k][pos[k]] : INT64_MAX;
        slot_job[slot] = j;
        end_t[slot] = t + dur[j];
        started_at[j] = t;
        running[k]++;
        long_running += is_long[j];
        // property 7: two long jobs never run at the same time
        if (gate.one_long && long_running > 1) return 7;
        if (gate.apart && (k == kKindSpmv || k == kKindGemm)) {
          const int other = k == kKindSpmv ? kKindGemm : kKindSpmv;
          // property 2: SpMV and GEMM never run at the same time
          if (running[other]) return 2;
          if (waiting[other] && ++run_in_phase > worst) worst = run_in_phase;
        }
      }
    }
    // property 3: a free slot stays free only if nothing it serves may start
    for (int pool = 0; pool < 2; pool++) {
      const int first = pool ? n_other : 0, cnt = pool ? n_gemm : n_other;
      bool free_slot = false;
      for (int s = first; s < first + cnt; s++) free_slot |= slot_job[s] < 0;
      const bool serves[kKinds] = {!pool, !pool, pool == 1 || n_gemm == 0};
      if (free_slot && cnt && pick_kind(serves, may, waiting, head) >= 0) return 3;
    }
    // property 4: without the rule every free slot is used while its pool has work
    if (!gate.apart) {
      for (int k = 0; k < kKinds; k++)
        if (waiting[k] && !may[k]) return 4;
    }
  }
  return 6;   // did not finish: a job was never started
}
