// Which admitted job the trace runner (sg_run_trace) starts next.
//
// Admission -- the policy pass, grant order and offsets -- happens in the
// device engine; this header only decides when an admitted job starts on a
// stream slot. By default SpMV and GEMM jobs are kept apart: the runner
// alternates phases of the two kinds and triads run beside either. On B300
// an SpMV's random gathers and a GEMM's operand stream both load L2, and
// running them in turn finishes the mixed trace sooner, with shorter tail
// turnaround under load, than overlapping them. SG_RUNF_OVERLAP turns the
// rule off. Long jobs (declared duration of 1 ms or more) run one at a time,
// with short jobs beside them: on B300 each fills the GPU alone, and two of
// them together finish later than one after the other. Host code only, no
// CUDA dependency (tested on the CPU).
#pragma once
#include <stdint.h>

namespace sg {

enum : int { kKindTriad = 0, kKindSpmv = 1, kKindGemm = 2, kKinds = 3 };

// A job declared to run this long fills the GPU on its own for long enough
// that company only slows it (launch gaps are a few percent of it at most).
constexpr uint64_t kLongJobNs = 1000000;

struct RunGate {
  bool apart = true;        // keep SpMV and GEMM jobs apart
  bool one_long = true;     // at most one long job runs at a time
  uint32_t quota = 64;      // starts of one kind per phase while the other kind waits
  int phase = -1;           // kKindSpmv or kKindGemm; -1 before the first phase
  uint32_t phase_started = 0;
  bool other_waits = false; // the kind outside the phase has jobs waiting

  // Kinds that may start now. waiting[k]: admitted jobs of kind k not yet
  // started; head_seq[k]: grant order of the first of them; running[k]:
  // jobs of kind k started and not yet finished.
  void gate(const bool waiting[kKinds], const int64_t head_seq[kKinds], const uint32_t running[kKinds],
            bool may[kKinds]) {
    may[kKindTriad] = may[kKindSpmv] = may[kKindGemm] = true;
    if (!apart) return;
    const bool ws = waiting[kKindSpmv], wg = waiting[kKindGemm];
    if (phase < 0) {
      if (ws || wg) {
        // the first phase is the kind admitted first
        phase = !wg ? kKindSpmv : !ws ? kKindGemm : head_seq[kKindSpmv] < head_seq[kKindGemm] ? kKindSpmv : kKindGemm;
        phase_started = 0;
      }
    } else {
      const int other = phase == kKindSpmv ? kKindGemm : kKindSpmv;
      // the phase ends when its kind has nothing left to start, or when it
      // has used its quota while the other kind waits
      if (waiting[other] && (!waiting[phase] || phase_started >= quota)) {
        phase = other;
        phase_started = 0;
      }
    }
    // the phase's kind starts only once the other kind has drained
    may[kKindSpmv] = phase == kKindSpmv && running[kKindGemm] == 0;
    may[kKindGemm] = phase == kKindGemm && running[kKindSpmv] == 0;
    other_waits = phase >= 0 && waiting[phase == kKindSpmv ? kKindGemm : kKindSpmv];
  }

  // May a job start while long_running long jobs run? `is_long`: its
  // declared duration is at least kLongJobNs.
  bool may_start(bool is_long, uint32_t long_running) const { return !one_long || !is_long || long_running == 0; }

  // A job of `kind` was started: count it against the phase and keep the
  // other kind from starting beside it.
  void started(int kind, bool may[kKinds]) {
    if (!apart) return;
    if (kind == phase && ++phase_started >= quota && other_waits) may[phase] = false;
    if (kind == kKindSpmv) may[kKindGemm] = false;
    if (kind == kKindGemm) may[kKindSpmv] = false;
  }
};

// Of the kinds a slot pool serves (`serves`) that may start and have a job
// waiting, the one whose waiting head was admitted first; -1 if none.
inline int pick_kind(const bool serves[kKinds], const bool may[kKinds], const bool waiting[kKinds],
                     const int64_t head_seq[kKinds]) {
  int kind = -1;
  for (int k = 0; k < kKinds; k++) {
    if (!serves[k] || !may[k] || !waiting[k]) continue;
    if (kind < 0 || head_seq[k] < head_seq[kind]) kind = k;
  }
  return kind;
}

}  // namespace sg
