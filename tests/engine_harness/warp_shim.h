// Host stand-ins for the CUDA intrinsics the device engine uses, so that the
// engine's own source (engine.cuh) runs on the CPU in tests: 32 host threads
// are the lanes of one warp and meet at every warp collective. One warp at a
// time uses the state, as under the engine's lock.
//
// Memory model: a lane's stores through the engine's accessors stay private
// to it (it reads its own) until the warp's next collective, where every
// lane publishes them while all lanes are stopped. That is the view a
// converged warp gives (every lane executes a load before any lane executes
// a later store) with no more ordering than CUDA promises: a value that one
// lane stores is seen by the others only after a warp barrier.
#pragma once
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "schedgpu.h"

#define __device__
#define __host__
#define __global__
#define __shared__
#define __forceinline__ inline
#define SG_FULL 0xffffffffu

struct ShimDim3 { unsigned x, y, z; };
extern thread_local ShimDim3 threadIdx;
extern ShimDim3 gridDim;

namespace sg {

struct WarpSim {
  pthread_barrier_t bar;
  uint64_t slot[32];
};
extern WarpSim* g_warp;
extern thread_local uint32_t t_lane;
extern std::atomic<uint64_t> g_clock;

struct PendingStore {
  void* p;
  uint64_t v;
  uint32_t size;
};
extern thread_local std::vector<PendingStore> t_pending;

inline uint32_t lane_id() { return t_lane; }
inline void publish_pending() {
  for (const PendingStore& x : t_pending) memcpy(x.p, &x.v, x.size);
  t_pending.clear();
}
inline void bar_wait() { pthread_barrier_wait(&g_warp->bar); }
// a warp barrier: all lanes stop, publish their stores, and go on together
inline void warp_bar() {
  bar_wait();
  publish_pending();
  bar_wait();
}
inline uint64_t lane_exchange(uint64_t v, uint32_t src) {
  g_warp->slot[t_lane] = v;
  bar_wait();
  publish_pending();
  const uint64_t r = g_warp->slot[src & 31u];
  bar_wait();
  return r;
}

inline uint64_t globaltimer_ns() { return g_clock.fetch_add(1); }
inline void fence_gpu() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }

template <typename T>
inline T ld_gpu(const T* p) {
  static_assert(sizeof(T) <= 8, "word access");
  for (auto it = t_pending.rbegin(); it != t_pending.rend(); ++it) {
    if (it->p == (const void*)p) {
      T r;
      memcpy(&r, &it->v, sizeof(T));
      return r;
    }
  }
  T r;
  memcpy(&r, (const void*)p, sizeof(T));
  return r;
}
template <typename T>
inline void st_gpu(T* p, T v) {
  PendingStore x{(void*)p, 0, (uint32_t)sizeof(T)};
  memcpy(&x.v, &v, sizeof(T));
  t_pending.push_back(x);
}

}  // namespace sg

inline void __syncwarp(unsigned = SG_FULL) { sg::warp_bar(); }
inline void __syncthreads() { sg::warp_bar(); }
inline unsigned __ballot_sync(unsigned, int p) {
  sg::g_warp->slot[sg::t_lane] = p != 0;
  sg::bar_wait();
  sg::publish_pending();
  unsigned m = 0;
  for (int i = 0; i < 32; i++) m |= (sg::g_warp->slot[i] ? 1u : 0u) << i;
  sg::bar_wait();
  return m;
}
inline int __any_sync(unsigned mask, int p) { return __ballot_sync(mask, p) != 0; }
template <typename T>
inline T __shfl_sync(unsigned, T v, int src) {
  uint64_t b = 0;
  memcpy(&b, &v, sizeof(T));
  b = sg::lane_exchange(b, (uint32_t)src);
  T r;
  memcpy(&r, &b, sizeof(T));
  return r;
}
template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int o) {
  return __shfl_sync(SG_FULL, v, (int)(sg::t_lane ^ (uint32_t)o));
}
inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
inline void __threadfence() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void __threadfence_system() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void __nanosleep(unsigned) {}
inline unsigned atomicCAS(unsigned* p, unsigned cmp, unsigned v) {
  __atomic_compare_exchange_n(p, &cmp, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
  return cmp;
}
inline unsigned atomicOr(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
inline unsigned atomicOr_system(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned atomicExch(unsigned* p, unsigned v) { return __atomic_exchange_n(p, v, __ATOMIC_SEQ_CST); }
