// Shared device helpers: SplitMix64 element generator, clock, GPU-scope
// memory access and fences. No scheduling logic here.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/schedgpu.h"

#define SG_FULL 0xffffffffu

namespace sg {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output i of the stream
// seeded with state k is mix64(k + (i + 1) * GAMMA).
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * kGamma);
}
// key of data stream s of a job with key k
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t k, uint64_t s) {
  return sm64_at(k, s);
}

// uniform[-1, 1): 24 high bits scaled by 2^-23, minus one; exact in fp32
__device__ __forceinline__ float uniform_pm1(uint64_t h) {
  return __fsub_rn(__fmul_rn((float)(uint32_t)(h >> 40), 0x1p-23f), 1.0f);
}

// Two N(0,1) values by Box-Muller on two 24-bit uniforms taken from one
// hash: r cos(2 pi u2) (even element of a pair) and r sin(2 pi u2) (odd).
__device__ __forceinline__ float2 normal_pair(uint64_t h) {
  float u1 = (float)((uint32_t)(h >> 40) + 1u) * 0x1p-24f;            // (0, 1]
  float u2 = (float)((uint32_t)(h >> 16) & 0xFFFFFFu) * 0x1p-24f;     // [0, 1)
  float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  return make_float2(r * cs, r * sn);
}

// column index in [0, n) from 32 random bits: multiply-shift
__device__ __forceinline__ uint32_t column_of32(uint32_t w, uint64_t n) {
  return (uint32_t)(((uint64_t)w * n) >> 32);
}

// bf16 bits of an fp32 value, round to nearest, ties to even (finite input)
__device__ __forceinline__ uint32_t bf16_rne_bits(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return b >> 16;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Accesses to state shared by kernels running on different SMs: strong
// (relaxed, GPU scope) loads and stores. A weak load may be served from a
// copy that the memory model lets go stale until the reading thread itself
// synchronises; a relaxed load at GPU scope reads the coherent value. Lock
// and flag protocols add the fences that order them (fence.acq_rel.gpu).
// The "memory" clobber keeps the compiler from moving them across other
// memory operations and warp barriers: a lane must see what another lane
// stored before a __syncwarp.
#define SG_LDCG(T, PTX, C)                                                              \
  __device__ __forceinline__ T ld_gpu(const T* p) {                                     \
    T v;                                                                                \
    asm volatile("ld.relaxed.gpu.global." PTX " %0, [%1];" : "=" C(v) : "l"(p) : "memory"); \
    return v;                                                                           \
  }                                                                                     \
  __device__ __forceinline__ void st_gpu(T* p, T v) {                                   \
    asm volatile("st.relaxed.gpu.global." PTX " [%0], %1;" ::"l"(p), C(v) : "memory");  \
  }
SG_LDCG(unsigned int, "u32", "r")
SG_LDCG(int, "s32", "r")
SG_LDCG(unsigned long, "u64", "l")
SG_LDCG(long, "s64", "l")
SG_LDCG(unsigned long long, "u64", "l")
SG_LDCG(long long, "s64", "l")
#undef SG_LDCG

// fence.acq_rel at GPU scope, executed by the calling thread
__device__ __forceinline__ void fence_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }


}  // namespace sg
