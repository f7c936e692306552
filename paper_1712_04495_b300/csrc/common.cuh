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

// uniform[-1, 1) from 24 random bits: b * 2^-23 - 1, exact in fp32 (the
// product is exact, so one fused multiply-add rounds like the
// product-then-difference it stands for)
__device__ __forceinline__ float uniform_pm1_bits(uint32_t b24) {
  return __fmaf_rn((float)b24, 0x1p-23f, -1.0f);
}
// The two uniforms one hash gives a uniform stream: element 2m takes bits
// 40..63 of h = out(K, m), element 2m + 1 bits 8..31.
__device__ __forceinline__ float2 uniform_pair(uint64_t h) {
  return make_float2(uniform_pm1_bits((uint32_t)(h >> 40)), uniform_pm1_bits((uint32_t)(h >> 8) & 0xFFFFFFu));
}
// element e of the uniform stream with key k
__device__ __forceinline__ float uniform_at(uint64_t k, uint64_t e) {
  const uint64_t h = sm64_at(k, e >> 1);
  return uniform_pm1_bits((e & 1) ? ((uint32_t)(h >> 8) & 0xFFFFFFu) : (uint32_t)(h >> 40));
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

// column index in [0, n) from 32 random bits: multiply-shift, (w * n) >> 32,
// which for n < 2^32 is the high word of the 32 x 32-bit product
__device__ __forceinline__ uint32_t column_of32(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// two fp32 values as a packed bf16 pair (lo in bits 0..15), each rounded to
// nearest, ties to even, by the hardware conversion
__device__ __forceinline__ uint32_t bf16x2_rne_bits(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
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
