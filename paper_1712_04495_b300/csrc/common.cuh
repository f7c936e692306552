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
// hash: r cos(2 pi u2) (even element of a pair) and r sin(2 pi u2) (odd),
// u1 = (b1 + 1) 2^-24 in (0, 1], u2 = b2 2^-24 in [0, 1), r = sqrt(-2 ln u1).
// Each value is within a few units in the last place of the exact one (the
// oracle's fp64 Box-Muller rounded once), in relative terms even near zero:
//  - ln u1 = k ln 2 + ln m, m in [sqrt(1/2), sqrt(2)] from the exact fp32
//    value of b1 + 1; ln m = 2 atanh(s), s = (m - 1) / (m + 1), by its odd
//    series to s^9 (|s| <= 0.172, next term below 2^-28 relative); ln 2 in
//    two parts (Cody and Waite) so that k ln 2 has no rounding for |k| <= 24;
//  - 2 pi u2 = (q + x) pi / 2 with q the nearest integer to 4 u2 and
//    x in [-1/2, 1/2], both exact from the bits of b2; sin and cos of
//    x pi / 2 by their Taylor series to the x^9 and x^10 terms (next terms
//    below 2^-28 on |x pi / 2| <= pi / 4), then the quadrant q.
__device__ __forceinline__ float2 normal_pair(uint64_t h) {
  // r
  const float v = (float)((uint32_t)(h >> 40) + 1u);   // b1 + 1 in [1, 2^24], exact
  const uint32_t vb = __float_as_uint(v);
  const uint32_t mb = vb & 0x7FFFFFu;
  const bool big = mb > 0x3504F3u;                        // mantissa above sqrt(2)
  const float m = __uint_as_float(mb | (big ? 0x3F000000u : 0x3F800000u));
  const float k = (float)((int)(vb >> 23) - 127 + (big ? 1 : 0) - 24);
  const float sq = __fdividef(m - 1.0f, m + 1.0f);
  const float s2 = sq * sq;
  float pl = fmaf(s2, 0x1.c71c72p-3f, 0x1.24924ap-2f);   // 2/9, 2/7
  pl = fmaf(s2, pl, 0x1.99999ap-2f);                     // 2/5
  pl = fmaf(s2, pl, 0x1.555556p-1f);                     // 2/3
  pl = fmaf(s2, pl, 2.0f);
  const float lnu = fmaf(k, 0x1.62e4p-1f, fmaf(k, 0x1.7f7d1cp-20f, sq * pl));   // ln 2 = hi + lo
  const float L = -2.0f * lnu;
  const float r = L > 0.0f ? L * rsqrtf(L) : 0.0f;
  // sin and cos of 2 pi u2
  const int32_t b2 = (int32_t)((h >> 16) & 0xFFFFFFu);
  const int32_t q = (b2 + (1 << 21)) >> 22;               // 0..4
  const float x = (float)(b2 - (q << 22)) * 0x1p-22f;     // [-1/2, 1/2)
  const float x2 = x * x;
  float ps = fmaf(x2, 0x1.507834p-13f, -0x1.32d2ccp-8f);  // (pi/2)^9/9!, -(pi/2)^7/7!
  ps = fmaf(x2, ps, 0x1.466bc6p-4f);                      // (pi/2)^5/5!
  ps = fmaf(x2, ps, -0x1.4abbcep-1f);                     // -(pi/2)^3/3!
  ps = fmaf(x2, ps, 0x1.921fb6p+0f);                      // pi/2
  const float sn = x * ps;
  float pc = fmaf(x2, -0x1.a6d1f2p-16f, 0x1.e1f506p-11f); // -(pi/2)^10/10!, (pi/2)^8/8!
  pc = fmaf(x2, pc, -0x1.55d3c8p-6f);                     // -(pi/2)^6/6!
  pc = fmaf(x2, pc, 0x1.03c1f0p-2f);                      // (pi/2)^4/4!
  pc = fmaf(x2, pc, -0x1.3bd3ccp+0f);                     // -(pi/2)^2/2!
  const float cs = fmaf(x2, pc, 1.0f);
  // quadrant: (sin, cos) of (q + x) pi/2
  const bool odd = q & 1, neg_s = q & 2, neg_c = (q + 1) & 2;
  const float sv = odd ? cs : sn, cv = odd ? sn : cs;
  return make_float2(r * (neg_c ? -cv : cv), r * (neg_s ? -sv : sv));
}

// column index in [0, n) from 32 random bits: multiply-shift, (w * n) >> 32,
// which for n < 2^32 is the high word of the 32 x 32-bit product
__device__ __forceinline__ uint32_t column_of32(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// The uniform of a 16-bit field b of a bf16 stream, b * 2^-15 - 1 (exact in
// fp32): 1 + b 2^-16 is built in the mantissa of a float in [1, 2), and
// 2 (1 + b 2^-16) - 3 is exact.
__device__ __forceinline__ float uniform16(uint32_t b16) {
  return __fmaf_rn(__uint_as_float(0x3F800000u | (b16 << 7)), 2.0f, -3.0f);
}

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
