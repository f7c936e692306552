// Per-chunk bodies of the job kernels. A chunk is the work one thread
// block does; the standalone kernels launch one block per chunk, the
// persistent batch kernel (batch.cu) pulls chunks from its work queue.
// Every function is called by all threads of a block with blockDim.x ==
// kChunkThreads.
#pragma once
#include "engine.cuh"

namespace sg {

constexpr int kChunkThreads = 256;
constexpr uint64_t kTriadChunk = 4096;       // elements per chunk (triad, its generator)
constexpr uint64_t kBf16Chunk = 8192;        // bf16 elements per generator chunk
constexpr uint64_t kSpmvRowsChunk = 256;     // rows per SpMV chunk (8 warps x 8 rows x 4 steps)
constexpr uint64_t kFillChunk = 4096;        // non-zeros per generator chunk
constexpr uint64_t kRowsPerScanChunk = 4096; // rows per scan chunk of the CSR build
constexpr uint64_t kDigestChunk = 4096;      // words per digest chunk

// The threads that work on one chunk: a whole block of kChunkThreads, or one
// kChunkThreads-wide quarter of a larger block with its own named barrier.
struct BlockGroup {
  __device__ __forceinline__ uint32_t t() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

struct SubGroup {
  uint32_t base;     // first thread of the group in the block
  uint32_t bar;      // named barrier id (1..15)
  __device__ __forceinline__ uint32_t t() const { return threadIdx.x - base; }
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"((uint32_t)kChunkThreads) : "memory");
  }
};

// ----------------------------------------------------------- job layouts
// Where each array of a job lives inside its grant (each 256-byte aligned).
struct SpmvLayoutHD {
  uint64_t row_ptr, col, val, x, y, scan, total, nchunks;
  bool ptr64;
};

__host__ __device__ inline uint64_t r256(uint64_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline SpmvLayoutHD spmv_layout_hd(uint64_t rows, uint64_t nnz_cap) {
  SpmvLayoutHD L;
  L.ptr64 = nnz_cap >= (1ull << 31);
  L.nchunks = (rows + kRowsPerScanChunk - 1) / kRowsPerScanChunk;
  uint64_t off = 0;
  L.row_ptr = off; off += r256((L.ptr64 ? 8 : 4) * (rows + 1));
  L.col = off; off += r256(4 * nnz_cap);
  L.val = off; off += r256(4 * nnz_cap);
  L.x = off; off += r256(4 * rows);
  L.y = off; off += r256(4 * rows);
  L.scan = off; off += r256(8 * (L.nchunks + 1));
  L.total = off;
  return L;
}

struct GemmLayoutHD {
  uint64_t A, B, C, total;
};

__host__ __device__ inline GemmLayoutHD gemm_layout_hd(uint64_t m, uint64_t n, uint64_t k) {
  GemmLayoutHD L;
  L.A = 0;
  L.B = r256(2 * m * k);
  L.C = L.B + r256(2 * n * k);
  L.total = L.C + r256(4 * m * n);
  return L;
}

// ------------------------------------------------------------------ triad
// a = b + s*c, product and sum rounded separately (STREAM); 128-bit when
// the three arrays are 16-byte aligned.
template <class G>
__device__ __forceinline__ void triad_chunk(const G& g, float* __restrict__ a, const float* __restrict__ b,
                                            const float* __restrict__ c, float s, uint64_t n, int vec,
                                            uint64_t chunk) {
  const uint64_t e0 = chunk * kTriadChunk;
  const uint64_t e1 = e0 + kTriadChunk < n ? e0 + kTriadChunk : n;
  if (vec && e1 - e0 == kTriadChunk) {
    const float4* b4 = reinterpret_cast<const float4*>(b + e0);
    const float4* c4 = reinterpret_cast<const float4*>(c + e0);
    float4* a4 = reinterpret_cast<float4*>(a + e0);
    float4 x[4], y[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      x[k] = __ldcs(b4 + g.t() + k * kChunkThreads);
      y[k] = __ldcs(c4 + g.t() + k * kChunkThreads);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float4 r;
      r.x = __fadd_rn(x[k].x, __fmul_rn(s, y[k].x));
      r.y = __fadd_rn(x[k].y, __fmul_rn(s, y[k].y));
      r.z = __fadd_rn(x[k].z, __fmul_rn(s, y[k].z));
      r.w = __fadd_rn(x[k].w, __fmul_rn(s, y[k].w));
      __stcs(a4 + g.t() + k * kChunkThreads, r);
    }
  } else {
    for (uint64_t i = e0 + g.t(); i < e1; i += kChunkThreads) a[i] = __fadd_rn(b[i], __fmul_rn(s, c[i]));
  }
}

// b and c from their uniform streams: one hash per two elements
template <class G>
__device__ __forceinline__ void gen_triad_chunk(const G& g, float* __restrict__ b, float* __restrict__ c, uint64_t n,
                                                uint64_t kb, uint64_t kc, int vec, uint64_t chunk) {
  const uint64_t e0 = chunk * kTriadChunk;
  const uint64_t e1 = e0 + kTriadChunk < n ? e0 + kTriadChunk : n;
  if (vec && e1 - e0 == kTriadChunk) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint64_t i = (e0 >> 2) + g.t() + k * kChunkThreads;
      const uint64_t m = i << 1;   // hashes 2i and 2i + 1 cover elements 4i .. 4i + 3
      const float2 b0 = uniform_pair(sm64_at(kb, m)), b1 = uniform_pair(sm64_at(kb, m + 1));
      const float2 c0 = uniform_pair(sm64_at(kc, m)), c1 = uniform_pair(sm64_at(kc, m + 1));
      reinterpret_cast<float4*>(b)[i] = make_float4(b0.x, b0.y, b1.x, b1.y);
      reinterpret_cast<float4*>(c)[i] = make_float4(c0.x, c0.y, c1.x, c1.y);
    }
  } else {
    for (uint64_t i = e0 + g.t(); i < e1; i += kChunkThreads) {
      b[i] = uniform_at(kb, i);
      c[i] = uniform_at(kc, i);
    }
  }
}

// ------------------------------------------------------------ bf16 inputs
// Element e of a bf16 stream: bits 16 (e mod 4) .. 16 (e mod 4) + 15 of
// out(key, e / 4) as a uniform, rounded to bf16. Eight per thread per step
// (two hashes, one 16-byte store); `out` 16-byte aligned.
__device__ __forceinline__ uint32_t bf16_field(uint64_t h, int j) { return (uint32_t)(h >> (16 * j)) & 0xFFFFu; }

template <class G>
__device__ __forceinline__ void gen_bf16_chunk(const G& g, uint16_t* __restrict__ out, uint64_t count, uint64_t key,
                                               uint64_t chunk) {
  const uint64_t e0 = chunk * kBf16Chunk;
  const uint64_t e1 = e0 + kBf16Chunk < count ? e0 + kBf16Chunk : count;
  for (uint64_t e = e0 + 8 * g.t(); e < e1; e += 8 * kChunkThreads) {
    if (e + 8 <= e1) {
      const uint64_t h0 = sm64_at(key, e >> 2), h1 = sm64_at(key, (e >> 2) + 1);
      const uint4 w = make_uint4(bf16x2_rne_bits(uniform16(bf16_field(h0, 0)), uniform16(bf16_field(h0, 1))),
                                 bf16x2_rne_bits(uniform16(bf16_field(h0, 2)), uniform16(bf16_field(h0, 3))),
                                 bf16x2_rne_bits(uniform16(bf16_field(h1, 0)), uniform16(bf16_field(h1, 1))),
                                 bf16x2_rne_bits(uniform16(bf16_field(h1, 2)), uniform16(bf16_field(h1, 3))));
      *reinterpret_cast<uint4*>(out + e) = w;
    } else {
      for (uint64_t i = e; i < e1; i++)
        out[i] = (uint16_t)bf16_rne_bits(uniform16(bf16_field(sm64_at(key, i >> 2), (int)(i & 3))));
    }
  }
}

// ------------------------------------------------------------------- SpMV
// Four lanes per row, eight rows per warp step, four steps per chunk. Each
// lane takes two 16-byte aligned vectors of col / val per round (aligned
// down from the row start; elements outside the row are masked), issues
// both loads before any x gather, and the four partial sums meet by
// shuffles. PtrT (int32 or int64 row_ptr) is also the element index type.
template <typename Idx>
__device__ __forceinline__ void spmv_vec(const int32_t* __restrict__ col, const float* __restrict__ val,
                                         Idx v, Idx nnz4, Idx e1, int4& c, float4& w) {
  if (v < nnz4) {
    c = __ldcs(reinterpret_cast<const int4*>(col + v));
    w = __ldcs(reinterpret_cast<const float4*>(val + v));
  } else {  // last partial vector of the arrays: element loads inside [0, e1)
    c = make_int4(0, 0, 0, 0);
    w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v < e1) { c.x = col[v]; w.x = val[v]; }
    if (v + 1 < e1) { c.y = col[v + 1]; w.y = val[v + 1]; }
    if (v + 2 < e1) { c.z = col[v + 2]; w.z = val[v + 2]; }
    if (v + 3 < e1) { c.w = col[v + 3]; w.w = val[v + 3]; }
  }
}

// How the SpMV reads x[c]: through the load path (XLoad), or through the
// texture path (XTex: a 1-D texture over linear memory in which x starts at
// element `base`). Both return the same float; on a B300 the texture path
// sustains more random 4-byte gathers per second than the load path.
struct XLoad {
  const float* __restrict__ x;
  __device__ __forceinline__ float operator()(int32_t c) const { return __ldg(x + c); }
};
// The persistent batch kernel generates x and runs the SpMV in one launch, so
// x is not read-only for that kernel's lifetime, which the non-coherent path
// of XLoad (and the texture path) requires: it gathers through L2 instead.
struct XLoadL2 {
  const float* __restrict__ x;
  __device__ __forceinline__ float operator()(int32_t c) const { return __ldcg(x + c); }
};
struct XTex {
  cudaTextureObject_t tex;
  int32_t base;
  __device__ __forceinline__ float operator()(int32_t c) const { return tex1Dfetch<float>(tex, base + c); }
};

template <typename Idx, class XG>
__device__ __forceinline__ float spmv_fma4(const XG& x, Idx v, Idx e0, Idx e1,
                                           const int4& c, const float4& w, float acc) {
  if (v >= e0 && v < e1) acc = fmaf(w.x, x(c.x), acc);
  if (v + 1 >= e0 && v + 1 < e1) acc = fmaf(w.y, x(c.y), acc);
  if (v + 2 >= e0 && v + 2 < e1) acc = fmaf(w.z, x(c.z), acc);
  if (v + 3 >= e0 && v + 3 < e1) acc = fmaf(w.w, x(c.w), acc);
  return acc;
}

template <class G, typename PtrT, class XG = XLoad>
__device__ __forceinline__ void spmv_chunk(const G& g, const PtrT* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                           const float* __restrict__ val, const XG& x,
                                           float* __restrict__ y, uint64_t rows, int vec, uint64_t chunk) {
  using Idx = PtrT;
  const uint32_t lane = g.t() & 31u, sub = lane & 3u, warp = g.t() >> 5;
  const Idx nnz = row_ptr[rows];
  const Idx nnz4 = nnz & ~(Idx)3;  // vectors wholly inside the arrays
  const uint64_t r_end = (chunk + 1) * kSpmvRowsChunk < rows ? (chunk + 1) * kSpmvRowsChunk : rows;
  for (uint64_t rb = chunk * kSpmvRowsChunk + warp * 8; rb < r_end; rb += (kChunkThreads / 32) * 8) {
    const uint64_t r = rb + (lane >> 2);
    Idx e0 = 0, e1 = 0;
    if (r < r_end) {
      e0 = row_ptr[r];
      e1 = row_ptr[r + 1];
    }
    float acc = 0.f;
    if (vec) {
      for (Idx v = (e0 & ~(Idx)3) + 4 * (Idx)sub; v < e1; v += 32) {
        const Idx u = v + 16;
        int4 ca, cb = make_int4(0, 0, 0, 0);
        float4 wa, wb = make_float4(0.f, 0.f, 0.f, 0.f);
        spmv_vec<Idx>(col, val, v, nnz4, e1, ca, wa);
        if (u < e1) spmv_vec<Idx>(col, val, u, nnz4, e1, cb, wb);
        acc = spmv_fma4<Idx, XG>(x, v, e0, e1, ca, wa, acc);
        if (u < e1) acc = spmv_fma4<Idx, XG>(x, u, e0, e1, cb, wb, acc);
      }
    } else {
      for (Idx e = e0 + (Idx)sub; e < e1; e += 4) acc = fmaf(val[e], x(col[e]), acc);
    }
    acc += __shfl_xor_sync(SG_FULL, acc, 2);
    acc += __shfl_xor_sync(SG_FULL, acc, 1);
    if (sub == 0 && r < r_end) y[r] = acc;
  }
}

// ------------------------------------------------------ SpMV CSR build
// Row length: number of table thresholds <= the row's 32-bit uniform u.
// T32 is T saturated to 32 bits (2^32 - 1 for thresholds at or above 2^32):
// for every u below 2^32 - 1 it gives the same count with 32-bit compares;
// u = 2^32 - 1 takes the 64-bit table.
__device__ __forceinline__ uint32_t table_u32(uint64_t t) { return (t >> 32) ? 0xFFFFFFFFu : (uint32_t)t; }

__device__ __forceinline__ uint32_t row_len(const uint64_t* T, const uint32_t* T32, uint64_t len_key, uint64_t r) {
  const uint32_t u = (uint32_t)(sm64_at(len_key, r) >> 32);
  uint32_t pos = 0;
  if (u != 0xFFFFFFFFu) {
#pragma unroll
    for (uint32_t step = 32; step; step >>= 1)
      if (T32[pos + step - 1] <= u) pos += step;
  } else {
#pragma unroll
    for (uint32_t step = 32; step; step >>= 1)
      if (T[pos + step - 1] <= (uint64_t)u) pos += step;
  }
  return pos;
}

// block-wide sum of a uint64 per thread (all threads get the result)
template <class G>
__device__ __forceinline__ uint64_t block_sum_u64(const G& g, uint64_t v, uint64_t* red /* [kChunkThreads/32] */) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(SG_FULL, v, o);
  g.sync();
  if ((g.t() & 31) == 0) red[g.t() >> 5] = v;
  g.sync();
  uint64_t t = 0;
  for (int w = 0; w < kChunkThreads / 32; w++) t += red[w];
  g.sync();
  return t;
}

// Row lengths of scan chunk `chunk`: each thread takes 16 consecutive rows,
// stores their lengths as 16 bytes (a length is at most 64) at lens[first
// row], and the block's total goes to scan[chunk]. `lens` is the job's y
// array, free until the SpMV writes y; the row_ptr pass reads the lengths
// back instead of hashing every row a second time. The last thread of a
// ragged chunk writes zeros past the last row, inside y (4 bytes per row,
// rounded up to 256). T and T32 (its 32-bit saturation) in shared memory.
template <class G>
__device__ __forceinline__ void spmv_chunk_sum(const G& g, const uint64_t* T, const uint32_t* T32, uint64_t len_key,
                                               uint64_t rows,
                                               uint8_t* __restrict__ lens, uint64_t* __restrict__ scan,
                                               uint64_t chunk, uint64_t* red) {
  constexpr int kPer = kRowsPerScanChunk / kChunkThreads;
  static_assert(kPer == 16, "one 16-byte store of lengths per thread");
  const uint64_t r0 = chunk * kRowsPerScanChunk + (uint64_t)g.t() * kPer;
  uint64_t sum = 0;
  if (r0 < rows) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const uint32_t l = (r0 + k < rows) ? row_len(T, T32, len_key, r0 + k) : 0u;
      w[k >> 2] |= l << (8 * (k & 3));
      sum += l;
    }
    *reinterpret_cast<uint4*>(lens + r0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  sum = block_sum_u64(g, sum, red);
  if (g.t() == 0) scan[chunk] = sum;
}

// exclusive scan of scan[0..n) in place, total at scan[n] (one block)
template <class G>
__device__ __forceinline__ void spmv_scan(const G& g, uint64_t* __restrict__ scan, uint64_t n, uint64_t* wsum,
                                          uint64_t* carry) {
  const uint32_t lane = g.t() & 31, w = g.t() >> 5;
  constexpr uint32_t nw = kChunkThreads / 32;
  if (g.t() == 0) *carry = 0;
  g.sync();
  for (uint64_t base = 0; base < n; base += kChunkThreads) {
    const uint64_t i = base + g.t();
    const uint64_t v = i < n ? scan[i] : 0;
    uint64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t t = __shfl_up_sync(SG_FULL, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    g.sync();
    if (g.t() == 0) {
      uint64_t run = 0;
      for (uint32_t k = 0; k < nw; k++) {
        uint64_t t = wsum[k];
        wsum[k] = run;
        run += t;
      }
      wsum[nw] = run;
    }
    g.sync();
    const uint64_t c = *carry;
    if (i < n) scan[i] = c + wsum[w] + incl - v;
    g.sync();
    if (g.t() == 0) *carry = c + wsum[nw];
    g.sync();
  }
  if (g.t() == 0) scan[n] = *carry;
}

// row_ptr of the rows of scan chunk `chunk` (16 consecutive rows per
// thread, their lengths read back from `lens` as one 16-byte load; the
// row_ptr entries leave as 16-byte stores).
template <class G, typename PtrT>
__device__ __forceinline__ void spmv_row_ptr_chunk(const G& g, const uint8_t* __restrict__ lens, uint64_t rows,
                                                   const uint64_t* __restrict__ scan, uint64_t nchunks,
                                                   PtrT* __restrict__ row_ptr, uint64_t cap, uint32_t* err,
                                                   uint64_t chunk, uint64_t* wsum) {
  constexpr int kPer = kRowsPerScanChunk / kChunkThreads;
  const uint64_t r0 = chunk * kRowsPerScanChunk + (uint64_t)g.t() * kPer;
  uint4 q = make_uint4(0u, 0u, 0u, 0u);
  if (r0 < rows) q = *reinterpret_cast<const uint4*>(lens + r0);
  const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
  uint32_t len[kPer];
  uint64_t mine = 0;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    len[k] = (qw[k >> 2] >> (8 * (k & 3))) & 0xFFu;
    mine += len[k];
  }
  const uint32_t lane = g.t() & 31, w = g.t() >> 5;
  uint64_t incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(SG_FULL, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  g.sync();
  if (lane == 31) wsum[w] = incl;
  g.sync();
  uint64_t woff = 0;
  for (uint32_t k = 0; k < w; k++) woff += wsum[k];
  uint64_t pos = scan[chunk] + woff + incl - mine;
  PtrT v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    v[k] = (PtrT)(pos < cap ? pos : cap);  // clamp keeps reads in bounds
    pos += len[k];
  }
  if (r0 + kPer <= rows) {  // row_ptr + r0 is 64-byte aligned: r0 is a multiple of 16
    constexpr int kVec = 16 / sizeof(PtrT);
#pragma unroll
    for (int k = 0; k < kPer; k += kVec) {
      uint4 u;
      memcpy(&u, &v[k], 16);
      *reinterpret_cast<uint4*>(row_ptr + r0 + k) = u;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPer; k++)
      if (r0 + k < rows) row_ptr[r0 + k] = v[k];
  }
  if (chunk == 0 && g.t() == 0) {
    uint64_t total = scan[nchunks];
    row_ptr[rows] = (PtrT)(total < cap ? total : cap);
    if (total > cap && err) atomicOr(err, ERR_NNZ);   // more non-zeros than declared room
  }
}

// Columns, values and x. Non-zeros come in pairs sharing one hash per
// quantity: the column pair takes the high / low 32 bits, the value pair
// Box-Muller's cos / sin. A thread writes four non-zeros (two pairs) with
// 16-byte stores. Chunk c covers non-zeros [c*kFillChunk, ...) and rows
// [c*kFillChunk/4, ...) of x, so ceil(max(nnz, 4 rows) / kFillChunk) chunks
// cover both.
template <class G>
__device__ __forceinline__ void spmv_fill_chunk(const G& g, int32_t* __restrict__ col, float* __restrict__ val,
                                                float* __restrict__ x, uint64_t nnz, uint64_t rows,
                                                uint64_t kc, uint64_t kv, uint64_t kx, uint64_t chunk) {
  const uint64_t e0 = chunk * kFillChunk;
  const uint64_t e1 = e0 + kFillChunk < nnz ? e0 + kFillChunk : nnz;
  const uint32_t n32 = (uint32_t)rows;   // rows < 2^32 (checked at launch)
  for (uint64_t e = e0 + 4 * g.t(); e < e1; e += 4 * kChunkThreads) {
    if (e + 4 <= e1) {
      const uint64_t m = e >> 1;
      const uint64_t hc0 = sm64_at(kc, m), hc1 = sm64_at(kc, m + 1);
      const int4 cc = make_int4((int)column_of32((uint32_t)(hc0 >> 32), n32), (int)column_of32((uint32_t)hc0, n32),
                                (int)column_of32((uint32_t)(hc1 >> 32), n32), (int)column_of32((uint32_t)hc1, n32));
      const float2 v0 = normal_pair(sm64_at(kv, m)), v1 = normal_pair(sm64_at(kv, m + 1));
      *reinterpret_cast<int4*>(col + e) = cc;
      *reinterpret_cast<float4*>(val + e) = make_float4(v0.x, v0.y, v1.x, v1.y);
    } else {
      for (uint64_t i = e; i < e1; i++) {
        const uint64_t hc = sm64_at(kc, i >> 1);
        col[i] = (int32_t)column_of32((i & 1) ? (uint32_t)hc : (uint32_t)(hc >> 32), n32);
        const float2 v = normal_pair(sm64_at(kv, i >> 1));
        val[i] = (i & 1) ? v.y : v.x;
      }
    }
  }
  // x: two rows per hash, one 8-byte store (x0 is even, x 8-byte aligned)
  const uint64_t x0 = chunk * (kFillChunk / 4);
  const uint64_t x1 = x0 + kFillChunk / 4 < rows ? x0 + kFillChunk / 4 : rows;
  for (uint64_t r = x0 + 2 * g.t(); r < x1; r += 2 * kChunkThreads) {
    const float2 u = uniform_pair(sm64_at(kx, r >> 1));
    if (r + 1 < x1) *reinterpret_cast<float2*>(x + r) = u;
    else x[r] = u.x;
  }
}

__host__ __device__ __forceinline__ uint64_t spmv_fill_chunks(uint64_t nnz_cap, uint64_t rows) {
  const uint64_t need = nnz_cap > 4 * rows ? nnz_cap : 4 * rows;
  return (need + kFillChunk - 1) / kFillChunk;
}

// ----------------------------------------------------------------- digest
// adds sum of mix64((i << 32) | w[i]) over the chunk into *out
template <class G>
__device__ __forceinline__ void digest_chunk(const G& g, const uint32_t* __restrict__ w, uint64_t n, uint64_t* out,
                                             uint64_t chunk) {
  const uint64_t e0 = chunk * kDigestChunk;
  const uint64_t e1 = e0 + kDigestChunk < n ? e0 + kDigestChunk : n;
  uint64_t s = 0;
  for (uint64_t i = e0 + g.t(); i < e1; i += kChunkThreads) s += mix64((i << 32) | (uint64_t)w[i]);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(SG_FULL, s, o);
  if ((g.t() & 31) == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)s);
}

}  // namespace sg
