// Job kernels for sm_103a: FP32 STREAM triad, FP32 CSR SpMV, the input
// generators of all three job kinds, and the output digest. Each kernel
// that ends a job carries a RelHook: its last block releases the job's
// ticket on the device engine (post-free of Sec. IV).
#include "engine.cuh"
#include "jobs.h"

namespace sg {

constexpr int kThreads = 256;
constexpr int kRowsPerChunk = 4096;  // SpMV CSR build: rows per scan chunk

static int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    g_num_sms = n;
  }
  return g_num_sms;
}

// Short-lived blocks with a fixed amount of work each (the loops stay
// grid-stride, so any grid is correct). Blocks that retire every few
// microseconds let the block scheduler interleave the blocks of every job
// running at the time, and let a co-running GEMM place its persistent CTAs
// as soon as an SM has room, instead of waiting for whole kernels to drain.
static unsigned grid_for(uint64_t work_items, uint64_t per_block) {
  uint64_t want = (work_items + per_block - 1) / per_block;
  if (want < 1) want = 1;
  if (want > (1ull << 30)) want = 1ull << 30;
  return (unsigned)want;
}

// ------------------------------------------------------------------ triad
// a = b + s*c with the product and the sum rounded separately (STREAM).
__global__ void __launch_bounds__(kThreads) k_triad(float* __restrict__ a, const float* __restrict__ b,
                                                    const float* __restrict__ c, float s, uint64_t n,
                                                    int vec, RelHook hook) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t done = 0;
  if (vec) {
    const uint64_t n4 = n >> 2;
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4* c4 = reinterpret_cast<const float4*>(c);
    float4* a4 = reinterpret_cast<float4*>(a);
    uint64_t i = tid;
    for (; i + stride < n4; i += 2 * stride) {
      float4 x0 = __ldcs(b4 + i), y0 = __ldcs(c4 + i);
      float4 x1 = __ldcs(b4 + i + stride), y1 = __ldcs(c4 + i + stride);
      float4 r0, r1;
      r0.x = __fadd_rn(x0.x, __fmul_rn(s, y0.x)); r0.y = __fadd_rn(x0.y, __fmul_rn(s, y0.y));
      r0.z = __fadd_rn(x0.z, __fmul_rn(s, y0.z)); r0.w = __fadd_rn(x0.w, __fmul_rn(s, y0.w));
      r1.x = __fadd_rn(x1.x, __fmul_rn(s, y1.x)); r1.y = __fadd_rn(x1.y, __fmul_rn(s, y1.y));
      r1.z = __fadd_rn(x1.z, __fmul_rn(s, y1.z)); r1.w = __fadd_rn(x1.w, __fmul_rn(s, y1.w));
      __stcs(a4 + i, r0);
      __stcs(a4 + i + stride, r1);
    }
    if (i < n4) {
      float4 x0 = __ldcs(b4 + i), y0 = __ldcs(c4 + i), r0;
      r0.x = __fadd_rn(x0.x, __fmul_rn(s, y0.x)); r0.y = __fadd_rn(x0.y, __fmul_rn(s, y0.y));
      r0.z = __fadd_rn(x0.z, __fmul_rn(s, y0.z)); r0.w = __fadd_rn(x0.w, __fmul_rn(s, y0.w));
      __stcs(a4 + i, r0);
    }
    done = n4 << 2;
  }
  for (uint64_t i = done + tid; i < n; i += stride) a[i] = __fadd_rn(b[i], __fmul_rn(s, c[i]));
  job_epilogue(hook);
}

__global__ void __launch_bounds__(kThreads) k_gen_triad(float* __restrict__ b, float* __restrict__ c,
                                                        uint64_t n, uint64_t kb, uint64_t kc, int vec) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t done = 0;
  if (vec) {
    const uint64_t n4 = n >> 2;
    for (uint64_t i = tid; i < n4; i += stride) {
      uint64_t e = i << 2;
      float4 vb, vc;
      vb.x = uniform_pm1(sm64_at(kb, e)); vb.y = uniform_pm1(sm64_at(kb, e + 1));
      vb.z = uniform_pm1(sm64_at(kb, e + 2)); vb.w = uniform_pm1(sm64_at(kb, e + 3));
      vc.x = uniform_pm1(sm64_at(kc, e)); vc.y = uniform_pm1(sm64_at(kc, e + 1));
      vc.z = uniform_pm1(sm64_at(kc, e + 2)); vc.w = uniform_pm1(sm64_at(kc, e + 3));
      reinterpret_cast<float4*>(b)[i] = vb;
      reinterpret_cast<float4*>(c)[i] = vc;
    }
    done = n4 << 2;
  }
  for (uint64_t i = done + tid; i < n; i += stride) {
    b[i] = uniform_pm1(sm64_at(kb, i));
    c[i] = uniform_pm1(sm64_at(kc, i));
  }
}

// ------------------------------------------------------------------- SpMV
// Four lanes per row, eight rows per warp step. Each lane takes two 16-byte
// aligned vectors of col / val per round (aligned down from the row start;
// elements outside the row are masked), issues both loads before any x
// gather, and the four partial sums meet by shuffles. Latency, not
// bandwidth, limits a CSR row walk, so the kernel runs at full occupancy
// and keeps 8 loads plus 8 gathers in flight per lane.
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

template <typename Idx>
__device__ __forceinline__ float spmv_fma4(const float* __restrict__ x, Idx v, Idx e0, Idx e1,
                                           const int4& c, const float4& w, float acc) {
  if (v >= e0 && v < e1) acc = fmaf(w.x, __ldg(x + c.x), acc);
  if (v + 1 >= e0 && v + 1 < e1) acc = fmaf(w.y, __ldg(x + c.y), acc);
  if (v + 2 >= e0 && v + 2 < e1) acc = fmaf(w.z, __ldg(x + c.z), acc);
  if (v + 3 >= e0 && v + 3 < e1) acc = fmaf(w.w, __ldg(x + c.w), acc);
  return acc;
}

// PtrT (int32 or int64 row_ptr) is also the element index type
template <typename PtrT>
__global__ void __launch_bounds__(kThreads, 6) k_spmv(const PtrT* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const float* __restrict__ val,
                                                      const float* __restrict__ x, float* __restrict__ y,
                                                      uint64_t rows, int vec, RelHook hook) {
  using Idx = PtrT;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t sub = lane & 3u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const Idx nnz = row_ptr[rows];
  const Idx nnz4 = nnz & ~(Idx)3;  // vectors wholly inside the arrays
  for (uint64_t rb = warp * 8; rb < rows; rb += nwarps * 8) {
    const uint64_t r = rb + (lane >> 2);
    Idx e0 = 0, e1 = 0;
    if (r < rows) {
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
        acc = spmv_fma4<Idx>(x, v, e0, e1, ca, wa, acc);
        if (u < e1) acc = spmv_fma4<Idx>(x, u, e0, e1, cb, wb, acc);
      }
    } else {
      for (Idx e = e0 + (Idx)sub; e < e1; e += 4) acc = fmaf(val[e], __ldg(x + col[e]), acc);
    }
    acc += __shfl_xor_sync(SG_FULL, acc, 2);
    acc += __shfl_xor_sync(SG_FULL, acc, 1);
    if (sub == 0 && r < rows) y[r] = acc;
  }
  job_epilogue(hook);
}

// Row length: number of table thresholds <= the row's 32-bit uniform.
__device__ __forceinline__ uint32_t row_len(const uint64_t* T, uint64_t len_key, uint64_t r) {
  uint64_t u = sm64_at(len_key, r) >> 32;
  uint32_t pos = 0;
#pragma unroll
  for (uint32_t step = 32; step; step >>= 1)
    if (T[pos + step - 1] <= u) pos += step;
  return pos;
}

// one block per chunk of kRowsPerChunk rows: sum of its row lengths
__global__ void __launch_bounds__(kThreads) k_spmv_chunk_sums(const uint64_t* __restrict__ table,
                                                              uint64_t len_key, uint64_t rows,
                                                              uint64_t* __restrict__ scan) {
  __shared__ uint64_t T[64];
  __shared__ uint64_t part[kThreads / 32];
  if (threadIdx.x < 64) T[threadIdx.x] = table[threadIdx.x];
  __syncthreads();
  const uint64_t r0 = (uint64_t)blockIdx.x * kRowsPerChunk;
  uint64_t sum = 0;
  for (uint32_t k = threadIdx.x; k < kRowsPerChunk; k += kThreads) {
    uint64_t r = r0 + k;
    if (r < rows) sum += row_len(T, len_key, r);
  }
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(SG_FULL, sum, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kThreads / 32; w++) t += part[w];
    scan[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the chunk sums in place; total at [n]
__global__ void __launch_bounds__(1024) k_spmv_scan_chunks(uint64_t* __restrict__ scan, uint64_t n) {
  __shared__ uint64_t wsum[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint64_t base = 0; base < n; base += 1024) {
    uint64_t i = base + threadIdx.x;
    uint64_t v = i < n ? scan[i] : 0;
    uint64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t t = __shfl_up_sync(SG_FULL, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      uint64_t s = wsum[lane], si = s;
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(SG_FULL, si, o);
        if (lane >= (uint32_t)o) si += t;
      }
      wsum[lane] = si - s;  // exclusive warp offsets
    }
    __syncthreads();
    uint64_t c = carry;
    if (i < n) scan[i] = c + wsum[w] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + wsum[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) scan[n] = carry;
}

// one block per chunk: row_ptr of its rows from the chunk's scanned offset
template <typename PtrT>
__global__ void __launch_bounds__(kThreads) k_spmv_row_ptr(const uint64_t* __restrict__ table,
                                                           uint64_t len_key, uint64_t rows,
                                                           const uint64_t* __restrict__ scan,
                                                           uint64_t nchunks, PtrT* __restrict__ row_ptr,
                                                           uint64_t nnz, uint32_t* err) {
  constexpr int kPer = kRowsPerChunk / kThreads;   // consecutive rows per thread
  __shared__ uint64_t T[64];
  __shared__ uint64_t wsum[kThreads / 32];
  if (threadIdx.x < 64) T[threadIdx.x] = table[threadIdx.x];
  __syncthreads();
  const uint64_t r0 = (uint64_t)blockIdx.x * kRowsPerChunk + (uint64_t)threadIdx.x * kPer;
  uint32_t len[kPer];
  uint64_t mine = 0;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    len[k] = (r0 + k < rows) ? row_len(T, len_key, r0 + k) : 0u;
    mine += len[k];
  }
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(SG_FULL, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  uint64_t woff = 0;
  for (uint32_t k = 0; k < w; k++) woff += wsum[k];
  uint64_t pos = scan[blockIdx.x] + woff + incl - mine;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    if (r0 + k < rows) row_ptr[r0 + k] = (PtrT)(pos < nnz ? pos : nnz);  // clamp keeps reads in bounds
    pos += len[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint64_t total = scan[nchunks];
    row_ptr[rows] = (PtrT)(total < nnz ? total : nnz);
    if (total > nnz && err) atomicOr(err, ERR_NNZ);   // more non-zeros than declared room
  }
}

// columns, values (index e < generated count, at most the capacity) and x.
// Non-zeros come in pairs sharing one hash per quantity: the column pair
// takes the high / low 32 bits, the value pair Box-Muller's cos / sin.
// A thread writes four non-zeros (two pairs) with 16-byte stores.
__global__ void __launch_bounds__(kThreads) k_spmv_fill(int32_t* __restrict__ col, float* __restrict__ val,
                                                        float* __restrict__ x, const uint64_t* total,
                                                        uint64_t cap, uint64_t rows, uint64_t kc,
                                                        uint64_t kv, uint64_t kx) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t nnz = *total < cap ? *total : cap;
  const uint64_t nq = nnz >> 2;
  for (uint64_t q = tid; q < nq; q += stride) {
    const uint64_t m = q << 1;
    const uint64_t hc0 = sm64_at(kc, m), hc1 = sm64_at(kc, m + 1);
    const int4 c = make_int4((int)column_of32((uint32_t)(hc0 >> 32), rows), (int)column_of32((uint32_t)hc0, rows),
                             (int)column_of32((uint32_t)(hc1 >> 32), rows), (int)column_of32((uint32_t)hc1, rows));
    const float2 v0 = normal_pair(sm64_at(kv, m)), v1 = normal_pair(sm64_at(kv, m + 1));
    reinterpret_cast<int4*>(col)[q] = c;
    reinterpret_cast<float4*>(val)[q] = make_float4(v0.x, v0.y, v1.x, v1.y);
  }
  for (uint64_t e = (nq << 2) + tid; e < nnz; e += stride) {
    const uint64_t hc = sm64_at(kc, e >> 1);
    col[e] = (int32_t)column_of32((e & 1) ? (uint32_t)hc : (uint32_t)(hc >> 32), rows);
    const float2 v = normal_pair(sm64_at(kv, e >> 1));
    val[e] = (e & 1) ? v.y : v.x;
  }
  for (uint64_t r = tid; r < rows; r += stride) x[r] = uniform_pm1(sm64_at(kx, r));
}

// -------------------------------------------------------------- GEMM inputs
// eight bf16 per thread per step (one 16-byte store)
__global__ void __launch_bounds__(kThreads) k_gen_bf16(uint16_t* __restrict__ out, uint64_t count,
                                                       uint64_t key) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n8 = count >> 3;
  for (uint64_t i = tid; i < n8; i += stride) {
    uint64_t e = i << 3;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      uint32_t lo = bf16_rne_bits(uniform_pm1(sm64_at(key, e + 2 * k)));
      uint32_t hi = bf16_rne_bits(uniform_pm1(sm64_at(key, e + 2 * k + 1)));
      w[k] = lo | (hi << 16);
    }
    reinterpret_cast<uint4*>(out)[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (uint64_t e = (n8 << 3) + tid; e < count; e += stride)
    out[e] = (uint16_t)bf16_rne_bits(uniform_pm1(sm64_at(key, e)));
}

// ----------------------------------------------------------------- digest
__global__ void __launch_bounds__(kThreads) k_digest(const uint32_t* __restrict__ w, uint64_t n,
                                                     uint64_t* out, RelHook hook) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t s = 0;
  for (uint64_t i = tid; i < n; i += stride) s += mix64((i << 32) | (uint64_t)w[i]);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(SG_FULL, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)s);
  job_epilogue(hook);
}

// ================================================================ launchers
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int launch_triad(float* a, const float* b, const float* c, float s, uint64_t n, const RelHook& h,
                 cudaStream_t st) {
  int vec = aligned16(a) && aligned16(b) && aligned16(c);
  k_triad<<<grid_for(n / 4 + 1, kThreads * 4), kThreads, 0, st>>>(a, b, c, s, n, vec, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_gen_triad(float* b, float* c, uint64_t n, uint64_t key, cudaStream_t st) {
  int vec = aligned16(b) && aligned16(c);
  k_gen_triad<<<grid_for(n / 4 + 1, kThreads * 4), kThreads, 0, st>>>(b, c, n, stream_key(key, 1),
                                                                     stream_key(key, 2), vec);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_spmv(const void* row_ptr, int ptr64, const int32_t* col, const float* val, const float* x,
                float* y, uint64_t rows, const RelHook& h, cudaStream_t st) {
  int vec = aligned16(col) && aligned16(val);
  unsigned grid = grid_for((rows + 7) / 8, (kThreads / 32) * 4);
  if (ptr64)
    k_spmv<int64_t><<<grid, kThreads, 0, st>>>((const int64_t*)row_ptr, col, val, x, y, rows, vec, h);
  else
    k_spmv<int32_t><<<grid, kThreads, 0, st>>>((const int32_t*)row_ptr, col, val, x, y, rows, vec, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

SpmvLayout spmv_layout(uint64_t rows, uint64_t nnz) {
  auto r256 = [](uint64_t x) { return (x + 255) / 256 * 256; };
  SpmvLayout L;
  L.ptr64 = nnz >= (1ull << 31);
  uint64_t nchunks = (rows + kRowsPerChunk - 1) / kRowsPerChunk;
  uint64_t off = 0;
  L.row_ptr = off; off += r256((L.ptr64 ? 8 : 4) * (rows + 1));
  L.col = off; off += r256(4 * nnz);
  L.val = off; off += r256(4 * nnz);
  L.x = off; off += r256(4 * rows);
  L.y = off; off += r256(4 * rows);
  L.scan = off; off += r256(8 * (nchunks + 1));
  L.total = off;
  L.nchunks = nchunks;
  return L;
}

int launch_gen_spmv(char* base, uint64_t rows, uint64_t nnz, const uint64_t* table, uint64_t key,
                    uint32_t* err, cudaStream_t st, uint64_t* launches) {
  if (rows == 0 || rows > 0xFFFFFFFFull) return SG_ERR_INVALID;
  SpmvLayout L = spmv_layout(rows, nnz);
  uint64_t* scan = (uint64_t*)(base + L.scan);
  uint64_t lk = stream_key(key, 1);
  unsigned nch = (unsigned)L.nchunks;
  k_spmv_chunk_sums<<<nch, kThreads, 0, st>>>(table, lk, rows, scan);
  k_spmv_scan_chunks<<<1, 1024, 0, st>>>(scan, L.nchunks);
  if (L.ptr64)
    k_spmv_row_ptr<int64_t><<<nch, kThreads, 0, st>>>(table, lk, rows, scan, L.nchunks,
                                                      (int64_t*)(base + L.row_ptr), nnz, err);
  else
    k_spmv_row_ptr<int32_t><<<nch, kThreads, 0, st>>>(table, lk, rows, scan, L.nchunks,
                                                      (int32_t*)(base + L.row_ptr), nnz, err);
  k_spmv_fill<<<grid_for((nnz / 4 > rows ? nnz / 4 : rows), kThreads * 4), kThreads, 0, st>>>(
      (int32_t*)(base + L.col), (float*)(base + L.val), (float*)(base + L.x), scan + L.nchunks, nnz,
      rows, stream_key(key, 2), stream_key(key, 3), stream_key(key, 4));
  if (launches) *launches += 4;
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_gen_bf16(uint16_t* out, uint64_t count, uint64_t key, cudaStream_t st) {
  if (!aligned16(out)) return SG_ERR_INVALID;
  k_gen_bf16<<<grid_for((count + 7) / 8, kThreads * 4), kThreads, 0, st>>>(out, count, key);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_digest(const void* p, uint64_t words, uint64_t* out, const RelHook& h, cudaStream_t st) {
  k_digest<<<grid_for(words, kThreads * 16), kThreads, 0, st>>>((const uint32_t*)p, words, out, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

GemmLayout gemm_layout(uint64_t m, uint64_t n, uint64_t k) {
  auto r256 = [](uint64_t x) { return (x + 255) / 256 * 256; };
  GemmLayout L;
  L.A = 0;
  L.B = r256(2 * m * k);
  L.C = L.B + r256(2 * n * k);
  L.total = L.C + r256(4 * m * n);
  return L;
}

// Generator + kernel (+ digest) of one job in its grant, on one stream.
int launch_job(const sg_job& job, char* base, const uint64_t* tables, const RelHook& hook,
               uint64_t* keep_slot, uint32_t* err, cudaStream_t st, uint64_t* launches) {
  RelHook none = hook;
  none.active = 0;
  const RelHook& last = keep_slot ? none : hook;
  int rc = SG_OK;
  uint64_t nl = 0;
  const void* out = nullptr;
  uint64_t out_words = 0;
  switch (job.kind) {
    case SG_KIND_TRIAD: {
      uint64_t n = job.p0;
      if (n == 0 || 12 * n > job.need + 0) return SG_ERR_INVALID;
      float* a = (float*)base;
      float* b = a + n;
      float* c = b + n;
      rc = launch_gen_triad(b, c, n, job.key, st);
      if (rc == SG_OK) rc = launch_triad(a, b, c, 3.0f, n, last, st);
      nl = 2;
      out = a;
      out_words = n;
      break;
    }
    case SG_KIND_SPMV: {
      uint64_t rows = job.p0, nnz = job.p1;
      SpmvLayout L = spmv_layout(rows, nnz);
      if (L.total > job.need || !tables) return SG_ERR_INVALID;
      const uint64_t* table = tables + 64ull * job.p2;
      rc = launch_gen_spmv(base, rows, nnz, table, job.key, err, st, &nl);
      if (rc == SG_OK)
        rc = launch_spmv(base + L.row_ptr, L.ptr64, (const int32_t*)(base + L.col),
                         (const float*)(base + L.val), (const float*)(base + L.x),
                         (float*)(base + L.y), rows, last, st);
      nl += 1;
      out = base + L.y;
      out_words = rows;
      break;
    }
    case SG_KIND_GEMM: {
      uint64_t m = job.p0, n = job.p1, k = job.p2;
      GemmLayout L = gemm_layout(m, n, k);
      if (L.total > job.need) return SG_ERR_INVALID;
      rc = launch_gen_bf16((uint16_t*)(base + L.A), m * k, stream_key(job.key, 1), st);
      if (rc == SG_OK) rc = launch_gen_bf16((uint16_t*)(base + L.B), n * k, stream_key(job.key, 2), st);
      if (rc == SG_OK)
        rc = launch_gemm((const uint16_t*)(base + L.A), (const uint16_t*)(base + L.B),
                         (float*)(base + L.C), (uint32_t)m, (uint32_t)n, (uint32_t)k, last, st);
      nl = 3;
      out = base + L.C;
      out_words = m * n;
      break;
    }
    default:
      return SG_ERR_INVALID;
  }
  if (rc == SG_OK && keep_slot) {
    rc = launch_digest(out, out_words, keep_slot, hook, st);
    nl += 1;
  }
  if (launches) *launches += nl;
  return rc;
}

}  // namespace sg

// ============================================================== C ABI
using namespace sg;

static RelHook no_hook() {
  RelHook h;
  memset(&h, 0, sizeof h);
  return h;
}

extern "C" int sg_triad(float* a, const float* b, const float* c, float s, uint64_t n, void* stream) {
  if (!a || !b || !c) return n == 0 ? SG_OK : SG_ERR_INVALID;
  if (n == 0) return SG_OK;
  return launch_triad(a, b, c, s, n, no_hook(), (cudaStream_t)stream);
}

extern "C" int sg_gen_triad(float* b, float* c, uint64_t n, uint64_t key, void* stream) {
  if (n == 0) return SG_OK;
  if (!b || !c) return SG_ERR_INVALID;
  return launch_gen_triad(b, c, n, key, (cudaStream_t)stream);
}

extern "C" int sg_spmv(const void* row_ptr, int ptr64, const int32_t* col, const float* val,
                       const float* x, float* y, uint64_t rows, void* stream) {
  if (rows == 0) return SG_OK;
  if (!row_ptr || !x || !y) return SG_ERR_INVALID;
  return launch_spmv(row_ptr, ptr64, col, val, x, y, rows, no_hook(), (cudaStream_t)stream);
}

extern "C" int sg_gen_spmv(void* base, uint64_t rows, uint64_t nnz, const uint64_t* table_dev,
                           uint64_t key, uint32_t* err_dev, void* stream) {
  if (!base || !table_dev || ((uintptr_t)base & 255u)) return SG_ERR_INVALID;
  return launch_gen_spmv((char*)base, rows, nnz, table_dev, key, err_dev, (cudaStream_t)stream, nullptr);
}

extern "C" int sg_gen_gemm(uint16_t* A, uint16_t* Bt, uint32_t M, uint32_t N, uint32_t K, uint64_t key,
                           void* stream) {
  if (!A || !Bt) return SG_ERR_INVALID;
  int rc = launch_gen_bf16(A, (uint64_t)M * K, stream_key(key, 1), (cudaStream_t)stream);
  if (rc == SG_OK) rc = launch_gen_bf16(Bt, (uint64_t)N * K, stream_key(key, 2), (cudaStream_t)stream);
  return rc;
}

extern "C" int sg_digest(const void* dev_ptr, uint64_t words, uint64_t* out_dev, void* stream) {
  if (!out_dev || (!dev_ptr && words)) return SG_ERR_INVALID;
  if (words == 0) return SG_OK;
  return launch_digest(dev_ptr, words, out_dev, no_hook(), (cudaStream_t)stream);
}
