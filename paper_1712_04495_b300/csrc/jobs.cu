// Job kernels for sm_103a: FP32 STREAM triad, FP32 CSR SpMV, the input
// generators of all three job kinds, and the output digest. Each kernel
// that ends a job carries a RelHook: its last block releases the job's
// ticket on the device engine (post-free of Sec. IV).
#include <nvtx3/nvToolsExt.h>
#include <mutex>
#include <vector>
#include "engine.cuh"
#include "jobs.h"
#include "texwin.h"
#include "tiles.cuh"

namespace sg {

constexpr uint64_t kRowsPerChunk = kRowsPerScanChunk;

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

// ---------------------------------------------------------------- kernels
// One block per chunk (tiles.cuh); the loops stay grid-stride over chunks.
__global__ void __launch_bounds__(kChunkThreads) k_triad(float* __restrict__ a, const float* __restrict__ b,
                                                         const float* __restrict__ c, float s, uint64_t n,
                                                         int vec, RelHook hook) {
  const uint64_t nch = (n + kTriadChunk - 1) / kTriadChunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) triad_chunk(BlockGroup{}, a, b, c, s, n, vec, ch);
  job_epilogue(hook);
}

__global__ void __launch_bounds__(kChunkThreads) k_gen_triad(float* __restrict__ b, float* __restrict__ c,
                                                             uint64_t n, uint64_t kb, uint64_t kc, int vec) {
  const uint64_t nch = (n + kTriadChunk - 1) / kTriadChunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) gen_triad_chunk(BlockGroup{}, b, c, n, kb, kc, vec, ch);
}

// XG: how x is gathered (XTex when x lies in a texture window of a pool,
// else XLoad); both give the same floats, so y is the same bit for bit.
template <typename PtrT, class XG>
__global__ void __launch_bounds__(kChunkThreads, 6) k_spmv(const PtrT* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col,
                                                           const float* __restrict__ val,
                                                           const XG x, float* __restrict__ y,
                                                           uint64_t rows, int vec, RelHook hook) {
  const uint64_t nch = (rows + kSpmvRowsChunk - 1) / kSpmvRowsChunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x)
    spmv_chunk<BlockGroup, PtrT, XG>(BlockGroup{}, row_ptr, col, val, x, y, rows, vec, ch);
  job_epilogue(hook);
}

__global__ void __launch_bounds__(kChunkThreads) k_spmv_scan_chunks(uint64_t* __restrict__ scan, uint64_t n) {
  __shared__ uint64_t wsum[kChunkThreads / 32 + 1];
  __shared__ uint64_t carry;
  spmv_scan(BlockGroup{}, scan, n, wsum, &carry);
}

template <typename PtrT>
__global__ void __launch_bounds__(kChunkThreads) k_spmv_row_ptr(const uint8_t* __restrict__ lens, uint64_t rows,
                                                                const uint64_t* __restrict__ scan,
                                                                uint64_t nchunks, PtrT* __restrict__ row_ptr,
                                                                uint64_t cap, uint32_t* err) {
  __shared__ uint64_t wsum[kChunkThreads / 32];
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x)
    spmv_row_ptr_chunk<BlockGroup, PtrT>(BlockGroup{}, lens, rows, scan, nchunks, row_ptr, cap, err, ch, wsum);
}

// The SpMV generator's first launch: the row lengths of the scan chunks
// (blocks [0, nchunks)) and, independent of them, the columns and values of
// all cap non-zero slots and x (the other blocks). Slots past the matrix's
// non-zeros get values too and are never read.
__global__ void __launch_bounds__(kChunkThreads) k_spmv_fill(const uint64_t* __restrict__ table, uint64_t len_key,
                                                             uint8_t* __restrict__ lens, uint64_t* __restrict__ scan,
                                                             uint64_t nchunks, int32_t* __restrict__ col,
                                                             float* __restrict__ val, float* __restrict__ x,
                                                             uint64_t cap, uint64_t rows, uint64_t kc,
                                                             uint64_t kv, uint64_t kx) {
  __shared__ uint64_t T[64];
  __shared__ uint32_t T32[64];
  __shared__ uint64_t red[kChunkThreads / 32];
  if (threadIdx.x < 64) {
    const uint64_t t = table[threadIdx.x];
    T[threadIdx.x] = t;
    T32[threadIdx.x] = table_u32(t);
  }
  __syncthreads();
  const uint64_t nch = nchunks + spmv_fill_chunks(cap, rows);
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    if (ch < nchunks) spmv_chunk_sum(BlockGroup{}, T, T32, len_key, rows, lens, scan, ch, red);
    else spmv_fill_chunk(BlockGroup{}, col, val, x, cap, rows, kc, kv, kx, ch - nchunks);
  }
}

__global__ void __launch_bounds__(kChunkThreads) k_gen_bf16(uint16_t* __restrict__ out, uint64_t count,
                                                            uint64_t key) {
  const uint64_t nch = (count + kBf16Chunk - 1) / kBf16Chunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) gen_bf16_chunk(BlockGroup{}, out, count, key, ch);
}

// Both GEMM operands in one launch: the chunks of A, then those of Bt.
__global__ void __launch_bounds__(kChunkThreads) k_gen_gemm(uint16_t* __restrict__ A, uint64_t count_a, uint64_t key_a,
                                                            uint16_t* __restrict__ Bt, uint64_t count_b,
                                                            uint64_t key_b) {
  const uint64_t na = (count_a + kBf16Chunk - 1) / kBf16Chunk;
  const uint64_t nch = na + (count_b + kBf16Chunk - 1) / kBf16Chunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    if (ch < na) gen_bf16_chunk(BlockGroup{}, A, count_a, key_a, ch);
    else gen_bf16_chunk(BlockGroup{}, Bt, count_b, key_b, ch - na);
  }
}

// Measurement kernel, not a step of a job: the random-gather rate that
// bounds the CSR SpMV. Sums x[col[i]] over chunks of kGatherChunk indices,
// one float per chunk (so the gathers are not dropped). Each thread loads four
// columns as one 16-byte vector, then gathers them; with 32 registers, eight
// blocks fill an SM. Of the shapes measured on a B300 (4 to 32 gathers per
// thread, 128 to 1024 threads, 1 to 8 blocks per SM, persistent or not) this
// one sustained the most gathers per second.
constexpr uint64_t kGatherChunk = 4 * kChunkThreads;
template <class XG>
__global__ void __launch_bounds__(kChunkThreads, 8) k_gather_sum(const int32_t* __restrict__ col,
                                                                 const XG x, uint64_t n,
                                                                 float* __restrict__ out) {
  __shared__ float wsum[kChunkThreads / 32];
  const uint64_t nch = (n + kGatherChunk - 1) / kGatherChunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const uint64_t e0 = ch * kGatherChunk + 4 * (uint64_t)threadIdx.x;
    float acc = 0.f;
    if (e0 + 4 <= n) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(col + e0));
      acc = x(c.x) + x(c.y) + x(c.z) + x(c.w);
    } else {
      for (uint64_t e = e0; e < n; e++) acc += x(col[e]);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(SG_FULL, acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < kChunkThreads / 32; w++) t += wsum[w];
      out[ch] = t;
    }
  }
}

__global__ void __launch_bounds__(kChunkThreads) k_digest(const uint32_t* __restrict__ w, uint64_t n,
                                                          uint64_t* out, RelHook hook) {
  const uint64_t nch = (n + kDigestChunk - 1) / kDigestChunk;
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) digest_chunk(BlockGroup{}, w, n, out, ch);
  job_epilogue(hook);
}

// ================================================================ launchers
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ----------------------------------------------- texture windows over pools
// The SpMV gathers x through the texture path when x lies in a pool that a
// context registered: on a B300 that path sustains about 8% more random
// 4-byte gathers per second than the load path. The windows' geometry (1 GiB
// windows every 512 MiB on a B300) is texwin.h's; arrays outside every
// window use loads.
struct TexPool {
  const void* owner = nullptr;
  uintptr_t lo = 0;
  uint64_t bytes = 0;
  TexWinLayout L;
  std::vector<cudaTextureObject_t> tex;
};
static std::mutex g_tex_mu;
static std::vector<TexPool> g_tex_pools;

static void tex_destroy(TexPool& P) {
  for (auto t : P.tex) cudaDestroyTextureObject(t);
  P.tex.clear();
}

void tex_windows_add(const void* owner, const void* base, uint64_t bytes) {
  int dev = 0, maxw = 0, align = 0;
  if (!base || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&align, cudaDevAttrTextureAlignment, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (maxw <= 0 || align <= 0 || ((uintptr_t)base % (uintptr_t)align)) return;
  TexPool P;
  P.owner = owner;
  P.lo = (uintptr_t)base;
  P.bytes = bytes;
  P.L = texwin_layout(bytes, (uint64_t)maxw, (uint64_t)align);
  for (uint64_t i = 0; i < P.L.count; i++) {
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = (char*)base + texwin_start(P.L, i);
    rd.res.linear.desc = cudaCreateChannelDesc<float>();
    rd.res.linear.sizeInBytes = texwin_size(P.L, bytes, i);
    cudaTextureDesc td;
    memset(&td, 0, sizeof td);
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t t = 0;
    if (cudaCreateTextureObject(&t, &rd, &td, nullptr) != cudaSuccess) {
      cudaGetLastError();
      tex_destroy(P);
      return;
    }
    P.tex.push_back(t);
  }
  if (P.tex.empty()) return;
  std::lock_guard<std::mutex> g(g_tex_mu);
  g_tex_pools.push_back(std::move(P));
}

void tex_windows_remove(const void* owner) {
  std::lock_guard<std::mutex> g(g_tex_mu);
  for (size_t i = 0; i < g_tex_pools.size(); i++)
    if (g_tex_pools[i].owner == owner) {
      tex_destroy(g_tex_pools[i]);
      g_tex_pools.erase(g_tex_pools.begin() + i);
      return;
    }
}

// The window holding x[0, n), if any: the texture and x's first element in it.
static bool tex_window_for(const float* x, uint64_t n, XTex* out);

// The texture window for a launch on stream st. A launch into a stream that
// is capturing a CUDA graph gathers with loads: the graph would otherwise
// hold the context's texture objects, which die with the context, while the
// graph may be launched after it.
static bool launch_window(const float* x, uint64_t n, cudaStream_t st, XTex* out) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone && tex_window_for(x, n, out);
}

static bool tex_window_for(const float* x, uint64_t n, XTex* out) {
  const uintptr_t a = (uintptr_t)x;
  std::lock_guard<std::mutex> g(g_tex_mu);
  for (const TexPool& P : g_tex_pools) {
    if (a < P.lo || a - P.lo >= P.bytes) continue;
    const uint64_t off = a - P.lo;
    if (n > (P.bytes >> 2)) return false;
    const int64_t i = texwin_pick(P.L, P.bytes, off, 4 * n);
    if (i < 0) return false;
    out->tex = P.tex[(size_t)i];
    out->base = (int32_t)((off - texwin_start(P.L, (uint64_t)i)) / 4);
    return true;
  }
  return false;
}

int launch_triad(float* a, const float* b, const float* c, float s, uint64_t n, const RelHook& h,
                 cudaStream_t st) {
  int vec = aligned16(a) && aligned16(b) && aligned16(c);
  k_triad<<<grid_for(n, kTriadChunk), kChunkThreads, 0, st>>>(a, b, c, s, n, vec, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_gen_triad(float* b, float* c, uint64_t n, uint64_t key, cudaStream_t st) {
  int vec = aligned16(b) && aligned16(c);
  k_gen_triad<<<grid_for(n, kTriadChunk), kChunkThreads, 0, st>>>(b, c, n, stream_key(key, 1),
                                                                     stream_key(key, 2), vec);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_spmv(const void* row_ptr, int ptr64, const int32_t* col, const float* val, const float* x,
                float* y, uint64_t rows, const RelHook& h, cudaStream_t st) {
  int vec = aligned16(col) && aligned16(val);
  unsigned grid = grid_for(rows, kSpmvRowsChunk);
  XTex xt;
  if (launch_window(x, rows, st, &xt)) {
    if (ptr64)
      k_spmv<int64_t, XTex><<<grid, kChunkThreads, 0, st>>>((const int64_t*)row_ptr, col, val, xt, y, rows, vec, h);
    else
      k_spmv<int32_t, XTex><<<grid, kChunkThreads, 0, st>>>((const int32_t*)row_ptr, col, val, xt, y, rows, vec, h);
  } else {
    if (ptr64)
      k_spmv<int64_t, XLoad><<<grid, kChunkThreads, 0, st>>>((const int64_t*)row_ptr, col, val, XLoad{x}, y, rows,
                                                             vec, h);
    else
      k_spmv<int32_t, XLoad><<<grid, kChunkThreads, 0, st>>>((const int32_t*)row_ptr, col, val, XLoad{x}, y, rows,
                                                             vec, h);
  }
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

SpmvLayout spmv_layout(uint64_t rows, uint64_t nnz) {
  SpmvLayoutHD h = spmv_layout_hd(rows, nnz);
  SpmvLayout L;
  L.row_ptr = h.row_ptr; L.col = h.col; L.val = h.val; L.x = h.x; L.y = h.y; L.scan = h.scan;
  L.total = h.total; L.nchunks = h.nchunks; L.ptr64 = h.ptr64;
  return L;
}

int launch_gen_spmv(char* base, uint64_t rows, uint64_t nnz, const uint64_t* table, uint64_t key,
                    uint32_t* err, cudaStream_t st, uint64_t* launches) {
  if (rows == 0 || rows > 0xFFFFFFFFull) return SG_ERR_INVALID;
  SpmvLayout L = spmv_layout(rows, nnz);
  uint64_t* scan = (uint64_t*)(base + L.scan);
  uint64_t lk = stream_key(key, 1);
  unsigned nch = (unsigned)L.nchunks;
  uint8_t* lens = (uint8_t*)(base + L.y);   // row lengths, in y until the SpMV writes it
  k_spmv_fill<<<grid_for(L.nchunks * kFillChunk + spmv_fill_chunks(nnz, rows) * kFillChunk, kFillChunk),
                kChunkThreads, 0, st>>>(table, lk, lens, scan, L.nchunks, (int32_t*)(base + L.col),
                                        (float*)(base + L.val), (float*)(base + L.x), nnz, rows,
                                        stream_key(key, 2), stream_key(key, 3), stream_key(key, 4));
  k_spmv_scan_chunks<<<1, kChunkThreads, 0, st>>>(scan, L.nchunks);
  if (L.ptr64)
    k_spmv_row_ptr<int64_t><<<nch, kChunkThreads, 0, st>>>(lens, rows, scan, L.nchunks,
                                                           (int64_t*)(base + L.row_ptr), nnz, err);
  else
    k_spmv_row_ptr<int32_t><<<nch, kChunkThreads, 0, st>>>(lens, rows, scan, L.nchunks,
                                                           (int32_t*)(base + L.row_ptr), nnz, err);
  if (launches) *launches += 3;
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_gen_gemm(uint16_t* A, uint64_t count_a, uint64_t key_a, uint16_t* Bt, uint64_t count_b, uint64_t key_b,
                    cudaStream_t st) {
  if (!aligned16(A) || !aligned16(Bt)) return SG_ERR_INVALID;
  k_gen_gemm<<<grid_for(count_a + count_b + kBf16Chunk, kBf16Chunk), kChunkThreads, 0, st>>>(A, count_a, key_a, Bt,
                                                                                            count_b, key_b);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_gen_bf16(uint16_t* out, uint64_t count, uint64_t key, cudaStream_t st) {
  if (!aligned16(out)) return SG_ERR_INVALID;
  k_gen_bf16<<<grid_for(count, kBf16Chunk), kChunkThreads, 0, st>>>(out, count, key);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int launch_digest(const void* p, uint64_t words, uint64_t* out, const RelHook& h, cudaStream_t st) {
  k_digest<<<grid_for(words, kDigestChunk), kChunkThreads, 0, st>>>((const uint32_t*)p, words, out, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

GemmLayout gemm_layout(uint64_t m, uint64_t n, uint64_t k) {
  GemmLayoutHD h = gemm_layout_hd(m, n, k);
  GemmLayout L;
  L.A = h.A; L.B = h.B; L.C = h.C; L.total = h.total;
  return L;
}

// Generator + kernel (+ digest) of one job in its grant, on one stream.
int launch_job(const sg_job& job, char* base, const uint64_t* tables, const RelHook& hook,
               uint64_t* keep_slot, uint32_t* err, cudaStream_t st, uint64_t* launches) {
  static const char* kRange[3] = {"job triad", "job spmv", "job gemm"};
  nvtxRangePushA(job.kind <= SG_KIND_GEMM ? kRange[job.kind] : "job");   // host side of the launch
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
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
      rc = launch_gen_gemm((uint16_t*)(base + L.A), m * k, stream_key(job.key, 1), (uint16_t*)(base + L.B), n * k,
                           stream_key(job.key, 2), st);
      if (rc == SG_OK)
        rc = launch_gemm((const uint16_t*)(base + L.A), (const uint16_t*)(base + L.B),
                         (float*)(base + L.C), (uint32_t)m, (uint32_t)n, (uint32_t)k, last, st);
      nl = 2;
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
  return launch_gen_gemm(A, (uint64_t)M * K, stream_key(key, 1), Bt, (uint64_t)N * K, stream_key(key, 2),
                         (cudaStream_t)stream);
}

extern "C" int sg_spmv_gather_path(const float* x, uint64_t rows) {
  XTex xt;
  return tex_window_for(x, rows, &xt) ? SG_GATHER_TEXTURE : SG_GATHER_LOAD;
}

extern "C" int sg_gather_sum(const int32_t* col, const float* x, uint64_t x_len, uint64_t n, float* out_dev,
                             void* stream) {
  if (n == 0) return SG_OK;
  if (!col || !x || !out_dev || ((uintptr_t)col & 15u)) return SG_ERR_INVALID;
  const unsigned grid = grid_for(n, kGatherChunk);
  XTex xt;
  if (launch_window(x, x_len, (cudaStream_t)stream, &xt))
    k_gather_sum<XTex><<<grid, kChunkThreads, 0, (cudaStream_t)stream>>>(col, xt, n, out_dev);
  else
    k_gather_sum<XLoad><<<grid, kChunkThreads, 0, (cudaStream_t)stream>>>(col, XLoad{x}, n, out_dev);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

extern "C" int sg_digest(const void* dev_ptr, uint64_t words, uint64_t* out_dev, void* stream) {
  if (!out_dev || (!dev_ptr && words)) return SG_ERR_INVALID;
  if (words == 0) return SG_OK;
  return launch_digest(dev_ptr, words, out_dev, no_hook(), (cudaStream_t)stream);
}
