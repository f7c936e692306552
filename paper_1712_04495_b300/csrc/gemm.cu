// BF16 GEMM with FP32 accumulation on the sm_100-family tensor cores
// (tcgen05): C[M x N] = A[M x K] * Bt[N x K]^T, all K-contiguous.
//
// Persistent, warp-specialised, one CTA per SM at most (its shared memory
// keeps a second one off the SM, so TMEM allocation never waits):
//   warp 0  TMA producer: BMx64 A tiles and BNx64 B tiles, 128-byte
//           swizzle, into a ring of shared-memory stages;
//   warp 1  TMEM allocator and MMA issuer: one elected lane issues
//           tcgen05.mma (M=128, N=BN, K=16), one per 128-row half of the
//           tile, and commits to mbarriers;
//   warps 2.. epilogue: tcgen05.ld of the accumulator (a warp reads the
//           32-lane quarter of TMEM its index selects); each 32 x 16 FP32
//           block goes through a swizzled 2 KB staging buffer of the warp
//           and leaves by TMA store (the tensor map clips the ragged
//           edges). Rows of C that are not 16-byte multiples (N % 4 != 0)
//           are stored directly instead.
// The largest tiles keep their shared memory at or below 209 KB, so blocks
// of other jobs' kernels still fit beside them on an SM when jobs are
// co-scheduled.
// Tiles 128 x BN (BN = 64, 128, 256) keep two accumulators in TMEM, so the
// next tile's MMAs overlap this tile's epilogue. The 256 x 256 tile fills
// TMEM with one accumulator (two 128 x 256 halves that share each B tile):
// a third less operand traffic per flop than 128 x 256, paid for with an
// epilogue that the next tile waits for, drained by eight warps.
// Every mbarrier wait is bounded (globaltimer); a wait that runs out raises
// a flag, the CTA drains its own in-flight tensor-core work, frees TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "engine.cuh"
#include "jobs.h"
#include "tc.cuh"

namespace sg {
namespace {

constexpr int kBK = 64;           // 64 bf16 = 128 bytes: one swizzle span
constexpr int kGroupM = 16;       // tile raster: 16 M-tiles per band

template <int BM, int BN>
struct TileCfg {
  static_assert(BM == 128 || (BM == 256 && BN == 256), "tiles: 128 x {64,128,256}, 256 x 256");
  static constexpr int kHalves = BM / 128;                     // M=128 MMAs per K step
  static constexpr uint32_t kABytes = BM * kBK * 2;
  static constexpr uint32_t kBBytes = BN * kBK * 2;
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = BM == 256 ? 3 : 4;
  static constexpr int kAcc = BM == 256 ? 1 : 2;               // accumulators in TMEM
  static constexpr uint32_t kAccCols = kHalves * BN;
  static constexpr uint32_t kTmemCols = kAcc * kAccCols;       // a power of two, <= 512
  static constexpr int kEpiWarps = 4 * kHalves;
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static constexpr uint32_t kStageOut = 32 * 16 * 4;               // per epilogue warp
  static constexpr uint32_t kSmem = kStages * kStageBytes + kEpiWarps * kStageOut + 1024;
};

// flags of GEMM kernels that gave up a bounded wait (read by sg_kernel_errors)
__device__ uint32_t g_tc_err;

__device__ __forceinline__ void tile_coords(uint32_t t, uint32_t mt, uint32_t nt, uint32_t& m, uint32_t& n) {
  uint32_t band = t / (kGroupM * nt);
  uint32_t in = t % (kGroupM * nt);
  uint32_t rows = mt - band * kGroupM;
  if (rows > kGroupM) rows = kGroupM;
  m = band * kGroupM + in % rows;
  n = in / rows;
}

template <int BM, int BN>
__global__ void __launch_bounds__(TileCfg<BM, BN>::kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
              const __grid_constant__ CUtensorMap map_c, float* __restrict__ C, uint32_t M, uint32_t N,
              uint32_t K, RelHook hook) {
  using Cfg = TileCfg<BM, BN>;
  uint32_t* err = &g_tc_err;
  constexpr uint32_t kABytes = Cfg::kABytes;
  constexpr uint32_t kStageBytes = Cfg::kStageBytes;
  constexpr int kStages = Cfg::kStages;
  constexpr int kAcc = Cfg::kAcc;
  constexpr uint32_t kTmemCols = Cfg::kTmemCols;
  constexpr uint32_t kIdesc = idesc_bf16(128, BN);
  constexpr uint32_t kEpiThreads = 32u * Cfg::kEpiWarps;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_acc_full[kAcc],
      bar_acc_empty[kAcc], bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile uint32_t s_abort;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 1024-byte aligned ring of stages (128-byte swizzle atoms)
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;

  // ragged edges: TMA fills rows / columns outside the tensors with zeros,
  // the epilogue masks rows >= M and columns >= N
  const uint32_t mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN, kb_n = (K + kBK - 1) / kBK;
  const uint32_t tiles = mt * nt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int a = 0; a < kAcc; a++) {
      mbar_init(smem_u32(&bar_acc_full[a]), 1);
      mbar_init(smem_u32(&bar_acc_empty[a]), kEpiThreads);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        uint32_t m, n;
        tile_coords(t, mt, nt, m, n);
        // Round t / gridDim.x of the grid: the odd rounds walk K backwards, so
        // that a round starts on the K slices of the band's A that the round
        // before loaded last and L2 still holds
        const bool back = ((t / gridDim.x) & 1u) != 0;
        for (uint32_t kb = 0; kb < kb_n; kb++) {
          if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &s_abort)) { ok = false; break; }
          const uint32_t sa = ring + stage * kStageBytes;
          const uint32_t fb = smem_u32(&bar_full[stage]);
          const int32_t kx = (int32_t)((back ? kb_n - 1 - kb : kb) * kBK);
          mbar_expect_tx(fb, kStageBytes);
          tma_load_2d(sa, &map_a, kx, (int32_t)(m * BM), fb);
          tma_load_2d(sa + kABytes, &map_b, kx, (int32_t)(n * BN), fb);
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok && err) atomicOr(err, 64u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
      bool ok = true;
      for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        if (!mbar_wait(smem_u32(&bar_acc_empty[acc]), acc_phase ^ 1u, &s_abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + acc * Cfg::kAccCols;
        for (uint32_t kb = 0; kb < kb_n; kb++) {
          if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &s_abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = ring + stage * kStageBytes;
          const uint32_t sb = sa + kABytes;
#pragma unroll
          for (uint32_t kk = 0; kk < kBK / 16; kk++) {
#pragma unroll
            for (uint32_t h = 0; h < (uint32_t)Cfg::kHalves; h++)   // rows h*128.. of A, one B tile
              mma_bf16(d + h * BN, smem_desc_sw128(sa + h * (128u * 128u) + kk * 32),
                       smem_desc_sw128(sb + kk * 32), kIdesc, (kb | kk) != 0);   // the first issued starts it
          }
          mma_commit(smem_u32(&bar_empty[stage]));   // frees the stage when the MMAs finish
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_acc_full[acc]));    // accumulator ready for the epilogue
        if (++acc == kAcc) { acc = 0; acc_phase ^= 1u; }
      }
      if (!ok) {
        // give up: let the tensor core finish what was issued before TMEM goes
        mma_commit(smem_u32(&bar_drain));
        volatile uint32_t dummy = 0;
        mbar_wait(smem_u32(&bar_drain), 0, &dummy);
        if (err) atomicOr(err, 64u);
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------- epilogue
    const uint32_t q = warp & 3u;                  // TMEM lane quarter of this warp
    const uint32_t half = (warp - 2u) >> 2;        // 128-row half of the tile it stores
    const uint32_t stg = ring + kStages * kStageBytes + (warp - 2u) * Cfg::kStageOut;   // 512-aligned
    const bool tma_out = (N & 3u) == 0;            // C rows are 16-byte multiples
    bool pending = false;                          // a TMA store may still read `stg`
    uint32_t acc = 0, acc_phase = 0;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
      uint32_t m, n;
      tile_coords(t, mt, nt, m, n);
      bool ok = mbar_wait(smem_u32(&bar_acc_full[acc]), acc_phase, &s_abort);
      if (!__all_sync(SG_FULL, ok)) break;
      tc_fence_after();
      const uint32_t row0 = m * BM + half * 128u + q * 32;   // first row of this warp's slab
      const uint32_t row = row0 + lane;
      const uint32_t col0 = n * BN;
      float* crow = C + (uint64_t)row * N + col0;
#pragma unroll 1
      for (uint32_t c = 0; c < BN / 32; c++) {
        if (col0 + c * 32 >= N) break;             // warp-uniform
        if (row0 >= M) break;                      // the whole slab is past the last row
        uint32_t r[32];
        tmem_ld_32cols(tmem + ((q * 32u) << 16) + acc * Cfg::kAccCols + half * BN + c * 32, r);
        if (tma_out) {
#pragma unroll
          for (uint32_t hs = 0; hs < 2; hs++) {    // two 32 x 16 blocks
            if (col0 + c * 32 + hs * 16 >= N) break;
            if (pending) {
              if (lane == 0) bulk_wait_read();
              __syncwarp();
            }
            // row `lane`: 64 bytes, 16-byte chunk v at chunk v ^ ((lane / 2) % 4)
            // (the 64-byte swizzle of the tensor map; conflict-free for the warp)
#pragma unroll
            for (uint32_t v = 0; v < 4; v++) {
              const uint32_t* x = r + hs * 16 + 4 * v;
              st_shared_v4(stg + lane * 64u + ((v ^ ((lane >> 1) & 3u)) << 4), x[0], x[1], x[2], x[3]);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&map_c, stg, (int32_t)(col0 + c * 32 + hs * 16), (int32_t)row0);
              bulk_commit();
            }
            pending = true;
          }
        } else if (row < M) {
#pragma unroll
          for (int v = 0; v < 32; v++)
            if (col0 + c * 32 + v < N) crow[c * 32 + v] = __uint_as_float(r[v]);
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&bar_acc_empty[acc]));
      if (++acc == kAcc) { acc = 0; acc_phase ^= 1u; }
    }
    // C is complete before the CTA finishes (and before a release hook runs)
    if (pending && lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
  if (s_abort && threadIdx.x == 0) atomicOr(err, 64u);
  job_epilogue(hook);
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// rows x N fp32 output, N contiguous (N % 4 == 0); box = 32 rows x 16, 64-byte swizzle
bool make_map_c(CUtensorMap* map, const float* ptr, uint64_t rows, uint64_t N) {
  cuuint64_t dims[2] = {N, rows};
  cuuint64_t strides[1] = {N * 4};
  cuuint32_t box[2] = {16, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// rows x K bf16 matrix, K contiguous; box = box_rows x 64, 128-byte swizzle
bool make_map(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t K, uint32_t box_rows) {
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {K * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// one-time kernel attribute (outside any stream capture)
template <int BM, int BN>
int prepare_tile() {
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(k_gemm_tc<BM, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)TileCfg<BM, BN>::kSmem);
  });
  return attr_rc == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

template <int BM, int BN>
int launch_tile(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                const RelHook& h, cudaStream_t st) {
  using Cfg = TileCfg<BM, BN>;
  if (prepare_tile<BM, BN>() != SG_OK) return SG_ERR_CUDA;
  CUtensorMap ma, mb, mc;
  if (!make_map(&ma, A, M, K, BM) || !make_map(&mb, Bt, N, K, BN)) return SG_ERR_CUDA;
  memset(&mc, 0, sizeof mc);                       // unused unless N % 4 == 0
  if ((N & 3u) == 0 && !make_map_c(&mc, C, M, N)) return SG_ERR_CUDA;
  uint32_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  uint32_t grid = tiles < (uint32_t)num_sms() ? tiles : (uint32_t)num_sms();
  k_gemm_tc<BM, BN><<<grid, Cfg::kThreads, Cfg::kSmem, st>>>(ma, mb, mc, C, M, N, K, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

}  // namespace

// Built-in output tile when the shape was not tuned: 256 x 256 when every
// SM gets a tile; else the widest 128-row tile that gives at least half of
// the SMs one; small GEMMs are latency-bound and take 128 x 64 (most tiles).
// Candidates must not waste more than 1/8 of the tile on the ragged edges.
uint32_t gemm_pick_tile(uint32_t M, uint32_t N) {
  const uint32_t sms = (uint32_t)num_sms();
  auto fits = [&](uint32_t bm, uint32_t bn, uint32_t min_tiles) {
    if (M < bm || N < bn) return false;
    const uint32_t mt = (M + bm - 1) / bm, nt = (N + bn - 1) / bn;
    const bool waste_ok = (nt * bn - N) * 8 <= N && (mt * bm - M) * 8 <= M;
    return waste_ok && mt * nt >= min_tiles;
  };
  if (fits(256, 256, sms)) return SG_GEMM_TILE(256, 256);
  if (fits(128, 256, sms / 2)) return SG_GEMM_TILE(128, 256);
  if (fits(128, 128, sms / 2)) return SG_GEMM_TILE(128, 128);
  return SG_GEMM_TILE(128, 64);
}

uint32_t gemm_tile_code(uint32_t tile) { return tile != 0 && tile < 65536u ? SG_GEMM_TILE(128, tile) : tile; }

bool gemm_tile_valid(uint32_t tile) {
  switch (gemm_tile_code(tile)) {
    case SG_GEMM_TILE(128, 64):
    case SG_GEMM_TILE(128, 128):
    case SG_GEMM_TILE(128, 256):
    case SG_GEMM_TILE(256, 256): return true;
    default: return false;
  }
}

int gemm_prepare() {
  if (!encode_fn()) return SG_ERR_CUDA;
  if (prepare_tile<128, 64>() != SG_OK || prepare_tile<128, 128>() != SG_OK || prepare_tile<128, 256>() != SG_OK ||
      prepare_tile<256, 256>() != SG_OK)
    return SG_ERR_CUDA;
  return SG_OK;
}

int launch_gemm_tile(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                     uint32_t tile, const RelHook& h, cudaStream_t st) {
  if (M == 0 || N == 0) return SG_OK;
  if (K == 0 || K % 8) return SG_ERR_INVALID;       // TMA row stride: a multiple of 16 bytes
  if (((uintptr_t)A & 15) || ((uintptr_t)Bt & 15) || ((uintptr_t)C & 15)) return SG_ERR_INVALID;
  if (!encode_fn()) return SG_ERR_CUDA;
  if (tile == 0) tile = tuned_tile(M, N);
  if (tile == 0) tile = gemm_pick_tile(M, N);
  switch (gemm_tile_code(tile)) {
    case SG_GEMM_TILE(128, 64): return launch_tile<128, 64>(A, Bt, C, M, N, K, h, st);
    case SG_GEMM_TILE(128, 128): return launch_tile<128, 128>(A, Bt, C, M, N, K, h, st);
    case SG_GEMM_TILE(128, 256): return launch_tile<128, 256>(A, Bt, C, M, N, K, h, st);
    case SG_GEMM_TILE(256, 256): return launch_tile<256, 256>(A, Bt, C, M, N, K, h, st);
    default: return SG_ERR_INVALID;
  }
}

int launch_gemm(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                const RelHook& h, cudaStream_t st) {
  return launch_gemm_tile(A, Bt, C, M, N, K, 0, h, st);
}

}  // namespace sg

extern "C" int sg_gemm_bf16(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N,
                            uint32_t K, void* stream) {
  if (!A || !Bt || !C) return SG_ERR_INVALID;
  sg::RelHook h;
  memset(&h, 0, sizeof h);
  return sg::launch_gemm(A, Bt, C, M, N, K, h, (cudaStream_t)stream);
}

extern "C" int sg_gemm_bf16_tiled(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N,
                                  uint32_t K, uint32_t tile, void* stream) {
  if (!A || !Bt || !C) return SG_ERR_INVALID;
  if (tile != 0 && !sg::gemm_tile_valid(tile)) return SG_ERR_INVALID;
  sg::RelHook h;
  memset(&h, 0, sizeof h);
  return sg::launch_gemm_tile(A, Bt, C, M, N, K, tile, h, (cudaStream_t)stream);
}

extern "C" uint32_t sg_gemm_tile(uint32_t M, uint32_t N) {
  const uint32_t t = sg::tuned_tile(M, N);
  return t ? t : sg::gemm_pick_tile(M, N);
}

extern "C" int sg_kernel_errors(uint32_t* flags_out) {
  if (!flags_out) return SG_ERR_INVALID;
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, sg::g_tc_err, sizeof v) != cudaSuccess) return SG_ERR_CUDA;
  if (cudaMemcpyToSymbol(sg::g_tc_err, &zero, sizeof zero) != cudaSuccess) return SG_ERR_CUDA;
  *flags_out = v;
  return SG_OK;
}
