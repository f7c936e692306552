// BF16 GEMM with FP32 accumulation on the sm_100-family tensor cores
// (tcgen05): C[M x N] = A[M x K] * Bt[N x K]^T, all K-contiguous.
//
// Persistent, warp-specialised, one CTA per SM at most (its shared memory
// keeps a second one off the SM, so TMEM allocation never waits):
//   warp 0  TMA producer: 128x64 A tiles and BNx64 B tiles, 128-byte
//           swizzle, into a ring of kStages shared-memory stages;
//   warp 1  TMEM allocator and MMA issuer: one elected lane issues
//           tcgen05.mma (M=128, N=BN, K=16) into one of two TMEM
//           accumulators and commits to mbarriers;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator (each warp owns its
//           32-lane quarter of TMEM), FP32 stores to C; the second
//           accumulator lets the next tile's MMAs overlap this epilogue.
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

constexpr int kBM = 128;
constexpr int kBK = 64;           // 64 bf16 = 128 bytes: one swizzle span
constexpr int kStages = 4;
constexpr int kThreadsG = 192;
constexpr int kGroupM = 16;       // tile raster: 16 M-tiles per band

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

template <int BN>
__global__ void __launch_bounds__(kThreadsG, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
              float* __restrict__ C, uint32_t M, uint32_t N, uint32_t K, RelHook hook) {
  uint32_t* err = &g_tc_err;
  constexpr uint32_t kABytes = kBM * kBK * 2;
  constexpr uint32_t kBBytes = BN * kBK * 2;
  constexpr uint32_t kStageBytes = kABytes + kBBytes;
  constexpr uint32_t kTmemCols = 2 * BN;          // two accumulators
  constexpr uint32_t kIdesc = idesc_bf16(kBM, BN);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_acc_full[2],
      bar_acc_empty[2], bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile uint32_t s_abort;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 1024-byte aligned ring of stages (128-byte swizzle atoms)
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;

  // ragged edges: TMA fills rows / columns outside the tensors with zeros,
  // the epilogue masks rows >= M and columns >= N
  const uint32_t mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN, kb_n = (K + kBK - 1) / kBK;
  const uint32_t tiles = mt * nt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(smem_u32(&bar_acc_full[a]), 1);
      mbar_init(smem_u32(&bar_acc_empty[a]), 128);
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
        for (uint32_t kb = 0; kb < kb_n; kb++) {
          if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &s_abort)) { ok = false; break; }
          const uint32_t sa = ring + stage * kStageBytes;
          const uint32_t fb = smem_u32(&bar_full[stage]);
          mbar_expect_tx(fb, kStageBytes);
          tma_load_2d(sa, &map_a, (int32_t)(kb * kBK), (int32_t)(m * kBM), fb);
          tma_load_2d(sa + kABytes, &map_b, (int32_t)(kb * kBK), (int32_t)(n * BN), fb);
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
        const uint32_t d = tmem + acc * BN;
        for (uint32_t kb = 0; kb < kb_n; kb++) {
          if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &s_abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = ring + stage * kStageBytes;
          const uint32_t sb = sa + kABytes;
#pragma unroll
          for (uint32_t kk = 0; kk < kBK / 16; kk++) {
            mma_bf16(d, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), kIdesc,
                     (kb | kk) != 0);
          }
          mma_commit(smem_u32(&bar_empty[stage]));   // frees the stage when the MMAs finish
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_acc_full[acc]));    // accumulator ready for the epilogue
        if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
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
    uint32_t acc = 0, acc_phase = 0;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
      uint32_t m, n;
      tile_coords(t, mt, nt, m, n);
      bool ok = mbar_wait(smem_u32(&bar_acc_full[acc]), acc_phase, &s_abort);
      if (!__all_sync(SG_FULL, ok)) break;
      tc_fence_after();
      const uint32_t row = m * kBM + q * 32 + lane;
      const uint32_t col0 = n * BN;
      float* crow = C + (uint64_t)row * N + col0;
      const bool vec_ok = (N & 3u) == 0;
#pragma unroll 1
      for (uint32_t c = 0; c < BN / 32; c++) {
        if (col0 + c * 32 >= N) break;             // warp-uniform
        uint32_t r[32];
        tmem_ld_32cols(tmem + ((q * 32u) << 16) + acc * BN + c * 32, r);
        if (row >= M) continue;
        if (vec_ok && col0 + c * 32 + 32 <= N) {
          float4* dst = reinterpret_cast<float4*>(crow + c * 32);
#pragma unroll
          for (int v = 0; v < 8; v++)
            dst[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                 __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
        } else {
#pragma unroll
          for (int v = 0; v < 32; v++)
            if (col0 + c * 32 + v < N) crow[c * 32 + v] = __uint_as_float(r[v]);
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&bar_acc_empty[acc]));
      if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
    }
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

template <int BN>
constexpr uint32_t smem_bytes() {
  return kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
}

// one-time kernel attribute (outside any stream capture)
template <int BN>
int prepare_bn() {
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_bytes<BN>());
  });
  return attr_rc == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

template <int BN>
int launch_bn(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
              const RelHook& h, cudaStream_t st) {
  constexpr uint32_t smem = smem_bytes<BN>();
  if (prepare_bn<BN>() != SG_OK) return SG_ERR_CUDA;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, kBM) || !make_map(&mb, Bt, N, K, BN)) return SG_ERR_CUDA;
  uint32_t tiles = ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
  uint32_t grid = tiles < (uint32_t)num_sms() ? tiles : (uint32_t)num_sms();
  k_gemm_tc<BN><<<grid, kThreadsG, smem, st>>>(ma, mb, C, M, N, K, h);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

}  // namespace

// Output-tile width: the widest of 256 / 128 / 64 that still gives every SM
// at least one tile with at most 1/8 of the width wasted on the ragged
// edge; small GEMMs are latency-bound and take the narrowest (most tiles).
int gemm_pick_bn(uint32_t M, uint32_t N) {
  const uint32_t mt = (M + kBM - 1) / kBM;
  const uint32_t sms = (uint32_t)num_sms();
  for (uint32_t bn : {256u, 128u}) {
    if (N < bn) continue;
    const uint32_t nt = (N + bn - 1) / bn;
    const bool waste_ok = (nt * bn - N) * 8 <= N;
    if (waste_ok && mt * nt >= sms) return (int)bn;
  }
  return 64;
}

int gemm_prepare() {
  if (!encode_fn()) return SG_ERR_CUDA;
  if (prepare_bn<64>() != SG_OK || prepare_bn<128>() != SG_OK || prepare_bn<256>() != SG_OK) return SG_ERR_CUDA;
  return SG_OK;
}

int launch_gemm_bn(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                   int bn, const RelHook& h, cudaStream_t st) {
  if (M == 0 || N == 0) return SG_OK;
  if (K == 0 || K % 8) return SG_ERR_INVALID;       // TMA row stride: a multiple of 16 bytes
  if (((uintptr_t)A & 15) || ((uintptr_t)Bt & 15) || ((uintptr_t)C & 15)) return SG_ERR_INVALID;
  if (!encode_fn()) return SG_ERR_CUDA;
  if (bn <= 0) bn = tuned_tile_n(M, N);
  if (bn <= 0) bn = gemm_pick_bn(M, N);
  if (bn == 256) return launch_bn<256>(A, Bt, C, M, N, K, h, st);
  if (bn == 128) return launch_bn<128>(A, Bt, C, M, N, K, h, st);
  if (bn == 64) return launch_bn<64>(A, Bt, C, M, N, K, h, st);
  return SG_ERR_INVALID;
}

int launch_gemm(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                const RelHook& h, cudaStream_t st) {
  return launch_gemm_bn(A, Bt, C, M, N, K, 0, h, st);
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
                                  uint32_t K, uint32_t tile_n, void* stream) {
  if (!A || !Bt || !C) return SG_ERR_INVALID;
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256) return SG_ERR_INVALID;
  sg::RelHook h;
  memset(&h, 0, sizeof h);
  return sg::launch_gemm_bn(A, Bt, C, M, N, K, (int)tile_n, h, (cudaStream_t)stream);
}

extern "C" uint32_t sg_gemm_tile_n(uint32_t M, uint32_t N) {
  const int t = sg::tuned_tile_n(M, N);
  return (uint32_t)(t > 0 ? t : sg::gemm_pick_bn(M, N));
}

extern "C" int sg_kernel_errors(uint32_t* flags_out) {
  if (!flags_out) return SG_ERR_INVALID;
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, sg::g_tc_err, sizeof v) != cudaSuccess) return SG_ERR_CUDA;
  if (cudaMemcpyToSymbol(sg::g_tc_err, &zero, sizeof zero) != cudaSuccess) return SG_ERR_CUDA;
  *flags_out = v;
  return SG_OK;
}
