// GEMM tile autotuner: on each shape, time every output tile the kernel
// supports (128 x 64, 128 x 128, 128 x 256, 256 x 256) with CUDA events and
// remember the fastest. sg_gemm_bf16 and every job launch consult the
// table before falling back to the built-in choice.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "jobs.h"

namespace sg {
namespace {
std::mutex g_tune_mu;
std::map<std::pair<uint32_t, uint32_t>, uint32_t> g_tuned;   // (M, N) -> tile code
}  // namespace

uint32_t tuned_tile(uint32_t M, uint32_t N) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned.find({M, N});
  return it == g_tuned.end() ? 0 : it->second;
}

}  // namespace sg

using namespace sg;

extern "C" int sg_autotune_gemm(const uint32_t* shapes, uint32_t n_shapes, void* scratch, uint64_t scratch_bytes,
                                uint32_t* chosen, float* best_ms, void* stream) {
  if (!shapes || (!scratch && n_shapes)) return SG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SG_ERR_CUDA;
  RelHook none;
  memset(&none, 0, sizeof none);
  int rc = SG_OK;
  for (uint32_t i = 0; i < n_shapes && rc == SG_OK; i++) {
    const uint32_t M = shapes[3 * i], N = shapes[3 * i + 1], K = shapes[3 * i + 2];
    if (chosen) chosen[i] = 0;
    if (best_ms) best_ms[i] = -1.f;
    const GemmLayout L = gemm_layout(M, N, K);
    if (M == 0 || N == 0 || K == 0 || K % 8 || L.total > scratch_bytes) continue;   // not tunable here
    char* base = (char*)scratch;
    uint16_t* A = (uint16_t*)(base + L.A);
    uint16_t* B = (uint16_t*)(base + L.B);
    float* C = (float*)(base + L.C);
    if (launch_gen_bf16(A, (uint64_t)M * K, 1, st) != SG_OK || launch_gen_bf16(B, (uint64_t)N * K, 2, st) != SG_OK) {
      rc = SG_ERR_CUDA;
      break;
    }
    float best = -1.f;
    uint32_t pick = 0;
    for (uint32_t w : {SG_GEMM_TILE(128, 64), SG_GEMM_TILE(128, 128), SG_GEMM_TILE(128, 256),
                       SG_GEMM_TILE(256, 256)}) {
      const uint32_t tm = w >> 16, tn = w & 0xFFFFu;
      if (w != SG_GEMM_TILE(128, 64) && (N < tn || M < tm)) continue;
      if (launch_gemm_tile(A, B, C, M, N, K, w, none, st) != SG_OK) { rc = SG_ERR_CUDA; break; }   // warm-up
      const int reps = 3;
      std::vector<float> t;
      for (int r = 0; r < reps && rc == SG_OK; r++) {
        cudaEventRecord(e0, st);
        if (launch_gemm_tile(A, B, C, M, N, K, w, none, st) != SG_OK) rc = SG_ERR_CUDA;
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          rc = SG_ERR_CUDA;
        t.push_back(ms);
      }
      if (rc != SG_OK) break;
      std::sort(t.begin(), t.end());
      const float med = t[t.size() / 2];
      if (best < 0.f || med < best) { best = med; pick = w; }
    }
    if (rc != SG_OK) break;
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned[{M, N}] = pick;
    }
    if (chosen) chosen[i] = pick;
    if (best_ms) best_ms[i] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int sg_autotune_clear(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned.clear();
  return SG_OK;
}
