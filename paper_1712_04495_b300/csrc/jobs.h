// Internal interface between the engine runtime and the job kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"

namespace sg {

struct SpmvLayout {
  uint64_t row_ptr, col, val, x, y, scan, total, nchunks;
  bool ptr64;
};
struct GemmLayout {
  uint64_t A, B, C, total;
};

int num_sms();
// texture windows over a context's pool (the SpMV's x gathers): registered
// by sg_init, removed before the context is freed; failures leave the pool
// without windows (the kernels then gather with loads)
void tex_windows_add(const void* owner, const void* base, uint64_t bytes);
void tex_windows_remove(const void* owner);
SpmvLayout spmv_layout(uint64_t rows, uint64_t nnz);
GemmLayout gemm_layout(uint64_t m, uint64_t n, uint64_t k);

int launch_triad(float* a, const float* b, const float* c, float s, uint64_t n, const RelHook& h,
                 cudaStream_t st);
int launch_gen_triad(float* b, float* c, uint64_t n, uint64_t key, cudaStream_t st);
int launch_spmv(const void* row_ptr, int ptr64, const int32_t* col, const float* val, const float* x,
                float* y, uint64_t rows, const RelHook& h, cudaStream_t st);
int launch_gen_spmv(char* base, uint64_t rows, uint64_t nnz, const uint64_t* table, uint64_t key,
                    uint32_t* err, cudaStream_t st, uint64_t* launches);
int launch_gen_bf16(uint16_t* out, uint64_t count, uint64_t key, cudaStream_t st);
int launch_digest(const void* p, uint64_t words, uint64_t* out, const RelHook& h, cudaStream_t st);
// tcgen05 GEMM (gemm.cu): C = A * Bt^T
int launch_gemm(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                const RelHook& h, cudaStream_t st);
// the same with an explicit output tile (an SG_GEMM_TILE code, or 64 / 128 /
// 256 for a 128-row tile of that width; 0 = tuned, else built-in choice)
int launch_gemm_tile(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N, uint32_t K,
                     uint32_t tile, const RelHook& h, cudaStream_t st);
uint32_t gemm_pick_tile(uint32_t M, uint32_t N);
uint32_t gemm_tile_code(uint32_t tile);   // 64 / 128 / 256 -> SG_GEMM_TILE(128, n)
bool gemm_tile_valid(uint32_t tile);
// tile code the autotuner recorded for an M x N output, or 0 (autotune.cu)
uint32_t tuned_tile(uint32_t M, uint32_t N);
// driver entry point and kernel attributes, once (call before stream capture)
int gemm_prepare();

// engine state of a batch that admits on the device (engine.cu, batch.cu)
uint64_t batch_engine_bytes(uint32_t n);
Eng batch_engine_at(char* base, uint32_t n);
int batch_engine_start(const Eng& E, const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
                       uint32_t policy, cudaStream_t st);
// a context's control stream and pool (engine.cu), for the scheduler server
cudaStream_t ctx_control_stream(sg_ctx* c);
char* ctx_pool_base(sg_ctx* c);
uint64_t ctx_pool_bytes(sg_ctx* c);
uint64_t ctx_granule(sg_ctx* c);
// generator + kernel (+ digest when keep_slot) of one job inside its grant
int launch_job(const sg_job& job, char* base, const uint64_t* tables, const RelHook& hook,
               uint64_t* keep_slot, uint32_t* err, cudaStream_t st, uint64_t* launches);

}  // namespace sg
