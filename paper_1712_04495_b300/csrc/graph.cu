// Batching through one captured CUDA graph: a static co-schedule.
//
// The device replay (sg_replay) decides, on the logical clock with declared
// durations, where each job lives in the pool and in what order jobs are
// granted. This file turns that plan into one CUDA graph: every job is a
// chain of kernel nodes (its generator kernels, then its kernel, then
// optionally its output digest), and a job depends on every job that used
// any byte of its extent before it in grant order. Jobs that share no memory run
// concurrently; jobs that share memory never overlap in time, so the graph
// is memory-safe by construction and needs no engine at run time. The
// graph is built and instantiated once and replayed as one launch.
#include <algorithm>
#include <map>
#include <vector>

#include "engine.cuh"
#include "jobs.h"
#include "plan.h"

struct sg_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  uint32_t jobs = 0;
  uint64_t edges = 0;
};

extern "C" int sg_graph_build(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                              const uint64_t* tables_dev, const sg_record* plan, uint64_t* keep_dev,
                              sg_graph** out) {
  using namespace sg;
  if (!out || !dev_pool || (!jobs && n) || (!plan && n)) return SG_ERR_INVALID;
  *out = nullptr;
  PlanDeps pd;
  if (!plan_deps(jobs, n, plan, pool_bytes, &pd)) return SG_ERR_INVALID;
  int rc = gemm_prepare();
  if (rc != SG_OK) return rc;
  sg_graph* g = new sg_graph();
  cudaStream_t cap = nullptr;
  std::vector<cudaGraphNode_t> tail(n, nullptr);   // each job's last node
  std::vector<cudaGraphNode_t> deps;
  RelHook none;
  memset(&none, 0, sizeof none);
  rc = SG_OK;
  do {
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
    // One capture for the whole batch: before each job the stream's capture
    // dependencies are set to the last nodes of the jobs it depends on, so
    // the job's kernels hang from exactly those (a root when there are
    // none), and its own kernels follow one another.
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
    for (uint32_t j : pd.order) {
      const uint64_t off = plan[j].offset;
      deps.clear();
      for (uint64_t e = pd.pred_ptr[j]; e < pd.pred_ptr[j + 1]; e++) deps.push_back(tail[pd.pred[e]]);
      if (cudaStreamUpdateCaptureDependencies(cap, deps.data(), nullptr, deps.size(),
                                              cudaStreamSetCaptureDependencies) != cudaSuccess) {
        rc = SG_ERR_CUDA;
        break;
      }
      uint64_t nl = 0;
      int lrc = launch_job(jobs[j], (char*)dev_pool + off, tables_dev, none, keep_dev ? keep_dev + j : nullptr,
                           nullptr, cap, &nl);
      if (lrc != SG_OK) { rc = lrc; break; }
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* d = nullptr;
      size_t nd = 0;
      if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess ||
          cs != cudaStreamCaptureStatusActive || nd != 1) {
        rc = SG_ERR_CUDA;
        break;
      }
      tail[j] = d[0];
      g->kernels += nl;
      g->edges += deps.size();
      g->jobs++;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);   // ends the capture on every path
    g->graph = graph;
    if (rc != SG_OK) break;
    if (ec != cudaSuccess || !graph) { rc = SG_ERR_CUDA; break; }
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
  } while (0);
  if (cap) cudaStreamDestroy(cap);
  if (rc != SG_OK) {
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return rc;
  }
  *out = g;
  return SG_OK;
}

extern "C" int sg_graph_launch(sg_graph* g, void* stream) {
  if (!g || !g->exec) return SG_ERR_INVALID;
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

extern "C" int sg_graph_info(const sg_graph* g, uint64_t* jobs, uint64_t* kernels, uint64_t* edges) {
  if (!g) return SG_ERR_INVALID;
  if (jobs) *jobs = g->jobs;
  if (kernels) *kernels = g->kernels;
  if (edges) *edges = g->edges;
  return SG_OK;
}

extern "C" int sg_graph_destroy(sg_graph* g) {
  if (!g) return SG_ERR_INVALID;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return SG_OK;
}
