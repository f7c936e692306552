// Batching through one captured CUDA graph: a static co-schedule.
//
// The device replay (sg_replay) decides, on the logical clock with declared
// durations, where each job lives in the pool and in what order jobs are
// granted. This file turns that plan into one CUDA graph: every job is a
// child graph (its generator kernels, then its kernel, then optionally its
// output digest), and a job depends on every job that used any byte of its
// extent before it in grant order. Jobs that share no memory run
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
  std::vector<cudaGraphNode_t> node(n, nullptr);
  std::vector<cudaGraphNode_t> deps;
  RelHook none;
  memset(&none, 0, sizeof none);
  rc = SG_OK;
  do {
    if (cudaGraphCreate(&g->graph, 0) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
    for (uint32_t j : pd.order) {
      const uint64_t off = plan[j].offset;
      deps.clear();
      for (uint64_t e = pd.pred_ptr[j]; e < pd.pred_ptr[j + 1]; e++) deps.push_back(node[pd.pred[e]]);
      cudaGraph_t child = nullptr;
      if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SG_ERR_CUDA; break; }
      uint64_t nl = 0;
      int lrc = launch_job(jobs[j], (char*)dev_pool + off, tables_dev, none, keep_dev ? keep_dev + j : nullptr,
                           nullptr, cap, &nl);
      cudaError_t ec = cudaStreamEndCapture(cap, &child);
      if (lrc != SG_OK || ec != cudaSuccess) {
        if (child) cudaGraphDestroy(child);
        rc = lrc != SG_OK ? lrc : SG_ERR_CUDA;
        break;
      }
      cudaError_t ea = cudaGraphAddChildGraphNode(&node[j], g->graph, deps.data(), deps.size(), child);
      cudaGraphDestroy(child);
      if (ea != cudaSuccess) { rc = SG_ERR_CUDA; break; }
      g->kernels += nl;
      g->edges += deps.size();
      g->jobs++;
    }
    if (rc != SG_OK) break;
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
