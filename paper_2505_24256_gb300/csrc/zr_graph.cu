// zr_graph.cu -- Zippel steps captured into CUDA graphs (one graph per batch
// shape): the descriptor tables are staged once into the graph's own
// workspace and the kernel sequence is captured, so a re-run of the same
// shapes on the same buffers is a single graph launch with no host-side
// planning, staging or per-kernel launch cost.
#include <cuda_runtime.h>

#include <vector>

#include "zr_internal.h"

using namespace zr;

struct zr_step_graph {
  zr_ctx* ctx = nullptr;
  char* ws = nullptr;
  uint32_t* d_status = nullptr;
  uint32_t* h_status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;
};

static void graph_free(zr_step_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->ws) cudaFree(g->ws);
  if (g->d_status) cudaFree(g->d_status);
  if (g->h_status) cudaFreeHost(g->h_status);
  delete g;
}

extern "C" zr_status zr_step_graph_create(zr_ctx* ctx, int32_t nsteps, const zr_step_desc* steps, void* stream,
                                          zr_step_graph** out) {
  if (!ctx || !out) return ZR_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsteps < 1 || !steps) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_step_graph_create: empty list");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<BatchItem> items;
  for (int i = 0; i < nsteps; i++) {
    const zr_step_desc& d = steps[i];
    zr_status r = check_step_args(ctx, &d.skel, d.newvar, d.y, d.S, d.samples, d.probes, d.ldb, d.offset, d.out_exps,
                                  d.out_coef, d.out_cap);
    if (r) return r;
    if (!d.out_count || d.skel.T < 1)
      return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_step_graph_create: every step needs T >= 1 and a count pointer");
    items.push_back(step_item(&d.skel, d.newvar, d.y, d.S, d.samples, d.probes, d.ldb, d.offset, d.out_exps,
                              d.out_coef, d.out_cap, d.out_count));
  }
  zr_step_graph* g = new (std::nothrow) zr_step_graph();
  if (!g) return ZR_ERR_OOM;
  g->ctx = ctx;
  const size_t need = batch_ws_need(ctx, items.data(), (int)items.size());
  cudaError_t e = cudaMalloc(&g->ws, need > 0 ? need : 256);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_status, sizeof(uint32_t));
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_err(ctx, e, "zr_step_graph_create");
  }
  for (auto& it : items) it.status = g->d_status;
  zr_status r = batch_graph_capture(ctx, items.data(), (int)items.size(), g->d_status, g->ws, st, &g->graph,
                                    &g->launches);
  if (r) {
    graph_free(g);
    return r;
  }
  // the warm-up run inside the capture helper already ran the steps once:
  // report its status like any other run
  e = cudaMemcpy(g->h_status, g->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_err(ctx, e, "zr_step_graph_create: instantiate");
  }
  *out = g;
  return status_from_flags(ctx, *g->h_status);
}

extern "C" zr_status zr_step_graph_launch(zr_step_graph* g, void* stream) {
  if (!g) return ZR_ERR_INVALID_ARG;
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_err(g->ctx, e, "zr_step_graph_launch");
  note_launches(g->launches);
  return ZR_OK;
}

extern "C" zr_status zr_step_graph_status(zr_step_graph* g, void* stream) {
  if (!g) return ZR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(g->h_status, g->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(g->ctx, e, "zr_step_graph_status");
  return status_from_flags(g->ctx, *g->h_status);
}

extern "C" uint64_t zr_step_graph_kernels(const zr_step_graph* g) { return g ? g->launches : 0; }

extern "C" void zr_step_graph_destroy(zr_step_graph* g) { graph_free(g); }
