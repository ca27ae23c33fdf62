// zr_tune.cu -- autotuner for the solve's launch plan.
//
// For a shape (T, S) the candidates are every compiled right-hand-side tile
// crossed with a set of k-block counts; the cost model of plan_step ranks
// them, the best `budget` of them are run on synthetic data of that shape
// (random nodes and right-hand sides in the context workspace, one warm-up
// and one timed launch each, CUDA events on the call's stream), and the
// fastest is stored in the context's plan table, which plan_step consults
// before its model.  The tuned plan changes the schedule only: every plan
// computes the same values.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "zr_internal.h"

namespace zr {

__global__ void k_synth(int64_t n, uint64_t seed, Mod M, uint64_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  z >>= 1;
  out[i] = z >= M.p ? z - M.p : z;
}

}  // namespace zr

using namespace zr;

extern "C" zr_status zr_autotune_step(zr_ctx* ctx, int64_t T, int32_t S, int32_t budget, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (T < 1 || S < 1 || S > 64 || budget < 1) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_autotune_step: bad shape");
  cudaStream_t st = (cudaStream_t)stream;
  // candidates, ranked by the model
  std::vector<std::pair<double, StepDims>> cand;
  int tiles[16];
  const int nt = solve_tiles(tiles, 16);
  const int nbs[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32};
  for (int ti = 0; ti < nt; ti++) {
    const int groups = (S + tiles[ti] - 1) / tiles[ti];
    if (groups > solve_max_groups() || !solve_instance_exists(tiles[ti], groups)) continue;
    for (int nb : nbs) {
      if (nb > 1 && T / nb < 64) continue;
      StepDims D;
      D.T = T;
      D.S = S;
      D.s_tile = tiles[ti];
      int64_t BK = (T + nb - 1) / nb;
      BK = ((BK + 31) / 32) * 32;
      D.BK = BK < 32 ? 32 : BK;
      D.NB = (int)((T + D.BK - 1) / D.BK);
      cand.push_back({plan_cost(ctx, D), D});
    }
  }
  std::sort(cand.begin(), cand.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  if ((int)cand.size() > budget) cand.resize(budget);
  // synthetic system of this shape in its own buffers (nodes, right-hand sides, output)
  uint64_t *v = nullptr, *b = nullptr, *cc = nullptr;
  cudaError_t e = cudaMalloc(&v, 8 * (size_t)T);
  if (e == cudaSuccess) e = cudaMalloc(&b, 8 * (size_t)S * T);
  if (e == cudaSuccess) e = cudaMalloc(&cc, 8 * (size_t)S * T);
  if (e != cudaSuccess) {
    cudaFree(v);
    cudaFree(b);
    cudaFree(cc);
    return cuda_err(ctx, e, "zr_autotune_step: buffers");
  }
  const unsigned g1 = (unsigned)((T + 255) / 256), g2 = (unsigned)((S * T + 255) / 256);
  { k_synth<<<g1, 256, 0, st>>>(T, 11, ctx->M, v); note_launch(); }
  { k_synth<<<g2, 256, 0, st>>>((int64_t)S * T, 14, ctx->M, b); note_launch(); }
  BatchItem it;
  it.mode = 1;
  it.T = T;
  it.S = S;
  it.vin = v;
  it.b = b;
  it.ldb = T;
  it.c = cc;
  it.ldc = T;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time each candidate through the batch runner with that plan forced
  std::vector<zr_plan_entry> saved;
  for (const auto& pe : ctx->plans)
    if (!(pe.T == T && pe.S == S)) saved.push_back(pe);
  double best_ms = -1;
  StepDims best = cand.empty() ? plan_step(ctx, T, S) : cand[0].second;
  zr_status r = ZR_OK;
  // the plan is the O(T^2) solve's: time that method whatever the context's choice
  const int method = ctx->solve_method;
  ctx->solve_method = 1;
  for (auto& c : cand) {
    ctx->plans = saved;
    ctx->plans.push_back({T, S, c.second});
    float ms = 0;
    for (int rep = 0; rep < 2 && r == ZR_OK; rep++) {
      cudaEventRecord(e0, st);
      r = run_batch(ctx, &it, 1, ctx->d_status_call, st);
      cudaEventRecord(e1, st);
    }
    if (r) break;
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      r = cuda_err(ctx, e, "zr_autotune_step");
      break;
    }
    if (best_ms < 0 || ms < best_ms) {
      best_ms = ms;
      best = c.second;
    }
  }
  ctx->plans = saved;
  ctx->solve_method = method;
  cudaStreamSynchronize(st);
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);   // synthetic nodes may collide: not an error here
  cudaFree(v);
  cudaFree(b);
  cudaFree(cc);
  if (r) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& e : ctx->plans)
    if (e.T == T && e.S == S) {
      e.D = best;
      return ZR_OK;
    }
  ctx->plans.push_back({T, S, best});
  return ZR_OK;
}

extern "C" zr_status zr_step_plan(zr_ctx* ctx, int64_t T, int32_t S, int32_t* s_tile, int32_t* nblocks) {
  if (!ctx || T < 0 || S < 1) return ZR_ERR_INVALID_ARG;
  StepDims D = plan_step(ctx, T, S);
  if (s_tile) *s_tile = D.s_tile;
  if (nblocks) *nblocks = D.NB;
  return ZR_OK;
}
