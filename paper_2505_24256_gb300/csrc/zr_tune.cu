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
    const int nst = (S + tiles[ti] - 1) / tiles[ti];
    if (nst > 8) continue;
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
  // workspace: the largest candidate's step layout plus synthetic inputs
  size_t need = 0;
  for (auto& c : cand) {
    Carver m0(nullptr);
    carve_step(m0, T, S, 0, c.second);
    m0.take<uint64_t>((size_t)S * T);
    need = std::max(need, m0.off);
  }
  zr_status r = ensure_ws(ctx, need, st);
  if (r) return r;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_err(ctx, ZR_ERR_CUDA, "zr_autotune_step: events");
  double best_ms = -1;
  StepDims best = cand.empty() ? plan_step(ctx, T, S) : cand[0].second;
  for (auto& c : cand) {
    const StepDims& D = c.second;
    Carver cv(ctx->ws);
    StepWs w = carve_step(cv, T, S, 0, D);
    uint64_t* b = cv.take<uint64_t>((size_t)S * T);
    const unsigned g1 = (unsigned)((T + 255) / 256), g2 = (unsigned)((S * T + 255) / 256);
    { k_synth<<<g1, 256, 0, st>>>(T, 11, ctx->M, w.v); note_launch(); }
    { k_synth<<<g1, 256, 0, st>>>(T, 12, ctx->M, w.m); note_launch(); }
    { k_synth<<<g1, 256, 0, st>>>(T, 13, ctx->M, w.vp); note_launch(); }
    { k_synth<<<g2, 256, 0, st>>>((int64_t)S * T, 14, ctx->M, b); note_launch(); }
    float ms = 0;
    for (int rep = 0; rep < 2; rep++) {
      cudaEventRecord(e0, st);
      launch_carry_partials(D, w.m, w.v, w.vp, ctx->M, w.R, st);
      launch_solve(D, w.m, w.v, w.vp, w.R, b, T, ctx->M, w.part, w.denp, st);
      cudaEventRecord(e1, st);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_err(ctx, e, "zr_autotune_step");
    }
    if (best_ms < 0 || ms < best_ms) {
      best_ms = ms;
      best = D;
    }
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
