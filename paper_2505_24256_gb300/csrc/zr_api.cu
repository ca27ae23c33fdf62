// zr_api.cu -- context, workspace and the C entry points of the Zippel step.
#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "zr_internal.h"

using namespace zr;

// ---------------------------------------------------------------------------
// host arithmetic used to set up the modulus descriptor
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

static uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }
static uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = h_mulmod(r, a, p);
    a = h_mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}
// deterministic Miller-Rabin (bases 2..37 decide every n < 2^64)
static bool h_is_prime(uint64_t n) {
  static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t b : bases) {
    if (n == b) return true;
    if (n % b == 0) return false;
  }
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) { d >>= 1; r++; }
  for (uint64_t b : bases) {
    uint64_t x = h_powmod(b, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r && comp; i++) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}

static Mod make_mod(uint64_t p) {
  Mod M;
  memset(&M, 0, sizeof(M));
  M.p = p;
  M.norm = (uint32_t)__builtin_clzll(p);
  M.d = p << M.norm;
  M.v = (uint64_t)((~(u128)0) / M.d - ((u128)1 << 64));
  return M;
}

// ---------------------------------------------------------------------------
// errors and workspace
// ---------------------------------------------------------------------------
namespace zr {

bool mod_for_prime(uint64_t p, Mod* out) {
  if (!out || p <= (1ull << 32) || p >= (1ull << 63) || !h_is_prime(p)) return false;
  *out = make_mod(p);
  return true;
}

zr_status set_err(zr_ctx* ctx, zr_status st, const std::string& msg) {
  if (ctx && st != ZR_OK) {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->err = msg;
  }
  return st;
}

cudaEvent_t prof_mark(zr_ctx* ctx, cudaStream_t st) {
  if (!ctx->prof.on) return nullptr;
  cudaEvent_t e = nullptr;
  if (!ctx->prof.pool.empty()) {
    e = ctx->prof.pool.back();
    ctx->prof.pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(e, st);
  return e;
}

void prof_add(zr_ctx* ctx, int phase, cudaEvent_t a, cudaEvent_t b, double work) {
  if (!a || !b) return;
  ctx->prof.pending.push_back({phase, a, b, work});
}

void prof_collect(zr_ctx* ctx) {
  // adjacent phases share their boundary event: return every event once
  std::vector<cudaEvent_t> used;
  for (auto& p : ctx->prof.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->prof.total_ms[p.phase] += ms;
      ctx->prof.count[p.phase] += 1;
      ctx->prof.work[p.phase] += p.work;
    }
    used.push_back(p.a);
    used.push_back(p.b);
  }
  std::sort(used.begin(), used.end());
  used.erase(std::unique(used.begin(), used.end()), used.end());
  for (cudaEvent_t e : used) ctx->prof.pool.push_back(e);
  ctx->prof.pending.clear();
}

zr_status cuda_err(zr_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return ZR_OK;
  return set_err(ctx, e == cudaErrorMemoryAllocation ? ZR_ERR_OOM : ZR_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

zr_status ensure_ws(zr_ctx* ctx, size_t need, cudaStream_t st) {
  if (need <= ctx->ws_cap) return ZR_OK;
  if (ctx->ws) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "workspace sync");
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
  }
  size_t cap = need + need / 4 + (1 << 20);
  cudaError_t e = cudaMalloc(&ctx->ws, cap);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    return cuda_err(ctx, e, "workspace allocation");
  }
  ctx->ws_cap = cap;
  return ZR_OK;
}

zr_status status_from_flags(zr_ctx* ctx, uint32_t f) {
  if (!f) return ZR_OK;
  if (f & ST_TIMEOUT) return set_err(ctx, ZR_ERR_TIMEOUT, "a bounded device wait gave up");
  if (f & (ST_DUP_NODE | ST_ZERO_NODE | ST_ZERO_DEN | ST_DUP_SAMPLE | ST_HASH_FULL))
    return set_err(ctx, ZR_ERR_SINGULAR,
                   (f & ST_DUP_SAMPLE) ? "two samples of the new variable coincide"
                                       : "anchor values not pairwise distinct (or zero with offset 1)");
  if (f & ST_POLE) return set_err(ctx, ZR_ERR_POLE, "the black box has a pole at a probe");
  if (f & ST_DEGREE) return set_err(ctx, ZR_ERR_DEGREE, "univariate reconstruction exceeds its degree bound");
  if (f & ST_THIELE) return set_err(ctx, ZR_ERR_UNLUCKY, "degenerate Thiele table");
  return set_err(ctx, ZR_ERR_CUDA, "unknown device status");
}

uint64_t hash_slots(int64_t T) {
  uint64_t h = 64;
  while (h < (uint64_t)(2 * T)) h <<= 1;
  return h;
}

// Launch plan of the solve: the right-hand sides per consumer thread (CG,
// "tile"; G = ceil(S / CG) consumer groups of 64 threads plus one producer
// warp per CTA) and the number of k-blocks NB.  For every compiled tile the
// resident CTAs per SM (occupancy query, cached) give the slots of one wave.
// Model, in 32-bit multiply issue slots per root and k:
//   cost_k = 8 G CG + 32   (four lo + four hi per MAC over the padded
//                           columns; two Shoup chain steps)
// and a wave with n CTAs on an SM takes BK cost_k n / min(1, w / 16), w the
// resident warps: fewer than 16 warps leave the multiplier partly idle.  The
// carry pass adds a Shoup Horner step per k.  The cheapest plan wins;
// measured plans from zr_autotune_step take precedence.
static int occupancy_cached(int tile, int groups) {
  static DeviceValue cache[16][9];   // per device: the occupancy query sets per-device attributes
  if (tile <= 0 || tile >= 16 || groups < 1 || groups > 8) return 1;
  return cache[tile][groups].get([&] { return solve_blocks_per_sm(tile, groups); });
}

// A forced plan: the context's tuned plan table, else ZR_SOLVE_PLAN="tile,NB"
// in the environment (a tuning override), else the model below.
static bool forced_plan(const zr_ctx* ctx, int64_t T, int S, StepDims& D) {
  if (ctx) {
    for (const auto& e : ctx->plans)
      if (e.T == T && e.S == S) {
        D = e.D;
        return true;
      }
  }
  const char* env = getenv("ZR_SOLVE_PLAN");
  int tile = 0, nb = 0;
  if (!env || sscanf(env, "%d,%d", &tile, &nb) != 2 || tile <= 0 || nb <= 0) return false;
  int tiles[16];
  const int nt = solve_tiles(tiles, 16);
  bool ok = false;
  for (int i = 0; i < nt; i++) ok |= tiles[i] == tile;
  if (!ok) return false;
  D.T = T;
  D.S = S;
  D.s_tile = tile;
  int64_t BK = (T + nb - 1) / nb;
  BK = ((BK + 31) / 32) * 32;
  D.BK = BK < 32 ? 32 : BK;
  D.NB = (int)((T + D.BK - 1) / D.BK);
  if (D.NB < 1) D.NB = 1;
  return true;
}

double plan_cost(const zr_ctx* ctx, const StepDims& D) {
  const int64_t sms = ctx && ctx->sms ? ctx->sms : 152;
  const int rt = solve_roots_per_item();
  const int64_t rows = (D.T + rt - 1) / rt;
  const int G = (D.S + D.s_tile - 1) / D.s_tile;
  if (G > solve_max_groups() || !solve_instance_exists(D.s_tile, G)) return 1e300;
  const int per_sm = occupancy_cached(D.s_tile, G);
  const int64_t slots = sms * per_sm;
  const double cost_k = 8.0 * G * D.s_tile + 32.0;
  const int64_t items = rows * D.NB;
  double cost = 0;
  for (int64_t left = items; left > 0; left -= slots) {
    const int64_t in_wave = left < slots ? left : slots;
    const int64_t n = (in_wave + sms - 1) / sms;
    const double warps = (double)n * (1 + 2 * G);
    const double eff = warps >= 16 ? 1.0 : warps / 16.0;
    cost += (double)D.BK * rt * cost_k * (double)n / eff;
  }
  // Terms calibrated on GB300 against a sweep of k-block counts (T = 10^4,
  // S = 21; about 8.7e7 units per millisecond):
  //  * each work item's prologue (the carry-in from the blocks above), ~15 ns;
  cost += 1300.0 * (double)items;
  //  * the finish reads NB partials per right-hand side and root;
  cost += (double)D.NB * D.S * D.T;
  //  * the carry kernel: (NB - 1) BK T chain steps at ~0.8 of the chain
  //    rate, but never faster than one root's serial chain of BK steps
  //    (~80 ns a step when few CTAs run).
  if (D.NB > 1) {
    const double through = 20.5 * (double)(D.NB - 1) * D.BK * D.T / (double)sms;
    const double serial = 6960.0 * (double)D.BK;
    cost += through > serial ? through : serial;
  }
  return cost;
}

StepDims plan_step(const zr_ctx* ctx, int64_t T, int S) {
  StepDims best;
  if (forced_plan(ctx, T, S, best)) return best;
  best.T = T;
  best.S = S;
  best.NB = 1;
  best.BK = ((T + 31) / 32) * 32;
  best.s_tile = 16;
  double best_cost = -1;
  int tiles[16];
  const int nt = solve_tiles(tiles, 16);
  for (int ti = 0; ti < nt; ti++) {
    const int tile = tiles[ti];
    const int groups = (S + tile - 1) / tile;
    if (groups > solve_max_groups() || !solve_instance_exists(tile, groups)) continue;
    for (int NBw = 1; NBw <= 64; NBw++) {
      int64_t BK = (T + NBw - 1) / NBw;
      BK = ((BK + 31) / 32) * 32;
      if (BK < 32) BK = 32;
      const int NB = (int)((T + BK - 1) / BK);
      if (NB != NBw) continue;
      StepDims D;
      D.T = T;
      D.S = S;
      D.NB = NB;
      D.BK = BK;
      D.s_tile = tile;
      const double cost = plan_cost(ctx, D);
      if (best_cost < 0 || cost < best_cost * 0.999) {
        best_cost = cost;
        best = D;
      }
    }
  }
  return best;
}

StepWs carve_step(Carver& cv, int64_t T, int S, int k, const StepDims& D, int Ssolve) {
  if (Ssolve < 0) Ssolve = S;
  StepWs w;
  const int64_t Tn = T > 0 ? T : 1;
  w.tab = cv.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
  w.v = cv.take<uint64_t>(Tn);
  w.vp = cv.take<uint64_t>(Tn);
  w.htab = cv.take<uint64_t>(hash_slots(T));
  w.m = cv.take<uint64_t>(Tn);
  w.tmp = cv.take<uint64_t>(2 * Tn);
  w.tpart = cv.take<uint64_t>((size_t)tree_split_max(Tn) * Tn);
  w.R = cv.take<uint64_t>((size_t)(D.NB > 1 ? D.NB - 1 : 1) * Tn);
  w.part = cv.take<uint64_t>((size_t)D.NB * Ssolve * Tn);
  w.denp = cv.take<uint64_t>((size_t)D.NB * Tn);
  w.invd = cv.take<uint64_t>((size_t)S * S);
  w.g = cv.take<uint64_t>((size_t)S * Tn);
  w.cnt = cv.take<int32_t>(Tn);
  w.bsum = cv.take<int64_t>((size_t)scan_blocks(Tn) + 1);
  return w;
}

}  // namespace zr

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------

static std::atomic<unsigned long long> g_launches{0};
namespace zr {
int current_device() {
  int d = 0;
  return cudaGetDevice(&d) == cudaSuccess ? d : 0;
}
unsigned long long launch_count() { return g_launches.load(); }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace zr

extern "C" uint64_t zr_launch_count(void) { return (uint64_t)zr::launch_count(); }

extern "C" zr_status zr_profile_enable(zr_ctx* ctx, int32_t on) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  prof_collect(ctx);
  ctx->prof.on = on != 0;
  for (int i = 0; i < PH_N; i++) {
    ctx->prof.total_ms[i] = 0;
    ctx->prof.count[i] = 0;
    ctx->prof.work[i] = 0;
  }
  return ZR_OK;
}

extern "C" zr_status zr_profile_query(zr_ctx* ctx, int32_t phase, double* total_ms, int64_t* count) {
  if (!ctx || phase < 0 || phase >= PH_N) return ZR_ERR_INVALID_ARG;
  prof_collect(ctx);
  if (total_ms) *total_ms = ctx->prof.total_ms[phase];
  if (count) *count = ctx->prof.count[phase];
  return ZR_OK;
}

extern "C" zr_status zr_profile_work(zr_ctx* ctx, int32_t phase, double* units) {
  if (!ctx || !units || phase < 0 || phase >= PH_N) return ZR_ERR_INVALID_ARG;
  prof_collect(ctx);
  *units = ctx->prof.work[phase];
  return ZR_OK;
}

static const char* kStatusNames[] = {"ok", "invalid argument", "singular", "pole", "out of memory", "timeout",
                                     "cuda error", "unlucky random choice", "busy", "capacity", "degree bound"};

extern "C" const char* zr_status_string(zr_status s) {
  if ((int)s < 0 || (int)s > 10) return "unknown status";
  return kStatusNames[(int)s];
}

extern "C" zr_status zr_create(uint64_t prime, zr_ctx** out) {
  if (!out) return ZR_ERR_INVALID_ARG;
  *out = nullptr;
  if (prime <= (1ull << 32) || prime >= (1ull << 63) || !h_is_prime(prime)) return ZR_ERR_INVALID_ARG;
  zr_ctx* ctx = new (std::nothrow) zr_ctx();
  if (!ctx) return ZR_ERR_OOM;
  ctx->M = make_mod(prime);
  ctx->ntt = make_ntt_consts(prime);
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_count, 4 * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_count, 4 * sizeof(int64_t));
  if (e == cudaSuccess) {
    // reconstructions allocate their per-request buffers from the device's
    // pool in stream order; keep freed blocks in the pool for the next ones
    // (a property of this process's pool, not a setting of the device)
    cudaMemPool_t pool;
    uint64_t keep = ~0ull;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess)
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
  }
  if (e != cudaSuccess) {
    zr_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? ZR_ERR_OOM : ZR_ERR_CUDA;
  }
  ctx->d_status_call = ctx->d_status + 1;
  *out = ctx;
  return ZR_OK;
}

extern "C" void zr_destroy(zr_ctx* ctx) {
  if (!ctx) return;
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->d_count) cudaFree(ctx->d_count);
  if (ctx->h_count) cudaFreeHost(ctx->h_count);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->stage_event) cudaEventDestroy(ctx->stage_event);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (int j = 0; j < 4; j++) {
    if (ctx->fstream[j]) cudaStreamDestroy(ctx->fstream[j]);
    if (ctx->fev_join[j]) cudaEventDestroy(ctx->fev_join[j]);
  }
  if (ctx->fev_fork) cudaEventDestroy(ctx->fev_fork);
  for (int j = 0; j < 5; j++) {
    if (ctx->faux[j]) cudaStreamDestroy(ctx->faux[j]);
    if (ctx->faux_fork[j]) cudaEventDestroy(ctx->faux_fork[j]);
    if (ctx->faux_join[j]) cudaEventDestroy(ctx->faux_join[j]);
  }
  if (ctx->ntt_tw) cudaFree(ctx->ntt_tw);
  if (ctx->fprobe_ws) cudaFree(ctx->fprobe_ws);
  for (int j = 0; j < zr_ctx::kProbeLanes; j++) {
    if (ctx->pl_ws[j]) cudaFree(ctx->pl_ws[j]);
    if (ctx->pl_fws[j]) cudaFree(ctx->pl_fws[j]);
  }
  delete ctx;
}

extern "C" const char* zr_last_error(const zr_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

// The automatic choice of solve method.  On GB300, for one system alone,
// the O(T log^2 T) path is faster than the O(T^2) batch from T = 768 at every
// S measured (1, 5, 21: 0.18 - 0.19 against 0.22 - 0.24 ms at T = 768, 0.49
// against 1.02 ms at T = 6144, S = 21); it is taken from T = 1024.  In a
// batch of several systems the O(T^2) ones share their launches while each
// fast system runs its own chain of about 45 kernels: there it is taken when
// T^2 (S + 5) >= 8e7 (about T >= 1750 at S = 21, 3600 at S = 1), the rule
// under which the serving mix measured best (1.53 - 1.57x the plain form,
// against 1.46x with the single-system rule).
static constexpr int64_t kFastFloorT = 1024;
static constexpr double kFastBatchCross = 8e7;

namespace zr {
bool use_fast_solve(const zr_ctx* ctx, int64_t T, int S, int batch_n) {
  if (T < 1 || T > kFastMaxT || ctx->solve_method == 1) return false;
  if (ctx->solve_method == 2) return true;
  if (ctx->fast_min_T > 0) return T >= ctx->fast_min_T;
  if (T < kFastFloorT) return false;
  return batch_n <= 1 || (double)T * (double)T * (double)(S + 5) >= kFastBatchCross;
}
}  // namespace zr

// The automatic choice of evaluator for T probes per sample of a function
// of Tf terms and S samples.  Measured on GB300 (Tf = T): the matrix-vector
// evaluator costs about S T Tf 5e-10 ms + 0.15 ms, the transposed tree 0.36
// to 1.3 ms from T = 2048 to 16384; they cross near T = 7800 (S = 21),
// 12500 (S = 5) and 14000 (S = 1), which T Tf (S + 8) >= 1.8e9 follows.
static constexpr double kFastProbeCross = 1.8e9;
static constexpr int64_t kFastProbeFloorT = 4096;

namespace zr {
bool use_fast_probes(const zr_ctx* ctx, int64_t T, int64_t Tf, int S) {
  if (T < 1 || Tf < 1 || T > kFastMaxT || S > kFastProbeMaxS || ctx->solve_method == 1) return false;
  if (ctx->solve_method == 2) return true;
  if (ctx->fast_min_T > 0) return T >= ctx->fast_min_T && Tf >= ctx->fast_min_T;
  return T >= kFastProbeFloorT && Tf >= kFastProbeFloorT && (double)T * (double)Tf * (double)(S + 8) >= kFastProbeCross;
}
}  // namespace zr

// Scheduling weights in multiply-accumulate equivalents (about 2e12 per
// second on GB300).  The O(T^2) solve does S T^2 + 2.5 T^2; the fast one was
// measured at 25 ms for T = 2^20, S = 9 and about 0.5 ms at small T, which
// 8 (S + 6) T log2(T)^2 + 1e9 follows.  The matrix-vector evaluator does
// S T Tf; the transposed tree is weighted like the fast solve on max(T, Tf).
namespace zr {
static double fast_work(double n, int S) {
  const double l = std::log2(std::max(n, 2.0));
  return 8.0 * (S + 6) * n * l * l + 1e9;
}
double solve_work(const zr_ctx* ctx, int64_t T, int S) {
  if (T <= 0) return 0;
  return use_fast_solve(ctx, T, S, 2) ? fast_work((double)T, S) : (S + 2.5) * (double)T * (double)T;
}
double probe_work(const zr_ctx* ctx, int64_t T, int S, int64_t Tf) {
  if (T <= 0 || Tf <= 0) return 0;
  return use_fast_probes(ctx, T, Tf, S) ? fast_work((double)std::max(T, Tf), S)
                                        : (double)S * (double)T * (double)Tf;
}
}  // namespace zr

extern "C" zr_status zr_solve_method(zr_ctx* ctx, int32_t method, int64_t crossover) {
  if (!ctx || method < 0 || method > 2 || crossover < 0) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_solve_method");
  ctx->solve_method = method;
  ctx->fast_min_T = crossover;
  return ZR_OK;
}
extern "C" uint64_t zr_prime(const zr_ctx* ctx) { return ctx ? ctx->M.p : 0; }
extern "C" size_t zr_workspace_bytes(const zr_ctx* ctx) { return ctx ? ctx->ws_cap : 0; }

// Reads and clears the per-call status word after the stream drains.
static zr_status finish_sync_call(zr_ctx* ctx, cudaStream_t st, int64_t* count_out) {
  cudaError_t e = cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && count_out)
    e = cudaMemcpyAsync(ctx->h_count, ctx->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "synchronise");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "kernel launch");
  if (count_out) *count_out = ctx->h_count[0];
  return status_from_flags(ctx, ctx->h_status[1]);
}

static zr_status check_vsys(zr_ctx* ctx, const zr_vsys& s) {
  if (s.T < 0 || s.S < 1 || s.S > 256 || (s.offset != 0 && s.offset != 1) || s.ldb < s.T || s.ldc < s.T)
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_vsys: sizes out of range");
  if (s.T > 0 && (!s.v || !s.b || !s.c)) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_vsys: null pointer");
  return ZR_OK;
}

static BatchItem vsys_item(const zr_vsys& s) {
  BatchItem it;
  it.mode = 1;
  it.T = s.T;
  it.S = s.S;
  it.offset = s.offset;
  it.vin = s.v;
  it.b = s.b;
  it.ldb = s.ldb;
  it.c = s.c;
  it.ldc = s.ldc;
  return it;
}

extern "C" zr_status zr_vandermonde_solve_plain(zr_ctx* ctx, int32_t nsys, const zr_vsys* sys, void* stream) {
  if (!ctx || nsys < 0 || (nsys > 0 && !sys)) return set_err(ctx, ZR_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < nsys; i++) {
    zr_status r = check_vsys(ctx, sys[i]);
    if (r) return r;
  }
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  for (int i = 0; i < nsys; i++) {
    if (sys[i].T == 0) continue;
    const BatchItem it = vsys_item(sys[i]);
    zr_status r = run_batch(ctx, &it, 1, ctx->d_status_call, st);
    if (r) return r;
  }
  return finish_sync_call(ctx, st, nullptr);
}

extern "C" zr_status zr_vandermonde_solve_batched(zr_ctx* ctx, int32_t nsys, const zr_vsys* sys, void* stream) {
  if (!ctx || nsys < 0 || (nsys > 0 && !sys)) return set_err(ctx, ZR_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<BatchItem> items;
  for (int i = 0; i < nsys; i++) {
    zr_status r = check_vsys(ctx, sys[i]);
    if (r) return r;
    if (sys[i].T > 0) items.push_back(vsys_item(sys[i]));
  }
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  zr_status r = run_batch(ctx, items.data(), (int)items.size(), ctx->d_status_call, st);
  if (r) return r;
  return finish_sync_call(ctx, st, nullptr);
}

extern "C" zr_status zr_newton_batched(zr_ctx* ctx, int64_t nterms, int32_t npts, const uint64_t* x,
                                       const uint64_t* vals, int64_t ld, uint64_t* coef, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (nterms < 0 || npts < 1 || npts > 64 || ld < nterms || (nterms > 0 && (!x || !vals || !coef)))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_newton_batched: sizes out of range (1 <= npts <= 64)");
  cudaStream_t st = (cudaStream_t)stream;
  Carver m0(nullptr);
  m0.take<uint64_t>((size_t)npts * npts);
  zr_status r = ensure_ws(ctx, m0.off, st);
  if (r) return r;
  Carver cv(ctx->ws);
  uint64_t* invd = cv.take<uint64_t>((size_t)npts * npts);
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  launch_newton_table(npts, x, ctx->M, invd, ctx->d_status_call, st);
  launch_newton(nterms, npts, invd, vals, ld, ctx->M, coef, st);
  return finish_sync_call(ctx, st, nullptr);
}

extern "C" zr_status zr_anchor_values(zr_ctx* ctx, int64_t T, int32_t nv, const uint8_t* exps, int32_t k,
                                      const uint64_t* y, int32_t offset, uint64_t* v, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (T < 0 || nv < 1 || nv > kMaxVars || k < 0 || k > nv || (offset != 0 && offset != 1) ||
      (T > 0 && (!exps || !v || (k > 0 && !y))))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_anchor_values: arguments out of range");
  cudaStream_t st = (cudaStream_t)stream;
  Carver m0(nullptr);
  m0.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
  m0.take<uint64_t>(T > 0 ? T : 1);
  m0.take<uint64_t>(hash_slots(T));
  zr_status r = ensure_ws(ctx, m0.off, st);
  if (r) return r;
  Carver cv(ctx->ws);
  uint64_t* tab = cv.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
  uint64_t* vp = cv.take<uint64_t>(T > 0 ? T : 1);
  uint64_t* htab = cv.take<uint64_t>(hash_slots(T));
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  cudaMemsetAsync(htab, 0xFF, hash_slots(T) * sizeof(uint64_t), st);
  launch_powtab(y, k, ctx->M, tab, st);
  launch_anchor(T, nv, exps, k, tab, offset, ctx->M, v, vp, htab, hash_slots(T) - 1, ctx->d_status_call, st);
  return finish_sync_call(ctx, st, nullptr);
}

namespace zr {
zr_status check_step_args(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                          const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                          uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap) {
  if (!skel) return set_err(ctx, ZR_ERR_INVALID_ARG, "null skeleton");
  if (skel->nv < 1 || skel->nv > kMaxVars || newvar < 0 || newvar >= skel->nv)
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step: need 0 <= newvar < nv <= 64");
  if (skel->T < 0 || skel->T >= (1ll << 31) || S < 1 || S > 64 || ldb < skel->T || out_cap < 0 ||
      (offset != 0 && offset != 1))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step: need 0 <= T < 2^31, 1 <= S <= 64, ldb >= T");
  if (!samples || (skel->T > 0 && (!skel->exps || !probes || (newvar > 0 && !y))) ||
      (out_cap > 0 && (!out_exps || !out_coef)))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step: null pointer");
  return ZR_OK;
}

BatchItem step_item(const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S, const uint64_t* samples,
                    const uint64_t* probes, int64_t ldb, int32_t offset, uint8_t* out_exps, uint64_t* out_coef,
                    int64_t out_cap, int64_t* d_count) {
  BatchItem it;
  it.mode = 0;
  it.T = skel->T;
  it.S = S;
  it.k = newvar;
  it.nv = skel->nv;
  it.offset = offset;
  it.exps = skel->exps;
  it.y = y;
  it.xs = samples;
  it.b = probes;
  it.ldb = ldb;
  it.out_exps = out_exps;
  it.out_coef = out_coef;
  it.out_cap = out_cap;
  it.out_count = d_count;
  return it;
}
}  // namespace zr

// A step with T = 0 still validates its samples (equal samples are an error).
static void empty_step(zr_ctx* ctx, int S, const uint64_t* samples, int64_t* d_count, uint32_t* status,
                       cudaStream_t st) {
  Carver cv(ctx->ws);
  uint64_t* invd = cv.take<uint64_t>((size_t)S * S);
  cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
  launch_newton_table(S, samples, ctx->M, invd, status, st);
}

extern "C" zr_status zr_zippel_step_async(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y,
                                          int32_t S, const uint64_t* samples, const uint64_t* probes, int64_t ldb,
                                          int32_t offset, uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap,
                                          int64_t* d_out_count, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  zr_status r = check_step_args(ctx, skel, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef, out_cap);
  if (r) return r;
  if (!d_out_count) return set_err(ctx, ZR_ERR_INVALID_ARG, "null count pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (skel->T == 0) {
    if ((r = ensure_ws(ctx, 8 * (size_t)S * S + 256, st))) return r;
    empty_step(ctx, S, samples, d_out_count, ctx->d_status, st);
    return cuda_err(ctx, cudaGetLastError(), "zr_zippel_step_async");
  }
  const BatchItem it = step_item(skel, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef, out_cap,
                                 d_out_count);
  return run_batch(ctx, &it, 1, ctx->d_status, st);
}

extern "C" zr_status zr_stream_status(zr_ctx* ctx, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_stream_status");
  return status_from_flags(ctx, ctx->h_status[0]);
}

extern "C" zr_status zr_zippel_step(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                                    const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                                    uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap, int64_t* out_count,
                                    void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  zr_status r = check_step_args(ctx, skel, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef, out_cap);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  if (skel->T == 0) {
    if ((r = ensure_ws(ctx, 8 * (size_t)S * S + 256, st))) return r;
    empty_step(ctx, S, samples, ctx->d_count, ctx->d_status_call, st);
  } else {
    const BatchItem it = step_item(skel, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef, out_cap,
                                   ctx->d_count);
    if ((r = run_batch(ctx, &it, 1, ctx->d_status_call, st))) return r;
  }
  int64_t n = 0;
  r = finish_sync_call(ctx, st, &n);
  if (out_count) *out_count = n;
  if (r == ZR_OK && n > out_cap) return set_err(ctx, ZR_ERR_CAPACITY, "output skeleton larger than out_cap");
  return r;
}

extern "C" zr_status zr_zippel_step_batched(zr_ctx* ctx, int32_t nsteps, const zr_step_desc* steps, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (nsteps < 0 || (nsteps > 0 && !steps)) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step_batched: bad list");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<BatchItem> items;
  for (int i = 0; i < nsteps; i++) {
    const zr_step_desc& d = steps[i];
    zr_status r = check_step_args(ctx, &d.skel, d.newvar, d.y, d.S, d.samples, d.probes, d.ldb, d.offset, d.out_exps,
                                  d.out_coef, d.out_cap);
    if (r) return r;
    if (!d.out_count) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step_batched: null count pointer");
  }
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  size_t empties = 0;
  for (int i = 0; i < nsteps; i++) {
    const zr_step_desc& d = steps[i];
    if (d.skel.T == 0) {
      empties = std::max(empties, 8 * (size_t)d.S * d.S + 256);
      continue;
    }
    items.push_back(step_item(&d.skel, d.newvar, d.y, d.S, d.samples, d.probes, d.ldb, d.offset, d.out_exps,
                              d.out_coef, d.out_cap, d.out_count));
  }
  zr_status r = run_batch(ctx, items.data(), (int)items.size(), ctx->d_status_call, st);
  if (r) return r;
  for (int i = 0; i < nsteps; i++)
    if (steps[i].skel.T == 0) {
      // samples of empty steps are still checked, after the batch (its workspace is free again)
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_step_batched");
      if ((r = ensure_ws(ctx, empties, st))) return r;
      empty_step(ctx, steps[i].S, steps[i].samples, steps[i].out_count, ctx->d_status_call, st);
    }
  return finish_sync_call(ctx, st, nullptr);
}

extern "C" zr_status zr_zippel_step_host(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y,
                                         int32_t S, const uint64_t* samples, const uint64_t* probes, int64_t ldb,
                                         int32_t offset, uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap,
                                         int64_t* out_count, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  zr_status r = check_step_args(ctx, skel, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef, out_cap);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t T = skel->T, nv = skel->nv;
  const int64_t cap = T * S;
  // device copies of the inputs and the output come first in the workspace
  auto carve_io = [&](Carver& cv, uint8_t** d_exps, uint64_t** d_y, uint64_t** d_s, uint64_t** d_b, uint8_t** d_oe,
                      uint64_t** d_oc) {
    *d_exps = cv.take<uint8_t>((size_t)(T > 0 ? T : 1) * nv);
    *d_y = cv.take<uint64_t>(newvar > 0 ? newvar : 1);
    *d_s = cv.take<uint64_t>(S);
    *d_b = cv.take<uint64_t>((size_t)S * (T > 0 ? T : 1));
    *d_oe = cv.take<uint8_t>((size_t)(cap > 0 ? cap : 1) * nv);
    *d_oc = cv.take<uint64_t>(cap > 0 ? cap : 1);
  };
  uint8_t *d_exps, *d_oe;
  uint64_t *d_y, *d_s, *d_b, *d_oc;
  Carver m0(nullptr);
  carve_io(m0, &d_exps, &d_y, &d_s, &d_b, &d_oe, &d_oc);
  const size_t io = (m0.off + 255) & ~(size_t)255;
  zr_poly probe_skel = {skel->nv, T, nullptr, nullptr};
  BatchItem it = step_item(&probe_skel, newvar, nullptr, S, nullptr, nullptr, T, offset, nullptr, nullptr, cap,
                           ctx->d_count);
  const size_t need = io + std::max(batch_ws_need(ctx, &it, 1), (size_t)(8 * S * S + 256));
  if ((r = ensure_ws(ctx, need, st))) return r;
  Carver cv(ctx->ws);
  carve_io(cv, &d_exps, &d_y, &d_s, &d_b, &d_oe, &d_oc);
  cudaError_t e = cudaSuccess;
  if (T > 0) e = cudaMemcpyAsync(d_exps, skel->exps, (size_t)T * nv, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && newvar > 0) e = cudaMemcpyAsync(d_y, y, sizeof(uint64_t) * newvar, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, samples, sizeof(uint64_t) * S, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && T > 0)
    e = cudaMemcpy2DAsync(d_b, sizeof(uint64_t) * T, probes, sizeof(uint64_t) * ldb, sizeof(uint64_t) * T, S,
                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_step_host: copy in");
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  if (T == 0) {
    Carver cz(ctx->ws + io);
    uint64_t* invd = cz.take<uint64_t>((size_t)S * S);
    cudaMemsetAsync(ctx->d_count, 0, sizeof(int64_t), st);
    launch_newton_table(S, d_s, ctx->M, invd, ctx->d_status_call, st);
  } else {
    zr_poly dsk = {skel->nv, T, d_exps, nullptr};
    it = step_item(&dsk, newvar, d_y, S, d_s, d_b, T, offset, d_oe, d_oc, cap, ctx->d_count);
    if ((r = run_batch(ctx, &it, 1, ctx->d_status_call, st, io))) return r;
  }
  // one transfer out and one synchronisation: the output's whole capacity
  // (min(T S, out_cap) terms; entries past the count are left unspecified)
  // goes out with the status and the count, instead of a second round trip
  // once the count is known
  const int64_t ncopy = cap < out_cap ? cap : out_cap;
  if (ncopy > 0) {
    e = cudaMemcpyAsync(out_exps, d_oe, (size_t)ncopy * nv, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_coef, d_oc, sizeof(uint64_t) * ncopy, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_step_host: copy out");
  }
  int64_t n = 0;
  r = finish_sync_call(ctx, st, &n);
  if (out_count) *out_count = n;
  if (r) return r;
  if (n > out_cap) return set_err(ctx, ZR_ERR_CAPACITY, "output skeleton larger than out_cap");
  return ZR_OK;
}

extern "C" zr_status zr_check_bounded_wait(zr_ctx* ctx, uint32_t tries, void* stream) {
  if (!ctx || tries < 1) return ZR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  launch_wait_check(tries, ctx->d_status_call, st);
  return finish_sync_call(ctx, st, nullptr);
}
