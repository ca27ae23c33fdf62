// zr_internal.h -- host-side context shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "zr.h"
#include "zr_kernels.cuh"
#include "zr_ntt.cuh"

// Phases of a step timed by the optional profiler (CUDA events recorded on
// the call's stream around each phase).
// PH_NTT times each launch of the transform tile kernel, PH_DESC each launch
// of the descent's cluster level kernel, inside PH_FAST; both count their
// butterflies as the phase's work.  PH_PSUM times each launch of the direct
// power sums kernel, its T^2 Shoup steps the work.
enum zr_phase {
  PH_ANCHOR = 0, PH_MASTER, PH_EXPAND, PH_CARRY, PH_SOLVE, PH_NEWTON, PH_COMPACT, PH_EVAL, PH_FAST, PH_NTT, PH_DESC,
  PH_PSUM, PH_N
};

struct zr_prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Pending { int phase; cudaEvent_t a, b; double work; };
  std::vector<Pending> pending;
  double total_ms[PH_N] = {};
  long long count[PH_N] = {};
  double work[PH_N] = {};
};

struct zr_plan_entry {
  int64_t T;
  int S;
  zr::StepDims D;
};

struct zr_ctx {
  zr::Mod M;
  zr_prof prof;
  std::vector<zr_plan_entry> plans;   // tuned launch plans by (T, S)
  int device = 0;
  int sms = 0;
  // grow-only device workspace
  char* ws = nullptr;
  size_t ws_cap = 0;
  // accumulated device status of _async calls (device word + pinned mirror)
  uint32_t* d_status = nullptr;
  uint32_t* h_status = nullptr;
  // scratch status word of the synchronous calls
  uint32_t* d_status_call = nullptr;
  int64_t* d_count = nullptr;   // scratch output counts
  int64_t* h_count = nullptr;   // pinned mirror
  void* h_stage = nullptr;      // pinned staging of batch tables
  size_t h_stage_cap = 0;
  cudaEvent_t stage_event = nullptr;   // last copy out of h_stage
  // the solve runs one wave of CTAs walking its work list (persistent), or
  // one CTA per work item, which lets higher-priority streams take SMs
  // between items (the serving loop's lane of large requests)
  bool solve_persistent = true;
  // side stream of a step batch (work that depends only on the samples runs
  // there, overlapping the tree and the solve), with its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // streams on which a batch's O(T log^2 T) entries run concurrently, with
  // their fork and join events
  cudaStream_t fstream[4] = {};
  cudaEvent_t fev_fork = nullptr, fev_join[4] = {};
  // the auxiliary stream and fork / join events of a fast solve on the call's
  // stream (slot 4) or on fstream[j] (slot j)
  cudaStream_t faux[5] = {};
  cudaEvent_t faux_fork[5] = {}, faux_join[5] = {};
  // the O(T log^2 T) solve: constants of the transform primes, the twiddle
  // tables (grown on demand) and the choice between the two solve methods
  zr::NttConsts ntt;
  void* ntt_tw = nullptr;
  int ntt_logN = 0;
  int solve_method = 0;            // 0: by size, 1: quadratic, 2: fast where supported
  int64_t fast_min_T = 0;          // size from which method 0 takes the fast path (0: built-in default)
  // workspace of the fast probe evaluator, sized once the group count is
  // known (grow-only, separate from the step workspace)
  char* fprobe_ws = nullptr;
  size_t fprobe_cap = 0;
  // scratch of the probe lanes (probes generated on streams of their own,
  // e.g. by the server for several requests at once): the evaluator's
  // workspace and the fast evaluator's, per lane (grow-only)
  static constexpr int kProbeLanes = 4;
  char* pl_ws[kProbeLanes] = {};
  size_t pl_cap[kProbeLanes] = {};
  char* pl_fws[kProbeLanes] = {};
  size_t pl_fcap[kProbeLanes] = {};
  std::string err;
  std::mutex mu;                // guards err for the serve thread
};

namespace zr {

// Bump allocator over the context workspace.  Used in two passes: measure
// (base == nullptr) then carve.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

zr_status set_err(zr_ctx* ctx, zr_status st, const std::string& msg);
// Modulus descriptor for a prime 2^32 < p < 2^63; false when p is out of
// range or composite.  Host arithmetic only (allocates nothing).
bool mod_for_prime(uint64_t p, Mod* out);
// profiler marks (no-ops when profiling is off)
cudaEvent_t prof_mark(zr_ctx* ctx, cudaStream_t st);
void prof_add(zr_ctx* ctx, int phase, cudaEvent_t a, cudaEvent_t b, double work = 0);
void prof_collect(zr_ctx* ctx);
zr_status cuda_err(zr_ctx* ctx, cudaError_t e, const char* where);
zr_status ensure_ws(zr_ctx* ctx, size_t need, cudaStream_t st);
zr_status status_from_flags(zr_ctx* ctx, uint32_t flags);
StepDims plan_step(const zr_ctx* ctx, int64_t T, int S);
double plan_cost(const zr_ctx* ctx, const StepDims& D);
uint64_t hash_slots(int64_t T);

// Workspace of one step or system (carved in the context workspace).
struct StepWs {
  uint64_t *tab, *v, *vp, *htab, *m, *tmp, *tpart, *R, *part, *denp, *invd, *g;
  int32_t* cnt;
  int64_t* bsum;
};
// S: samples of the step (Newton points); Ssolve: systems solved (S, or S - 1
// when the first sample's solution is given)
StepWs carve_step(Carver& cv, int64_t T, int S, int k, const StepDims& D, int Ssolve = -1);

// One entry of a batch: a Zippel step (mode 0) or a transposed Vandermonde
// system with given nodes (mode 1).  All pointers are device pointers.
struct BatchItem {
  int mode = 0;
  int64_t T = 0;
  int S = 1, k = 0, nv = 1, offset = 0;
  const uint8_t* exps = nullptr;
  const uint64_t *y = nullptr, *xs = nullptr, *b = nullptr, *vin = nullptr;
  int64_t ldb = 0;
  uint8_t* out_exps = nullptr;
  uint64_t* out_coef = nullptr;
  int64_t out_cap = 0;
  int64_t* out_count = nullptr;
  uint64_t* c = nullptr;
  int64_t ldc = 0;
  uint32_t* status = nullptr;   // the entry's own status word (else the batch's)
  // Zippel steps (mode 0) with S >= 2 only: the skeleton's coefficients (T,
  // device), which are the solution at the first sample (the value of x_k
  // they were taken at).  The step then solves only samples 1..S-1 (b's row
  // 0 is not read) and interpolates through all S.
  const uint64_t* c0 = nullptr;
  int solve_S() const { return c0 && mode == 0 && S >= 2 ? S - 1 : S; }
};
// Workspace bytes a batch needs (its regions plus the device tables).
size_t batch_ws_need(const zr_ctx* ctx, const BatchItem* items, int n);
// Enqueues a batch; its workspace starts `base` bytes into the context
// workspace (the caller ensured base + batch_ws_need, or the call grows it
// when nothing before `base` is live).  status: device word of ST_* flags.
zr_status run_batch(zr_ctx* ctx, const BatchItem* items, int n, uint32_t* status, cudaStream_t st, size_t base = 0);
// The same batch with its workspace at `ws` (batch_ws_need bytes, owned by
// the caller): the tables are staged and the batch run once on `st`, then its
// kernels are captured into *graph; *launches counts the captured kernels.
zr_status batch_graph_capture(zr_ctx* ctx, const BatchItem* items, int n, uint32_t* status, char* ws,
                              cudaStream_t st, cudaGraph_t* graph, uint64_t* launches);
// argument checks and batch entry of one Zippel step (zr_zippel_step's arguments)
zr_status check_step_args(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                          const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                          uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap);
BatchItem step_item(const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S, const uint64_t* samples,
                    const uint64_t* probes, int64_t ldb, int32_t offset, uint8_t* out_exps, uint64_t* out_coef,
                    int64_t out_cap, int64_t* d_count);

// the O(T log^2 T) solve (zr_fast.cu)
constexpr int64_t kFastMaxT = 1ll << 21;   // largest T of the fast path (transforms up to 2^22)
zr::NttConsts make_ntt_consts(uint64_t p);
size_t fast_ws_need(int64_t T, int R);
// (aux, ev_fork, ev_join: a second stream and two events on which the power
// sums run beside the right-hand sides' descent; null: all on st)
zr_status fast_solve_enqueue(zr_ctx* ctx, int64_t T, int S, const uint64_t* v, const uint64_t* vp, const uint64_t* b,
                             int64_t ldb, uint64_t* part, uint64_t* den, char* ws, cudaStream_t st,
                             cudaStream_t aux = nullptr, cudaEvent_t ev_fork = nullptr, cudaEvent_t ev_join = nullptr);
// whether a system of T unknowns takes the fast path in this context
// (batch_n: the number of systems in the call; alone, the fast path is taken from a smaller T)
bool use_fast_solve(const zr_ctx* ctx, int64_t T, int S, int batch_n = 1);
// grows the transform tables for fast solves of up to T unknowns
zr_status fast_tables_for(zr_ctx* ctx, int64_t T, cudaStream_t st);
// scheduling weights (multiply-accumulate equivalents) of a step's solve and
// of its probes, by the method each takes in this context
double solve_work(const zr_ctx* ctx, int64_t T, int S);
double probe_work(const zr_ctx* ctx, int64_t T, int S, int64_t Tf);
// whether T probes of a function of Tf terms take the fast evaluator (the
// transposed tree), which reads the group count G <= Tf on the host and
// falls back to the matrix-vector kernel when G > kFastMaxT
constexpr int kFastProbeMaxS = 64;            // columns of the fast evaluator
bool use_fast_probes(const zr_ctx* ctx, int64_t T, int64_t Tf, int S);
size_t fast_probes_ws_need(int64_t G, int64_t T, int S);
zr_status fast_probes_enqueue(zr_ctx* ctx, int64_t G, const uint64_t* U, const uint64_t* W, int64_t ldw, int S,
                              int64_t T, uint64_t* out, int64_t ldo, char* ws, cudaStream_t st);

// evaluator (zr_eval.cu)
size_t probes_ws_need(const zr_ctx* ctx, const zr_poly* f, int k, int S, int64_t T);
// (fws, fcap: the grow-only workspace of the fast evaluator; null: the context's)
zr_status probes_enqueue(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                         const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                         char* base, cudaStream_t st, char** fws = nullptr, size_t* fcap = nullptr);
// (lane: -1 the context's workspace, which the batch runner shares in stream
// order; 0 .. kProbeLanes-1 that probe lane's own scratch, for probes run
// concurrently on streams of their own)
zr_status probes_impl(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                      const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                      cudaStream_t st, int lane = -1);

// argument check of a reconstruction request (zr_recon.cu)
zr_status check_recon_args(zr_ctx* ctx, const zr_blackbox* bb, const zr_recon_params* prm);

// balanced step pieces (zr_balance.cu)
void launch_probe_points(int64_t T, int S, int nv, int k, int offset, const uint64_t* y, const uint64_t* cs,
                         const uint64_t* z, const Mod& M, uint64_t* pts, cudaStream_t st);
void launch_ratio(int64_t T, int S, const uint64_t* Nv, const uint64_t* Dv, int64_t ld, const Mod& M, uint64_t* pre,
                  uint64_t* out, int64_t ldo, uint32_t* status, cudaStream_t st);
size_t thiele_scratch_words(int64_t Tmax, int n);
void launch_thiele_balance(int64_t Tmax, int n, const uint64_t* xs, const uint64_t* fvals, int64_t ldf,
                           const uint64_t* dprev, int dN, int dD, int64_t TN, int64_t TD, uint64_t* scratch,
                           const Mod& M, uint64_t* bN, int64_t ldN, uint64_t* bD, int64_t ldD, uint32_t* status,
                           cudaStream_t st);
void launch_normalise(int64_t n1, uint64_t* a1, int64_t n2, uint64_t* a2, const uint64_t* pivot, uint64_t* tmp,
                      const Mod& M, uint32_t* status, cudaStream_t st);
// kernels used by the reconstruction driver
void launch_eval_points(const zr_poly* f, int64_t npts, const uint64_t* pts, const Mod& M, uint64_t* out,
                        cudaStream_t st);

}  // namespace zr
