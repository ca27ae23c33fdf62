// zr_kernels.cuh -- declarations shared by the library's CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "zr_arith.cuh"

namespace zr {

// Number of kernels the library has launched (a diagnostic counter).
unsigned long long launch_count();
void note_launch();
void note_launches(uint64_t n);   // kernels of a replayed graph

// Kernel attributes (the dynamic shared-memory limit) belong to a device, so
// a once-per-process flag would configure only the first device a process
// uses.  DeviceOnce runs its set-up once per device (the current one at the
// call); DeviceValue caches a per-device integer such as an occupancy.
// Devices beyond kAttrDevices simply redo the set-up on every call.  Two
// threads may both run a set-up the first time: setting an attribute twice is
// harmless.
constexpr int kAttrDevices = 64;
int current_device();
struct DeviceOnce {
  std::atomic<uint64_t> done{0};
  template <class F>
  void run(F&& fn) {
    const int d = current_device();
    const uint64_t bit = (d >= 0 && d < kAttrDevices) ? 1ull << d : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return;
    fn();
    if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
  }
};
struct DeviceValue {
  std::atomic<int> v[kAttrDevices] = {};
  template <class F>
  int get(F&& compute) {
    const int d = current_device();
    if (d < 0 || d >= kAttrDevices) return compute();
    int x = v[d].load(std::memory_order_acquire);
    if (!x) {
      x = compute();
      v[d].store(x, std::memory_order_release);
    }
    return x;
  }
};

// Device status flags (OR-ed into one 32-bit word per call).
enum : uint32_t {
  ST_DUP_NODE = 1u,      // two skeleton monomials take the same anchor value
  ST_ZERO_NODE = 2u,     // an anchor value is 0 while the exponents start at 1
  ST_ZERO_DEN = 4u,      // a Lagrange denominator q_j(v_j) vanished
  ST_DUP_SAMPLE = 8u,    // two samples of the new variable coincide
  ST_POLE = 16u,         // a denominator vanished at a probe
  ST_THIELE = 32u,       // univariate rational reconstruction failed
  ST_TIMEOUT = 64u,      // a bounded wait gave up
  ST_HASH_FULL = 128u,   // node table overflow (cannot happen with the sizes used)
  ST_DEGREE = 256u,      // a reconstruction exceeded its degree bound
};

constexpr int kMaxVars = 64;
constexpr int kPowTab = 256;          // exponents are bytes

// ---- host-side launchers (zr_step.cu) ----
struct StepDims {
  int64_t T;
  int32_t S;
  int32_t NB;      // k-blocks
  int64_t BK;      // k-block length (the top block may be shorter)
  int32_t s_tile;  // right-hand sides per consumer thread of the solve
};

// One step (mode 0: a Zippel step whose nodes are the anchor values of a
// skeleton) or one transposed Vandermonde system (mode 1: given nodes) of a
// batch, with its plan and its workspace.  The batched kernels take a device
// array of these plus prefix sums that map flattened indices to entries.
struct BDesc {
  int64_t T, BK, ldb, ldc, out_cap;
  uint64_t hmask;
  int32_t S, k, nv, offset, mode, NB, s_tile, nst, levels;
  int32_t Sn;   // samples interpolated: S (systems solved), or S + 1 with c0
  const uint8_t* exps;
  const uint64_t *y, *xs, *b;
  uint64_t *tab, *v, *vp, *htab, *m, *tmp, *tpart, *R, *part, *denp, *invd, *g, *c;
  int32_t* cnt;
  int64_t *bsum, *out_count;
  uint8_t* out_exps;
  uint64_t* out_coef;
  uint32_t* status;
  const uint64_t* c0;   // the solution at samples[0] (then b starts at the second sample), or null
};

void launch_powtab(const uint64_t* y, int k, const Mod& M, uint64_t* tab, cudaStream_t st);
void launch_anchor(int64_t T, int nv, const uint8_t* exps, int k, const uint64_t* tab, int offset, const Mod& M,
                   uint64_t* v, uint64_t* vp, uint64_t* htab, uint64_t hmask, uint32_t* status, cudaStream_t st);
void launch_shoup_pre(int64_t T, const uint64_t* v, const Mod& M, uint64_t* vp, int offset, uint32_t* status,
                      cudaStream_t st);
void launch_node_check(int64_t T, const uint64_t* v, uint64_t* htab, uint64_t hmask, uint32_t* status, cudaStream_t st);
// batched carry and solve (zr_solve.cu)
void launch_wait_check(uint32_t limit, uint32_t* status, cudaStream_t st);
void launch_b_carry(const BDesc* Ds, const int64_t* pre, int n, int64_t nctas, const Mod& M, cudaStream_t st);
// false when no solve kernel is built for (s_tile, groups): nothing launched
bool launch_b_solve(int s_tile, int groups, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                    cudaStream_t st);
// right-hand-side tiles the solve kernel is built for, and its resident CTAs per SM
int solve_tiles(int* out, int cap);
int solve_blocks_per_sm(int s_tile, int groups);
bool solve_instance_exists(int s_tile, int groups);
int solve_roots_per_item();   // roots of one work item
int solve_max_groups();       // consumer groups per CTA: S <= groups * s_tile
// Newton on shared nodes: W (S x S) from the nodes, then vals (npts x ld) ->
// monomial coefficients coef (npts x ld) through W
void launch_newton_table(int S, const uint64_t* xs, const Mod& M, uint64_t* W, uint32_t* status, cudaStream_t st);
void launch_newton(int64_t nterms, int npts, const uint64_t* W, const uint64_t* vals, int64_t ld, const Mod& M,
                   uint64_t* coef, cudaStream_t st);
constexpr int kFinB = 32;                 // terms per block of a step's finish and compaction
constexpr int kFinSplit = 4;              // warps sharing a block's terms in the finish (by right-hand side and output)
size_t newton_smem(int S, int terms);     // dynamic shared memory of one block of `terms` terms
int64_t scan_blocks(int64_t n);           // number of kFinB-term compaction blocks
// split partials the product tree may use for T leaves (words = that x T)
inline int64_t tree_split_max(int64_t T) {
  const int64_t s = T > 0 ? (4 * 152 * 512 + T - 1) / T : 1;
  return s < 1 ? 1 : (s > 16 ? 16 : s);
}

}  // namespace zr
