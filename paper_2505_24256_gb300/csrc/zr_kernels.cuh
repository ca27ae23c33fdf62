// zr_kernels.cuh -- declarations shared by the library's CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "zr_arith.cuh"

namespace zr {

// Number of kernels the library has launched (a diagnostic counter).
unsigned long long launch_count();
void note_launch();

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
  int32_t s_tile;  // right-hand sides per thread
};

void launch_powtab(const uint64_t* y, int k, const Mod& M, uint64_t* tab, cudaStream_t st);
void launch_anchor(int64_t T, int nv, const uint8_t* exps, int k, const uint64_t* tab, int offset, const Mod& M,
                   uint64_t* v, uint64_t* vp, uint64_t* htab, uint64_t hmask, uint32_t* status, cudaStream_t st);
void launch_shoup_pre(int64_t T, const uint64_t* v, const Mod& M, uint64_t* vp, int offset, uint32_t* status,
                      cudaStream_t st);
void launch_node_check(int64_t T, const uint64_t* v, uint64_t* htab, uint64_t hmask, uint32_t* status, cudaStream_t st);
// master polynomial: m[0..T-1] (monic, m_T = 1 implicit).  tmp: 2*T words.
void launch_master_poly(int64_t T, const uint64_t* v, const Mod& M, uint64_t* m, uint64_t* tmp, cudaStream_t st);
void launch_expand_b(int64_t T, int S, const uint64_t* b, int64_t ldb, const Mod& M, BX* bx, cudaStream_t st);
void launch_carry_partials(const StepDims& D, const uint64_t* m, const uint64_t* v, const uint64_t* vp,
                           const Mod& M, uint64_t* R, cudaStream_t st);
void launch_solve(const StepDims& D, const uint64_t* m, const uint64_t* v, const uint64_t* vp, const uint64_t* R,
                  const uint64_t* b, int64_t ldb, const Mod& M, uint64_t* part, uint64_t* denp, cudaStream_t st);
// right-hand-side tiles the solve kernel is built for, and its resident CTAs per SM
int solve_tiles(int* out, int cap);
int solve_blocks_per_sm(int s_tile);
// finish: combine partials, batch-invert the denominators, scale.  Writes
// c (S x ldc) when c != nullptr.
void launch_finish_solve(const StepDims& D, int offset, const uint64_t* v, const uint64_t* part,
                         const uint64_t* denp, const Mod& M, uint64_t* c, int64_t ldc, uint32_t* status,
                         cudaStream_t st);
// finish fused with Newton in the new variable: g (S x T, monomial
// coefficients) and cnt[j] = number of nonzero g[.][j].
void launch_newton_table(int S, const uint64_t* xs, const Mod& M, uint64_t* invd, uint32_t* status, cudaStream_t st);
void launch_finish_newton(const StepDims& D, int offset, const uint64_t* v, const uint64_t* part,
                          const uint64_t* denp, const uint64_t* xs, const uint64_t* invd, const Mod& M,
                          uint64_t* g, int32_t* cnt, uint32_t* status, cudaStream_t st);
// plain batched Newton: vals (npts x ld) -> coef (npts x ld)
void launch_newton(int64_t nterms, int npts, const uint64_t* xs, const uint64_t* invd, const uint64_t* vals,
                   int64_t ld, const Mod& M, uint64_t* coef, cudaStream_t st);
// compaction of the new skeleton
int64_t scan_blocks(int64_t n);  // number of scan blocks
void launch_compact(int64_t T, int S, int nv, int k, const uint8_t* exps, const uint64_t* g, const int32_t* cnt,
                    int64_t* bsum, int64_t cap, uint8_t* out_exps, uint64_t* out_coef, int64_t* out_count,
                    cudaStream_t st);

}  // namespace zr
