// zr_solve.cu -- the hot loop of the Zippel step: blocked synthetic division
// with the multi-right-hand-side deferred dot products (Sec. 2.2: a vector of
// powers generated in parallel, multiplied by the vector of values, and the
// modular addition deferred to one reduction per dot product).
#include <cuda_runtime.h>

#include "zr_solve.cuh"

namespace zr {

// ---------------------------------------------------------------------------
// a4: block partials of the tail Horner value for the k-blocked chain,
//   R_kb(v_j) = sum_{l in block kb} m_l v_j^{l - k_lo(kb)},  kb >= 1,
// with m_T = 1 included in the top block, so that the chain's carry-in at the
// top of block kb is sum_{kk > kb} R_kk v_j^{(kk - kb - 1) BK}.
// One CTA = 256 roots of one entry and one k-block (flattened over a batch).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_b_carry(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre, int n,
                                                 Mod M) {
  const int i = seg_of(pre, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int64_t local = blockIdx.x - pre[i];
  const int64_t rows = (D.T + 255) / 256;
  const int kb = 1 + (int)(local / rows);
  const int64_t j = (local % rows) * 256 + threadIdx.x;
  if (j >= D.T) return;
  const int64_t klo = kb * D.BK, khi = (klo + D.BK) < D.T ? (klo + D.BK) : D.T;
  const uint64_t vj = D.v[j], vpj = D.vp[j];
  const uint64_t* __restrict__ m = D.m;
  uint64_t r = kb == D.NB - 1 ? 1 : 0;
  for (int64_t l = khi - 1; l >= klo; l--) r = canon(shoup_lazy(r, vj, vpj, M), M) + __ldg(m + l);
  D.R[(int64_t)(kb - 1) * D.T + j] = canon(r, M);
}

// ---------------------------------------------------------------------------
// Self-check of the bounded waits: one warp waits on an mbarrier that nothing
// arrives on; the wait must give up after `limit` tries and report
// ST_TIMEOUT, and the kernel must return.
// ---------------------------------------------------------------------------

__global__ void k_wait_check(uint32_t limit, uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x < 32 && !mbar_wait(&bar, 0, limit) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

void launch_wait_check(uint32_t limit, uint32_t* status, cudaStream_t st) {
  k_wait_check<<<1, 64, 0, st>>>(limit, status);
  note_launch();
}

void launch_b_carry(const BDesc* Ds, const int64_t* pre, int n, int64_t nctas, const Mod& M, cudaStream_t st) {
  if (nctas > 0) { k_b_carry<<<(unsigned)nctas, 256, 0, st>>>(Ds, pre, n, M); note_launch(); }
}

// Right-hand sides per consumer thread (CG) the solve is built for; each
// exists for a range of consumer-warp counts G (S <= G CG).
int solve_tiles(int* out, int cap) {
  static const int t[] = {2, 3, 4, 6, 8};
  int n = 0;
  for (int x : t)
    if (n < cap) out[n++] = x;
  return n;
}

int solve_roots_per_item() { return 32; }
int solve_max_groups() { return 8; }

bool solve_instance_exists(int cg, int groups) {
  return solve_occupancy_narrow(cg, groups) > 0 || solve_occupancy_wide(cg, groups) > 0;
}

int solve_blocks_per_sm(int cg, int groups) {
  const int n = solve_occupancy_narrow(cg, groups);
  if (n > 0) return n;
  const int w = solve_occupancy_wide(cg, groups);
  return w > 0 ? w : 1;
}

bool launch_b_solve(int cg, int groups, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                    cudaStream_t st) {
  if (nitems <= 0) return true;
  return solve_launch_narrow(cg, groups, Ds, items, nitems, sms, M, st) ||
         solve_launch_wide(cg, groups, Ds, items, nitems, sms, M, st);
}

}  // namespace zr
