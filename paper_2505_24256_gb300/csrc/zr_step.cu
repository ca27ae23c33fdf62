// zr_step.cu -- kernels of the Zippel step (Sec. 1, Sec. 2.2).
//
//   anchor values + node check   v_j = prod_{m<k} y_m^{e_{j,m}}, distinct   (a2)
//   master polynomial            M(z) = prod_j (z - v_j)                    (a3)
//   synthetic division + dots    acc[s][j] = sum_k q_{j,k} b[s][k],
//                                q_{j,k-1} = m_k + v_j q_{j,k}, den_j = q_j(v_j)   (a4, a5)
//   finish                       c[s][j] = acc[s][j] / den_j (batch inverse)
//   Newton in the new variable   divided differences, monomial form, compaction (a6)
#include <cuda_runtime.h>

#include "zr_device.cuh"
#include "zr_kernels.cuh"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Standalone kernels of zr_anchor_values and zr_newton_batched; the step
// itself runs through the batched kernels of zr_batch.cu.
// ---------------------------------------------------------------------------
// a2: per-variable power tables y_m^e (the paper's power table, Sec. 2.2) and
// anchor values.
// ---------------------------------------------------------------------------

__global__ void k_powtab(const uint64_t* __restrict__ y, int k, Mod M, uint64_t* __restrict__ tab) {
  int m = blockIdx.x, e = threadIdx.x;
  if (m < k && e < kPowTab) tab[m * kPowTab + e] = pow_mod(y[m], (uint64_t)e, M);
}

__global__ void k_anchor(int64_t T, int nv, const uint8_t* __restrict__ exps, int k,
                         const uint64_t* __restrict__ tab, int offset, Mod M, uint64_t* __restrict__ v,
                         uint64_t* __restrict__ vp, uint64_t* htab, uint64_t hmask, uint32_t* status) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  const uint8_t* e = exps + j * nv;
  uint64_t acc = 1;
  for (int m = 0; m < k; m++) acc = mul_mod(acc, tab[m * kPowTab + e[m]], M);
  v[j] = acc;
  vp[j] = shoup_pre(acc, M);
  if (offset == 1 && acc == 0) atomicOr(status, ST_ZERO_NODE);
  if (htab) node_insert(acc, htab, hmask, status);
}

__global__ void k_shoup_pre(int64_t T, const uint64_t* __restrict__ v, Mod M, uint64_t* __restrict__ vp,
                            int offset, uint32_t* status) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  uint64_t x = v[j];
  if (x >= M.p) { atomicOr(status, ST_DUP_NODE | ST_ZERO_NODE); x = 0; }
  vp[j] = shoup_pre(x, M);
  if (offset == 1 && x == 0) atomicOr(status, ST_ZERO_NODE);
}

__global__ void k_node_check(int64_t T, const uint64_t* __restrict__ v, uint64_t* htab, uint64_t hmask,
                             uint32_t* status) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < T) node_insert(v[j], htab, hmask, status);
}

void launch_powtab(const uint64_t* y, int k, const Mod& M, uint64_t* tab, cudaStream_t st) {
  if (k > 0) { k_powtab<<<k, kPowTab, 0, st>>>(y, k, M, tab); note_launch(); }
}
void launch_anchor(int64_t T, int nv, const uint8_t* exps, int k, const uint64_t* tab, int offset, const Mod& M,
                   uint64_t* v, uint64_t* vp, uint64_t* htab, uint64_t hmask, uint32_t* status, cudaStream_t st) {
  if (T > 0) { k_anchor<<<cdiv(T, 256), 256, 0, st>>>(T, nv, exps, k, tab, offset, M, v, vp, htab, hmask, status); note_launch(); }
}
void launch_shoup_pre(int64_t T, const uint64_t* v, const Mod& M, uint64_t* vp, int offset, uint32_t* status,
                      cudaStream_t st) {
  if (T > 0) { k_shoup_pre<<<cdiv(T, 256), 256, 0, st>>>(T, v, M, vp, offset, status); note_launch(); }
}
void launch_node_check(int64_t T, const uint64_t* v, uint64_t* htab, uint64_t hmask, uint32_t* status,
                       cudaStream_t st) {
  if (T > 0) { k_node_check<<<cdiv(T, 256), 256, 0, st>>>(T, v, htab, hmask, status); note_launch(); }
}

// ---------------------------------------------------------------------------
// a6: Newton in the new variable, Eq. (newton).
//   invd[l S + s] = 1 / (x_s - x_{s-l}),  1 <= l <= s < S   (shared by all terms)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kNewtonThreads) k_newton_table(int S, const uint64_t* __restrict__ xs, Mod M,
                                                                  uint64_t* __restrict__ W, uint32_t* status) {
  extern __shared__ uint64_t tsm[];
  newton_table_block(S, xs, W, status, tsm, M);
}

void launch_newton_table(int S, const uint64_t* xs, const Mod& M, uint64_t* W, uint32_t* status, cudaStream_t st) {
  static DeviceOnce attr;
  attr.run([] {
    cudaFuncSetAttribute(k_newton_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(8 * newton_table_words(kNewtonMax)));
  });
  const size_t smem = 8 * (size_t)newton_table_words(S);
  { k_newton_table<<<1, kNewtonThreads, smem, st>>>(S, xs, M, W, status); note_launch(); }
}

// One block of 128 terms: the block's values and W in shared memory, then
// S^2 multiply-accumulates per term.  coef may alias vals: a thread reads its
// whole column before it writes it.
__global__ void __launch_bounds__(128) k_newton(int64_t nterms, int S, const uint64_t* __restrict__ Wg,
                                                const uint64_t* vals, int64_t ld, Mod M, uint64_t* coef) {
  extern __shared__ uint64_t nsm[];
  uint64_t* W = nsm;
  uint64_t* val = nsm + S * S;
  for (int idx = threadIdx.x; idx < S * S; idx += blockDim.x) W[idx] = Wg[idx];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < nterms;
  if (active)
    for (int s = 0; s < S; s++) val[s * 128 + threadIdx.x] = canon(vals[(int64_t)s * ld + j], M);
  __syncthreads();
  if (!active) return;
  newton_apply(S, W, val + threadIdx.x, 128, 1, coef + j, ld, M);
}

size_t newton_smem(int S, int terms) { return sizeof(uint64_t) * ((size_t)S * S + (size_t)S * terms); }

void launch_newton(int64_t nterms, int npts, const uint64_t* W, const uint64_t* vals, int64_t ld, const Mod& M,
                   uint64_t* coef, cudaStream_t st) {
  if (nterms <= 0) return;
  static DeviceOnce attr;
  attr.run([] {
    cudaFuncSetAttribute(k_newton, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)newton_smem(kNewtonMax, 128));
  });
  const unsigned grid = cdiv(nterms, 128);
  { k_newton<<<grid, 128, newton_smem(npts, 128), st>>>(nterms, npts, W, vals, ld, M, coef); note_launch(); }
}

int64_t scan_blocks(int64_t n) { return (n + kFinB - 1) / kFinB; }

}  // namespace zr
