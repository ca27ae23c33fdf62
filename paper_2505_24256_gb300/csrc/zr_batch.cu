// zr_batch.cu -- batched Zippel steps and Vandermonde systems.
//
// Steps (or systems) of different T and S share every launch: each kernel
// gets the device array of descriptors (BDesc) and a prefix sum over the
// entries' work (roots, leaf chunks, tree tiles, kFinB-term blocks); a flattened
// index is mapped back to (entry, local index) by binary search.  The solve
// kernel is persistent and walks a device work list of (entry, root tile,
// k-block, right-hand-side tile) items, longest first.  A batch of one is the
// single step, so every step goes through these kernels.
//
// Phases (Sec. 1, Sec. 2.2):
//   anchor values v_j and the distinctness check (hash table)      a2
//   master polynomial by a product tree                             a3
//   k-block carries, then the synthetic-division / dot kernel       a4, a5
//   denominators, Montgomery batch inversion, Newton, counts        a4, a6
//   compaction of the new skeleton                                  a6
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "zr_device.cuh"
#include "zr_internal.h"
#include "zr_launch.cuh"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---- a2 ---------------------------------------------------------------------

__global__ void k_b_fill_hash(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre, int n) {
  pdl_enter();
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[n]) return;
  const int i = seg_of(pre, n, x);
  Ds[i].htab[x - pre[i]] = kEmptySlot;
}

__global__ void k_b_powtab(const BDesc* __restrict__ Ds, Mod M) {
  pdl_enter();
  const BDesc& D = Ds[blockIdx.y];
  const int m = blockIdx.x, e = threadIdx.x;
  if (D.mode == 0 && m < D.k) D.tab[m * kPowTab + e] = pow_mod(D.y[m], (uint64_t)e, M);
}

__global__ void k_b_anchor(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre, int n, Mod M) {
  pdl_enter();
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[n]) return;
  const int i = seg_of(pre, n, x);
  const BDesc& D = Ds[i];
  const int64_t j = x - pre[i];
  uint64_t acc;
  if (D.mode == 0) {
    const uint8_t* e = D.exps + j * D.nv;
    acc = 1;
    for (int m = 0; m < D.k; m++) acc = mul_mod(acc, D.tab[m * kPowTab + e[m]], M);
    D.v[j] = acc;
  } else {
    acc = D.v[j];
    if (acc >= M.p) {
      atomicOr(D.status, ST_DUP_NODE);
      acc = 0;
    }
  }
  D.vp[j] = shoup_pre(acc, M);
  if (D.offset == 1 && acc == 0) atomicOr(D.status, ST_ZERO_NODE);
  node_insert(acc, D.htab, D.hmask, D.status);
}

// ---- a3: product tree ---------------------------------------------------------

constexpr int kTreeL1 = 7;   // levels 0..6 inside one CTA (128 leaves, one per thread)

__global__ void __launch_bounds__(1 << kTreeL1) k_b_tree_leaf(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre,
                                                     int n, Mod M) {
  __shared__ uint64_t buf[2][1 << kTreeL1];
  const int i = seg_of(pre, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int64_t base = (blockIdx.x - pre[i]) << kTreeL1;
  const int cnt = (int)((D.T - base) < (1 << kTreeL1) ? (D.T - base) : (1 << kTreeL1));
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const uint64_t x = D.v[base + t];
    buf[0][t] = x ? M.p - x : 0;               // z - v_j
  }
  __syncthreads();
  int cur = 0;
  for (int l = 0; l < kTreeL1; l++) {
    const int size = 1 << l, pair = 2 << l;
    for (int pos = threadIdx.x; pos < cnt; pos += blockDim.x) {
      const int po = pos & ~(pair - 1);
      uint64_t r;
      if (cnt - po <= size) r = buf[cur][pos];
      else r = conv_coef(buf[cur], po, size, min(size, cnt - po - size), pos - po, M);
      buf[cur ^ 1][pos] = r;
    }
    __syncthreads();
    cur ^= 1;
  }
  uint64_t* out = D.levels <= kTreeL1 ? D.m : D.tmp;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) out[base + t] = buf[cur][t];
}

// Levels >= kTreeL1: each pair (A, B) of sibling polynomials (monic, leading
// 1 implicit) is multiplied by a schoolbook convolution.  A CTA owns up to
// kTNO consecutive output coefficients of one pair; thread t keeps kTR of them
// (t, t + NT, .. : conflict-free shared-memory reads) in 160-bit accumulators,
// so every staged A coefficient feeds kTR multiply-accumulates.  When a level
// has too few output tiles to fill the GPU, the inner (A) range is split over
// gridDim.y CTAs whose partial sums a second kernel adds.
constexpr int kTR = 4;
constexpr int kTNO = 512;
constexpr int kTIC = 256;

__host__ __device__ inline int tree_tile(int l) {
  const int pair = 2 << l;
  return pair < kTNO ? pair : kTNO;
}

__device__ __forceinline__ void tree_bufs(const BDesc& D, int l, const uint64_t*& in, uint64_t*& out) {
  const bool even = ((l - kTreeL1) & 1) == 0;
  in = even ? D.tmp : D.tmp + D.T;
  out = (l == D.levels - 1) ? D.m : (even ? D.tmp + D.T : D.tmp);
}

__global__ void __launch_bounds__(kTNO / kTR) k_b_tree_conv(const BDesc* __restrict__ Ds,
                                                            const int64_t* __restrict__ pre, int n, int l, int split,
                                                            Mod M) {
  __shared__ uint64_t As[kTIC];
  __shared__ uint64_t Bs[kTIC + kTNO];
  const int i = seg_of(pre, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int64_t T = D.T;
  const int NO = tree_tile(l), NT = NO / kTR;
  const int64_t t0 = (int64_t)(blockIdx.x - pre[i]) * NO;
  const uint64_t* in;
  uint64_t* out;
  tree_bufs(D, l, in, out);
  uint64_t* dst = split > 1 ? D.tpart + (int64_t)blockIdx.y * T : out;
  const int64_t size = 1ll << l, pair = 2ll << l;
  const int64_t po = t0 & ~(pair - 1);
  const int tid = threadIdx.x;
  if (T - po <= size) {   // no sibling: the coefficients pass through
#pragma unroll
    for (int r = 0; r < kTR; r++) {
      const int64_t x = t0 + tid + NT * r;
      if (x < T) dst[x] = blockIdx.y == 0 ? in[x] : 0;
    }
    return;
  }
  const int64_t a = size, b = (T - po - size) < size ? (T - po - size) : size;
  const int64_t n0 = t0 - po;                                           // first output of the tile
  const int64_t ilo = n0 - b > 0 ? n0 - b : 0;
  const int64_t ihi = (n0 + NO - 1) < a ? (n0 + NO - 1) : a;            // inclusive; A_a = 1
  const int64_t per = (ihi - ilo + split) / split;
  const int64_t slo = ilo + per * blockIdx.y;
  const int64_t shi = (slo + per - 1) < ihi ? (slo + per - 1) : ihi;
  Acc8 acc[kTR];
#pragma unroll
  for (int r = 0; r < kTR; r++) acc[r] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i0 = slo; i0 <= shi; i0 += kTIC) {
    const int64_t i1 = (i0 + kTIC - 1) < shi ? (i0 + kTIC - 1) : shi;  // inclusive
    const int ic = (int)(i1 - i0 + 1);
    const int64_t jlo = n0 - i1;                                        // smallest B index of the chunk
    __syncthreads();
    for (int t = tid; t < ic; t += NT) {
      const int64_t ii = i0 + t;
      As[t] = ii < a ? in[po + ii] : 1;
    }
    for (int t = tid; t < NO + ic - 1; t += NT) {
      const int64_t jj = jlo + t;
      Bs[t] = (jj < 0 || jj > b) ? 0 : (jj == b ? 1 : in[po + a + jj]);
    }
    __syncthreads();
    // output n = n0 + tid + NT r takes A_{i0+t} B_{n-i0-t} = As[t] Bs[tid + NT r + ic - 1 - t]
    const uint64_t* bw = Bs + tid + ic - 1;
    for (int t = 0; t < ic; t++) {
      const uint64_t x = As[t];
      const uint32_t x0 = lo32(x), x1 = hi32(x);
#pragma unroll
      for (int r = 0; r < kTR; r++) {
        const uint64_t w = bw[NT * r - t];
        mac8(acc[r], lo32(w), hi32(w), x0, x1);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kTR; r++) {
    const int64_t nn = n0 + tid + NT * r;
    if (nn < a + b) dst[po + nn] = acc8_value(acc[r], M);
  }
}

// out = sum of the split partials, for the entries that have level l
__global__ void k_b_tree_combine(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre, int n, int l,
                                 int split, Mod M) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[n]) return;
  const int i = seg_of(pre, n, x);
  const BDesc& D = Ds[i];
  if (D.levels <= l) return;
  const int64_t j = x - pre[i];
  const uint64_t* in;
  uint64_t* out;
  tree_bufs(D, l, in, out);
  uint64_t s = 0;
  for (int y = 0; y < split; y++) s = add_mod(s, D.tpart[(int64_t)y * D.T + j], M);
  out[j] = s;
}

// ---- a4/a6: finish ---------------------------------------------------------------

// The value to invert for root j and the factor its inverse is scaled by:
// q_j(v_j) (times v_j for offset 1) from the solve's k-block partials u_kb,
// q_j(v_j) = sum_kb u_kb v_j^{kb BK} (Horner in v_j^BK from the top block
// down, the partials loaded eight at a time).
__device__ __forceinline__ uint64_t root_den(const BDesc& D, int64_t j, uint64_t vj, const Mod& M, uint64_t& mult) {
  mult = 1;
  const uint64_t vBK = D.NB > 1 ? pow_mod(vj, (uint64_t)D.BK, M) : 1;
  uint64_t den = 0;
  for (int kt = D.NB; kt > 0; kt -= 8) {
    uint64_t x[8];
#pragma unroll
    for (int q = 0; q < 8; q++) x[q] = kt - 1 - q >= 0 ? D.denp[(int64_t)(kt - 1 - q) * D.T + j] : 0;
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (kt - 1 - q >= 0) den = add_mod(mul_mod(den, vBK, M), x[q], M);
  }
  if (D.offset == 1) den = mul_mod(den, vj, M);
  return den;
}

// W of every step entry (one block each): the values -> monomial map of Newton
// interpolation on the entry's S samples.
__global__ void __launch_bounds__(kNewtonThreads) k_b_newton_table(const BDesc* __restrict__ Ds, Mod M) {
  pdl_enter();
  extern __shared__ uint64_t tsm[];
  const BDesc& D = Ds[blockIdx.x];
  if (D.mode != 0 || D.T == 0) return;
  newton_table_block(D.Sn, D.xs, D.invd, D.status, tsm, M);
}

// a4 + a6 per term: the denominator q_j(v_j) from its k-block partials, its
// inverse (one inversion per warp), the S dot products from their k-block
// partials, then the monomial coefficients through W.  Blocks of kFinB terms
// never straddle entries (pre counts blocks), so W sits in shared memory.
// kFinSplit warps share a block: the first inverts, all sum the partials of
// every kFinSplit-th right-hand side and compute every kFinSplit-th output.
__global__ void __launch_bounds__(kFinB * kFinSplit) k_b_finish_newton(const BDesc* __restrict__ Ds,
                                                                      const int64_t* __restrict__ pre_blk, int n,
                                                                      Mod M) {
  pdl_enter();
  extern __shared__ uint64_t fsm[];
  __shared__ uint64_t sh_inv[kFinB];
  __shared__ int sh_cnt[kFinSplit][kFinB];
  const int i = seg_of(pre_blk, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int S = D.S, Sn = D.Sn, s1 = Sn - S;   // s1 = 1: sample 0 is given (c0)
  uint64_t* W = fsm;
  uint64_t* num = fsm + Sn * Sn;
  for (int idx = threadIdx.x; idx < Sn * Sn; idx += blockDim.x) W[idx] = D.invd[idx];
  const int t = threadIdx.x & (kFinB - 1), q = threadIdx.x / kFinB;   // term, warp of the split
  const int64_t j = (blockIdx.x - pre_blk[i]) * kFinB + t;
  const bool active = j < D.T;
  if (q == 0) {
    uint64_t den = 1, mult = 1;
    if (active) {
      den = root_den(D, j, D.v[j], M, mult);
      if (den == 0) atomicOr(D.status, ST_ZERO_DEN);
    }
    sh_inv[t] = mul_mod(warp_batch_inverse(den, M), mult, M);
  }
  if (active) {
    // sum of the k-block partials, right-hand sides q, q + kFinSplit, .. per warp
    uint64_t* nm = num + t + s1 * kFinB;
    for (int s = q; s < S; s += kFinSplit) {
      uint64_t acc = D.part[(int64_t)s * D.T + j];
      for (int kb = 1; kb < D.NB; kb++) acc = add_mod(acc, D.part[((int64_t)kb * S + s) * D.T + j], M);
      nm[s * kFinB] = acc;
    }
  }
  __syncthreads();
  const uint64_t inv = sh_inv[t];
  if (active && s1) {
    // the given solution at sample 0, the solved ones scaled by the inverse
    uint64_t* nm = num + t;
    if (q == 0) nm[0] = D.c0[j];
    for (int s = 1 + q; s < Sn; s += kFinSplit) nm[s * kFinB] = mul_mod(nm[s * kFinB], inv, M);
  }
  __syncthreads();
  // the monomial coefficients e = q, q + kFinSplit, .. of each term
  sh_cnt[q][t] = active ? newton_apply(Sn, W, num + t, kFinB, s1 ? 1 : inv, D.g + j, D.T, M, q, kFinSplit) : 0;
  __syncthreads();
  if (q == 0) {
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < kFinSplit; r++) cnt += sh_cnt[r][t];
    if (active) D.cnt[j] = cnt;
    // nonzero coefficients of this block of terms, for the compaction
    int64_t total = cnt;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(0xffffffffu, total, off);
    if (t == 0) D.bsum[blockIdx.x - pre_blk[i]] = total;
  }
}

__global__ void __launch_bounds__(256) k_b_finish_solve(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre,
                                                        int n, Mod M) {
  pdl_enter();
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = x < pre[n];
  const int i = active ? seg_of(pre, n, x) : 0;
  const BDesc& D = Ds[i];
  const int64_t j = x - pre[i];
  uint64_t den = 1, mult = 1;
  if (active) {
    den = root_den(D, j, D.v[j], M, mult);
    if (den == 0) atomicOr(D.status, ST_ZERO_DEN);
  }
  const uint64_t inv = mul_mod(warp_batch_inverse(den, M), mult, M);
  if (!active) return;
  for (int s = 0; s < D.S; s++) {
    // the NB partials of one right-hand side, loaded eight at a time
    uint64_t num = 0;
    for (int k0 = 0; k0 < D.NB; k0 += 8) {
      uint64_t x[8];
#pragma unroll
      for (int q = 0; q < 8; q++) x[q] = k0 + q < D.NB ? D.part[((int64_t)(k0 + q) * D.S + s) * D.T + j] : 0;
#pragma unroll
      for (int q = 0; q < 8; q++) num = add_mod(num, x[q], M);
    }
    D.c[(int64_t)s * D.ldc + j] = mul_mod(num, inv, M);
  }
}

// ---- a6: compaction ---------------------------------------------------------------

constexpr int kScanB = 1024;   // width of the block-offset scan
constexpr int kCompB = kFinB;  // terms per compaction block (the finish kernel's blocks)

// Exclusive offsets of the blocks' nonzero counts, one CTA per entry.
__global__ void __launch_bounds__(kScanB) k_b_scan(const BDesc* __restrict__ Ds) {
  pdl_enter();
  __shared__ int64_t sh[33];
  const BDesc& D = Ds[blockIdx.x];
  if (D.mode != 0) return;
  const int64_t nb = (D.T + kCompB - 1) / kCompB;
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanB) {
    const int64_t t = base + threadIdx.x;
    int64_t total;
    const int64_t ex = block_exclusive_scan(t < nb ? D.bsum[t] : 0, sh, total);
    if (t < nb) D.bsum[t] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *D.out_count = carry;
}

// The new skeleton: the nonzero coefficients of every term j in order of j,
// then of the power s of x_k.  One block per kCompB terms and kFinSplit warps:
// the first warp takes a term per lane (its nonzero mask and offset), then
// all threads walk the block's output slots, so consecutive threads write
// consecutive outputs.
__global__ void __launch_bounds__(kCompB * kFinSplit) k_b_scatter(const BDesc* __restrict__ Ds,
                                                                  const int64_t* __restrict__ pre_blk, int n) {
  pdl_enter();
  __shared__ int64_t sh[33];
  __shared__ int32_t offs[kCompB];
  __shared__ uint64_t masks[kCompB];
  const int i = seg_of(pre_blk, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int64_t blk = blockIdx.x - pre_blk[i];
  const int64_t j0 = blk * kCompB, j = j0 + threadIdx.x;
  const int S = D.Sn;
  uint64_t mask = 0;
  if (threadIdx.x < kCompB && j < D.T)
    for (int s = 0; s < S; s++)
      if (D.g[(int64_t)s * D.T + j] != 0) mask |= 1ull << s;
  int64_t total;
  const int64_t ex = block_exclusive_scan(__popcll(mask), sh, total);
  if (threadIdx.x < kCompB) {
    offs[threadIdx.x] = (int32_t)ex;
    masks[threadIdx.x] = mask;
  }
  __syncthreads();
  const int64_t base = D.bsum[blk];
  const int nv = D.nv, k = D.k;
  for (int slot = threadIdx.x; slot < total; slot += blockDim.x) {
    int lo = 0, hi = kCompB - 1;   // the term owning this slot: largest t with offs[t] <= slot
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= slot) lo = mid;
      else hi = mid - 1;
    }
    // the (slot - offs[lo])-th set bit of the term's mask
    const uint64_t m = masks[lo];
    const int r = slot - offs[lo];
    const unsigned mlo = (unsigned)m, mhi = (unsigned)(m >> 32);
    const int nlo = __popc(mlo);
    const int s = r < nlo ? (int)__fns(mlo, 0, r + 1) : 32 + (int)__fns(mhi, 0, r - nlo + 1);
    const int64_t jj = j0 + lo, o = base + slot;
    if (o < D.out_cap) {
      const uint8_t* e = D.exps + jj * nv;
      uint8_t* oe = D.out_exps + o * nv;
      for (int q = 0; q < nv; q++) oe[q] = q < k ? e[q] : 0;
      oe[k] = (uint8_t)s;
      D.out_coef[o] = D.g[(int64_t)s * D.T + jj];
    }
  }
}

// ---- host side ---------------------------------------------------------------------

static int tree_levels(int64_t T) {
  int l = 0;
  while ((1ll << l) < T) l++;
  return l;
}

static void push_prefix(std::vector<int64_t>& all, const std::vector<int64_t>& counts, size_t& off) {
  off = all.size();
  int64_t s = 0;
  for (int64_t c : counts) {
    all.push_back(s);
    s += c;
  }
  all.push_back(s);
}

// Plans, prefix tables and work lists of a batch (host side).
struct Prepared {
  std::vector<StepDims> plan;
  std::vector<int64_t> pre;
  size_t o_hash = 0, o_roots = 0, o_leaf = 0, o_carry = 0, o_nblk = 0;
  std::vector<size_t> o_lvl;
  std::vector<int> tiles_used;        // solve instances: tile * 16 + consumer groups
  std::vector<std::vector<int4>> work;
  std::vector<char> fast;             // entries solved by the O(T log^2 T) path
  int kmax = 0, smax = 0, lmax = 0, mode = 0;
  size_t ws_bytes = 0, table_bytes = 0, fast_bytes = 0;
  int nfast = 0, fstreams = 0;        // fast entries, concurrent streams for them (0: the call's stream)
  size_t fast_slot = 0;               // workspace of one fast stream
};

// A batch with several O(T log^2 T) entries, or such entries beside O(T^2)
// ones, runs them on up to kFastStreams streams of their own (each with its
// workspace slot, entries round-robin) from the anchor values on, beside the
// tree, carries and ring solve of the others, and joins them before the
// finish; a lone fast entry runs on the call's stream.
constexpr int kFastStreams = 4;

// The auxiliary stream and events of fast-solve slot j (created on first
// use, the stream with the device's greatest priority: it carries the
// solve's critical branch); false when they cannot be had (the solve then
// runs on one stream).
static bool fast_aux(zr_ctx* ctx, int j) {
  int least = 0, greatest = 0;
  if (!ctx->faux[j] && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) greatest = 0;
  if (!ctx->faux[j] && cudaStreamCreateWithPriority(&ctx->faux[j], cudaStreamNonBlocking, greatest) != cudaSuccess) {
    ctx->faux[j] = nullptr;
    return false;
  }
  if (!ctx->faux_fork[j] && cudaEventCreateWithFlags(&ctx->faux_fork[j], cudaEventDisableTiming) != cudaSuccess) {
    ctx->faux_fork[j] = nullptr;
    return false;
  }
  if (!ctx->faux_join[j] && cudaEventCreateWithFlags(&ctx->faux_join[j], cudaEventDisableTiming) != cudaSuccess) {
    ctx->faux_join[j] = nullptr;
    return false;
  }
  return true;
}

static bool prepare(const zr_ctx* ctx, const BatchItem* items, int n, Prepared& P) {
  P.mode = items[0].mode;
  P.plan.resize(n);
  P.fast.assign(n, 0);
  for (int i = 0; i < n; i++) {
    const BatchItem& it = items[i];
    if (it.mode != P.mode) return false;
    P.fast[i] = use_fast_solve(ctx, it.T, it.solve_S(), n) ? 1 : 0;
    if (P.fast[i]) {
      // one k-block: the finish kernels read the numerators and M'(v_j) as a
      // single block's partials
      StepDims D;
      D.T = it.T;
      D.S = it.solve_S();
      D.NB = 1;
      D.BK = it.T;
      D.s_tile = 2;
      P.plan[i] = D;
      P.fast_slot = std::max(P.fast_slot, (fast_ws_need(it.T, it.solve_S() + 1) + 255) & ~(size_t)255);
      P.nfast++;
    } else {
      P.plan[i] = plan_step(ctx, it.T, it.solve_S());
      P.lmax = std::max(P.lmax, tree_levels(it.T));
    }
    P.kmax = std::max(P.kmax, it.k);
    P.smax = std::max(P.smax, it.S);
  }
  Carver m0(nullptr);
  for (int i = 0; i < n; i++) carve_step(m0, items[i].T, items[i].S, items[i].k, P.plan[i], items[i].solve_S());
  P.ws_bytes = m0.off;
  std::vector<int64_t> c_hash(n), c_roots(n), c_leaf(n), c_carry(n), c_nblk(n);
  for (int i = 0; i < n; i++) {
    const int64_t T = items[i].T;
    c_hash[i] = T > 0 ? (int64_t)hash_slots(T) : 0;
    c_roots[i] = T;
    c_leaf[i] = P.fast[i] ? 0 : (T + (1 << kTreeL1) - 1) >> kTreeL1;
    c_nblk[i] = (T + kFinB - 1) / kFinB;
    c_carry[i] = (T > 0 && P.plan[i].NB > 1) ? (int64_t)((T + 255) / 256) * (P.plan[i].NB - 1) : 0;
  }
  push_prefix(P.pre, c_hash, P.o_hash);
  push_prefix(P.pre, c_roots, P.o_roots);
  push_prefix(P.pre, c_leaf, P.o_leaf);
  push_prefix(P.pre, c_carry, P.o_carry);
  push_prefix(P.pre, c_nblk, P.o_nblk);
  for (int l = kTreeL1; l < P.lmax; l++) {
    std::vector<int64_t> c(n);
    for (int i = 0; i < n; i++)
      c[i] = (!P.fast[i] && tree_levels(items[i].T) > l) ? (items[i].T + tree_tile(l) - 1) / tree_tile(l) : 0;
    size_t o;
    push_prefix(P.pre, c, o);
    P.o_lvl.push_back(o);
  }
  for (int i = 0; i < n; i++) {
    if (items[i].T == 0 || P.fast[i]) continue;
    // one work list per (tile, consumer groups): the solve kernel instance
    const int tile = P.plan[i].s_tile, groups = (items[i].solve_S() + tile - 1) / tile;
    const int key = tile * 16 + groups;
    int w = (int)(std::find(P.tiles_used.begin(), P.tiles_used.end(), key) - P.tiles_used.begin());
    if (w == (int)P.tiles_used.size()) {
      P.tiles_used.push_back(key);
      P.work.emplace_back();
    }
    const int rt = solve_roots_per_item();
    const int rows = (int)((items[i].T + rt - 1) / rt);
    for (int kb = 0; kb < P.plan[i].NB; kb++)
      for (int r = 0; r < rows; r++) P.work[w].push_back(make_int4(i, r, kb, 0));
  }
  const std::vector<StepDims>& plan = P.plan;
  for (auto& wl : P.work)
    std::stable_sort(wl.begin(), wl.end(), [&](const int4& a, const int4& b) {
      return plan[a.x].BK * plan[a.x].S > plan[b.x].BK * plan[b.x].S;
    });
  P.table_bytes = sizeof(BDesc) * n + sizeof(int64_t) * P.pre.size();
  for (auto& wl : P.work) P.table_bytes += sizeof(int4) * wl.size() + 16;
  P.fstreams = (P.nfast >= 2 || (P.nfast >= 1 && P.nfast < n)) ? std::min(P.nfast, kFastStreams) : 0;
  P.fast_bytes = P.nfast ? P.fast_slot * (size_t)std::max(P.fstreams, 1) : 0;
  return true;
}

size_t batch_ws_need(const zr_ctx* ctx, const BatchItem* items, int n) {
  if (n <= 0) return 0;
  Prepared P;
  if (!prepare(ctx, items, n, P)) return 0;
  return P.ws_bytes + P.table_bytes + 512 + (P.fast_bytes ? P.fast_bytes + 256 : 0);
}

// A batch whose descriptor tables are on the device: everything launch_batch
// needs to enqueue (or to have captured) the kernels.
struct StagedBatch {
  Prepared P;
  int n = 0;
  const BDesc* dD = nullptr;
  const int64_t* dpre = nullptr;
  std::vector<const int4*> dwork;
  std::vector<int64_t*> zero_counts;   // out_count of entries with T = 0
  std::vector<BDesc> hD;               // host copy of the descriptors (the fast entries' pointers)
  char* fast_ws = nullptr;             // workspace of the fast entries: one slot per fast stream
};

// Plans the batch, carves its workspace at `ws` (batch_ws_need bytes) and
// copies the descriptor tables to the device on `st` (through the context's
// pinned staging buffer).
static zr_status stage_batch(zr_ctx* ctx, const BatchItem* items, int n, uint32_t* status, cudaStream_t st, char* ws,
                             StagedBatch& SB) {
  Prepared& P = SB.P;
  SB.n = n;
  if (!prepare(ctx, items, n, P)) return set_err(ctx, ZR_ERR_INVALID_ARG, "batch mixes steps and systems");
  const std::vector<StepDims>& plan = P.plan;
  const std::vector<int64_t>& pre = P.pre;
  const std::vector<std::vector<int4>>& work = P.work;
  const size_t table_bytes = P.table_bytes;
  std::vector<BDesc> D(n);
  // carve for real
  Carver cv(ws);
  for (int i = 0; i < n; i++) {
    const BatchItem& it = items[i];
    StepWs w = carve_step(cv, it.T, it.S, it.k, plan[i], it.solve_S());
    const bool given0 = it.solve_S() != it.S;
    BDesc& d = D[i];
    memset(&d, 0, sizeof(d));
    d.T = it.T;
    d.S = it.solve_S();
    d.Sn = it.S;
    d.c0 = given0 ? it.c0 : nullptr;
    d.k = it.k;
    d.nv = it.nv;
    d.offset = it.offset;
    d.mode = it.mode;
    d.NB = plan[i].NB;
    d.BK = plan[i].BK;
    d.s_tile = plan[i].s_tile;
    d.nst = (d.S + plan[i].s_tile - 1) / plan[i].s_tile;   // consumer groups of the solve
    d.levels = P.fast[i] ? 0 : tree_levels(it.T);
    d.hmask = hash_slots(it.T) - 1;
    d.exps = it.exps;
    d.y = it.y;
    d.xs = it.xs;
    d.b = given0 ? it.b + it.ldb : it.b;   // the solved samples' rows
    d.ldb = it.ldb;
    d.tab = w.tab;
    d.v = it.mode == 1 ? const_cast<uint64_t*>(it.vin) : w.v;
    d.vp = w.vp;
    d.htab = w.htab;
    d.m = w.m;
    d.tmp = w.tmp;
    d.R = w.R;
    d.tpart = w.tpart;
    d.part = w.part;
    d.denp = w.denp;
    d.invd = w.invd;
    d.g = w.g;
    d.cnt = w.cnt;
    d.bsum = w.bsum;
    d.out_exps = it.out_exps;
    d.out_coef = it.out_coef;
    d.out_cap = it.out_cap;
    d.out_count = it.out_count;
    d.c = it.c;
    d.ldc = it.ldc;
    d.status = it.status ? it.status : status;
  }
  // stage the tables in pinned memory, then one copy
  char* dtab = cv.take<char>(table_bytes + 256);
  SB.fast_ws = P.fast_bytes ? cv.take<char>(P.fast_bytes) : nullptr;
  if (ctx->stage_event) cudaEventSynchronize(ctx->stage_event);
  if (ctx->h_stage_cap < table_bytes) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    if (cudaMallocHost(&ctx->h_stage, table_bytes * 2) != cudaSuccess)
      return set_err(ctx, ZR_ERR_OOM, "pinned staging buffer");
    ctx->h_stage_cap = table_bytes * 2;
  }
  char* hs = static_cast<char*>(ctx->h_stage);
  size_t pos = 0;
  memcpy(hs + pos, D.data(), sizeof(BDesc) * n);
  const BDesc* dD = reinterpret_cast<const BDesc*>(dtab + pos);
  pos += sizeof(BDesc) * n;
  memcpy(hs + pos, pre.data(), sizeof(int64_t) * pre.size());
  const int64_t* dpre = reinterpret_cast<const int64_t*>(dtab + pos);
  pos += sizeof(int64_t) * pre.size();
  std::vector<const int4*> dwork(work.size());
  for (size_t w = 0; w < work.size(); w++) {
    pos = (pos + 15) & ~(size_t)15;
    memcpy(hs + pos, work[w].data(), sizeof(int4) * work[w].size());
    dwork[w] = reinterpret_cast<const int4*>(dtab + pos);
    pos += sizeof(int4) * work[w].size();
  }
  cudaError_t e = cudaMemcpyAsync(dtab, hs, pos, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "batch tables");
  if (!ctx->stage_event) cudaEventCreateWithFlags(&ctx->stage_event, cudaEventDisableTiming);
  cudaEventRecord(ctx->stage_event, st);
  SB.dD = dD;
  SB.dpre = dpre;
  SB.dwork = dwork;
  SB.hD = D;
  SB.zero_counts.clear();
  for (int i = 0; i < n; i++)
    if (items[i].T == 0 && P.mode == 0 && items[i].out_count) SB.zero_counts.push_back(items[i].out_count);
  return ZR_OK;
}

// Shared-memory limits of the Newton kernels, set once per device.
static void configure_newton_kernels() {
  static DeviceOnce attr;
  attr.run([] {
    cudaFuncSetAttribute(k_b_newton_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(8 * newton_table_words(kNewtonMax)));
    cudaFuncSetAttribute(k_b_finish_newton, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)newton_smem(kNewtonMax, kFinB));
  });
}

// Enqueues the batch's kernels on `st` (capturable: no host synchronisation,
// no allocation).  `prof` records the profiler's phase events.
static zr_status launch_batch(zr_ctx* ctx, const StagedBatch& SB, cudaStream_t st, bool prof) {
  const Prepared& P = SB.P;
  const int n = SB.n;
  const Mod& M = ctx->M;
  const int mode = P.mode, kmax = P.kmax, smax = P.smax, lmax = P.lmax;
  const std::vector<int64_t>& pre = P.pre;
  const size_t o_hash = P.o_hash, o_roots = P.o_roots, o_leaf = P.o_leaf, o_carry = P.o_carry, o_nblk = P.o_nblk;
  const std::vector<size_t>& o_lvl = P.o_lvl;
  const std::vector<int>& tiles_used = P.tiles_used;
  const std::vector<std::vector<int4>>& work = P.work;
  const BDesc* dD = SB.dD;
  const int64_t* dpre = SB.dpre;
  const std::vector<const int4*>& dwork = SB.dwork;
  auto mark = [&]() -> cudaEvent_t { return prof ? prof_mark(ctx, st) : nullptr; };

  const int64_t nroots = pre[o_roots + n], nhash = pre[o_hash + n], nleaf = pre[o_leaf + n];
  const int64_t ncarry = pre[o_carry + n];
  // entries with T = 0 report an empty skeleton
  for (int64_t* c : SB.zero_counts) cudaMemsetAsync(c, 0, 8, st);
  // Newton's matrix W depends only on the samples: build it on the side
  // stream while the tree, carries and solve run (joined before the finish)
  bool side = false;
  if (mode == 0 && nroots) {
    if (!ctx->side) cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (!ctx->ev_fork) cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (!ctx->ev_join) cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (ctx->side && ctx->ev_fork && ctx->ev_join) {
      configure_newton_kernels();
      cudaEventRecord(ctx->ev_fork, st);
      cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
      launch_k(k_b_newton_table, n, kNewtonThreads, 8 * (size_t)newton_table_words(smax), ctx->side, dD, M);
      note_launch();
      cudaEventRecord(ctx->ev_join, ctx->side);
      side = true;
    }
  }
  cudaEvent_t e0 = mark();
  // a2
  // the step's own kernels are programmatic dependent launches too (each
  // starts with pdl_enter), like the O(T log^2 T) path's
  if (nhash) { launch_k(k_b_fill_hash, cdiv(nhash, 256), 256, 0, st, dD, dpre + o_hash, n); note_launch(); }
  if (mode == 0 && kmax > 0) { launch_k(k_b_powtab, dim3(kmax, n), kPowTab, 0, st, dD, M); note_launch(); }
  if (nroots) { launch_k(k_b_anchor, cdiv(nroots, 256), 256, 0, st, dD, dpre + o_roots, n, M); note_launch(); }
  cudaEvent_t e1 = mark();
  // the O(T log^2 T) entries need only the anchor values: with several of
  // them, or beside O(T^2) entries, they start here on their own streams
  int fs_used = 0;
  if (P.fstreams > 0) {
    int64_t tmax = 0;
    for (int i = 0; i < n; i++)
      if (P.fast[i]) tmax = std::max(tmax, SB.hD[i].T);
    if (zr_status r = fast_tables_for(ctx, tmax, st)) return r;
    bool ok = true;
    if (!ctx->fev_fork) ok = cudaEventCreateWithFlags(&ctx->fev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; ok && j < P.fstreams; j++) {
      if (!ctx->fstream[j]) ok = cudaStreamCreateWithFlags(&ctx->fstream[j], cudaStreamNonBlocking) == cudaSuccess;
      if (ok && !ctx->fev_join[j]) ok = cudaEventCreateWithFlags(&ctx->fev_join[j], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) return cuda_err(ctx, cudaErrorMemoryAllocation, "fast streams");
    cudaEventRecord(ctx->fev_fork, st);
    for (int j = 0; j < P.fstreams; j++) cudaStreamWaitEvent(ctx->fstream[j], ctx->fev_fork, 0);
    int k = 0;
    for (int i = 0; i < n; i++) {
      if (!P.fast[i]) continue;
      const int j = k++ % P.fstreams;
      const BDesc& d = SB.hD[i];
      const bool ax = fast_aux(ctx, j);
      zr_status r = fast_solve_enqueue(ctx, d.T, d.S, d.v, d.vp, d.b, d.ldb, d.part, d.denp,
                                       SB.fast_ws + (size_t)j * P.fast_slot, ctx->fstream[j],
                                       ax ? ctx->faux[j] : nullptr, ctx->faux_fork[j], ctx->faux_join[j]);
      if (r) return r;
    }
    fs_used = std::min(k, P.fstreams);
    for (int j = 0; j < fs_used; j++) cudaEventRecord(ctx->fev_join[j], ctx->fstream[j]);
  }
  // a3
  if (nleaf) { k_b_tree_leaf<<<(unsigned)nleaf, 1 << kTreeL1, 0, st>>>(dD, dpre + o_leaf, n, M); note_launch(); }
  for (int l = kTreeL1; l < lmax; l++) {
    const size_t o = o_lvl[l - kTreeL1];
    const int64_t nt = pre[o + n];
    if (!nt) continue;
    // split the inner range when the level has fewer than ~4 tiles per SM,
    // within every participating entry's partial-sum capacity
    const int64_t want = 4ll * (ctx->sms ? ctx->sms : 152);
    int split = (int)((want + nt - 1) / nt);
    for (int i = 0; i < n; i++)
      if (!P.fast[i] && tree_levels(P.plan[i].T) > l) split = std::min(split, (int)tree_split_max(P.plan[i].T));
    // and keep at least 128 inner terms per split: below that the combine
    // launch costs more than the shorter serial work saves
    split = std::min(split, (int)std::max<int64_t>(1, (1ll << l) / 128));
    split = std::max(1, std::min(split, 16));
    {
      k_b_tree_conv<<<dim3((unsigned)nt, (unsigned)split), tree_tile(l) / kTR, 0, st>>>(dD, dpre + o, n, l, split, M);
      note_launch();
    }
    if (split > 1) {
      k_b_tree_combine<<<cdiv(nroots, 256), 256, 0, st>>>(dD, dpre + o_roots, n, l, split, M);
      note_launch();
    }
  }
  cudaEvent_t e2 = mark();
  // a4 + a5
  if (ncarry) launch_b_carry(dD, dpre + o_carry, n, ncarry, M, st);
  cudaEvent_t e3 = mark();
  for (size_t w = 0; w < work.size(); w++)
    if (!launch_b_solve(tiles_used[w] / 16, tiles_used[w] % 16, dD, dwork[w], (int)work[w].size(),
                        ctx->solve_persistent ? (ctx->sms ? ctx->sms : 152) : 0, M, st))
      return set_err(ctx, ZR_ERR_INVALID_ARG, "no solve kernel for this launch plan");
  cudaEvent_t e4 = mark();
  // entries of the O(T log^2 T) solve: numerators and M'(v_j) into the
  // single-block partials the finish reads (on this stream, or joined here
  // from their own streams: the phase is then the wait for them)
  if (P.fstreams == 0)
    for (int i = 0; i < n; i++) {
      if (!P.fast[i]) continue;
      const BDesc& d = SB.hD[i];
      const bool ax = fast_aux(ctx, 4);
      zr_status r = fast_solve_enqueue(ctx, d.T, d.S, d.v, d.vp, d.b, d.ldb, d.part, d.denp, SB.fast_ws, st,
                                       ax ? ctx->faux[4] : nullptr, ctx->faux_fork[4], ctx->faux_join[4]);
      if (r) return r;
    }
  for (int j = 0; j < fs_used; j++) cudaStreamWaitEvent(st, ctx->fev_join[j], 0);
  cudaEvent_t e4f = mark();
  // a6 (or the plain finish of a system)
  if (nroots) {
    if (mode == 0) {
      configure_newton_kernels();
      if (side) cudaStreamWaitEvent(st, ctx->ev_join, 0);   // W of every entry (forked above)
      else {
        launch_k(k_b_newton_table, n, kNewtonThreads, 8 * (size_t)newton_table_words(smax), st, dD, M);
        note_launch();
      }
      const int64_t nblk = pre[o_nblk + n];
      {
        launch_k(k_b_finish_newton, (unsigned)nblk, kFinB * kFinSplit, newton_smem(smax, kFinB), st, dD,
                 dpre + o_nblk, n, M);
        note_launch();
      }
    } else {
      { launch_k(k_b_finish_solve, cdiv(nroots, 256), 256, 0, st, dD, dpre + o_roots, n, M); note_launch(); }
    }
  }
  cudaEvent_t e5 = mark();
  if (mode == 0 && nroots) {
    { launch_k(k_b_scan, n, kScanB, 0, st, dD); note_launch(); }
    {
      launch_k(k_b_scatter, (unsigned)pre[o_nblk + n], kCompB * kFinSplit, 0, st, dD, dpre + o_nblk, n);
      note_launch();
    }
  }
  cudaEvent_t e6 = mark();
  prof_add(ctx, PH_ANCHOR, e0, e1);
  prof_add(ctx, PH_MASTER, e1, e2);
  prof_add(ctx, PH_CARRY, e2, e3);
  prof_add(ctx, PH_SOLVE, e3, e4);
  prof_add(ctx, PH_FAST, e4, e4f);
  prof_add(ctx, PH_NEWTON, e4f, e5);
  prof_add(ctx, PH_COMPACT, e5, e6);
  return cuda_err(ctx, cudaGetLastError(), "batch launch");
}

zr_status run_batch(zr_ctx* ctx, const BatchItem* items, int n, uint32_t* status, cudaStream_t st, size_t base) {
  if (n <= 0) return ZR_OK;
  const size_t need = batch_ws_need(ctx, items, n);
  zr_status r = ensure_ws(ctx, base + need, st);
  if (r) return r;
  StagedBatch SB;
  r = stage_batch(ctx, items, n, status, st, ctx->ws + base, SB);
  if (r) return r;
  return launch_batch(ctx, SB, st, true);
}

// ---- captured batches (CUDA graphs) ----------------------------------------------

zr_status batch_graph_capture(zr_ctx* ctx, const BatchItem* items, int n, uint32_t* status, char* ws,
                              cudaStream_t st, cudaGraph_t* graph, uint64_t* launches) {
  StagedBatch SB;
  zr_status r = stage_batch(ctx, items, n, status, st, ws, SB);
  if (r) return r;
  // one uncaptured run first: the tables land, and every kernel's one-time
  // attribute setup happens outside the capture
  cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if ((r = launch_batch(ctx, SB, st, false))) return r;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "graph warm-up");
  cudaStream_t cs;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_err(ctx, e, "graph");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const uint64_t c0 = launch_count();
    cudaMemsetAsync(status, 0, sizeof(uint32_t), cs);
    r = launch_batch(ctx, SB, cs, false);
    *launches = launch_count() - c0;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && !r) *graph = g;
    else if (g) cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  if (r) return r;
  return cuda_err(ctx, e, "graph capture");
}

}  // namespace zr
