// zr_device.cuh -- device helpers shared by the step kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "zr_arith.cuh"
#include "zr_kernels.cuh"

namespace zr {

constexpr uint64_t kEmptySlot = ~0ull;

// Open-addressing node table (the distinctness check of the anchor values).
__device__ __forceinline__ uint64_t hash64(uint64_t x) {
  x ^= x >> 31;
  x *= 0x9E3779B97F4A7C15ull;
  return x ^ (x >> 29);
}

// Insert x into the open-addressing table; flags a duplicate.  Every probe
// sequence ends: the table has at least 2T slots and each thread inserts one key.
__device__ __forceinline__ void node_insert(uint64_t x, uint64_t* htab, uint64_t hmask, uint32_t* status) {
  uint64_t idx = hash64(x) & hmask;
  for (uint64_t probe = 0; probe <= hmask; probe++) {
    unsigned long long prev = atomicCAS((unsigned long long*)&htab[idx], (unsigned long long)kEmptySlot,
                                        (unsigned long long)x);
    if (prev == kEmptySlot) return;
    if (prev == x) { atomicOr(status, ST_DUP_NODE); return; }
    idx = (idx + 1) & hmask;
  }
  atomicOr(status, ST_HASH_FULL);
}

// Dot products of the product tree: a full 128-bit product per term.
__device__ __forceinline__ uint64_t conv_coef(const uint64_t* in, int po, int a, int b, int n, const Mod& M) {
  Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
  int ilo = n - b > 0 ? n - b : 0, ihi = n < a ? n : a;
  for (int i = ilo; i <= ihi; i++) {
    uint64_t Ai = (i < a) ? in[po + i] : 1;
    int jj = n - i;
    uint64_t Bj = (jj < b) ? in[po + a + jj] : 1;
    mac8(acc, lo32(Ai), hi32(Ai), lo32(Bj), hi32(Bj));
  }
  return acc8_value(acc, M);
}

// Inverse of d for every lane of a full warp; lanes with d = 0 get 0.
__device__ __forceinline__ uint64_t warp_batch_inverse(uint64_t d, const Mod& M) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint64_t x = d ? d : 1;
  uint64_t pre = x, suf = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint64_t t = __shfl_up_sync(FULL, pre, off);
    if (lane >= off) pre = mul_mod(pre, t, M);
    uint64_t w = __shfl_down_sync(FULL, suf, off);
    if (lane + off < 32) suf = mul_mod(suf, w, M);
  }
  const uint64_t total = __shfl_sync(FULL, pre, 31);
  const uint64_t inv_total = inv_mod(total, M);
  uint64_t ep = __shfl_up_sync(FULL, pre, 1);
  uint64_t es = __shfl_down_sync(FULL, suf, 1);
  if (lane == 0) ep = 1;
  if (lane == 31) es = 1;
  uint64_t r = mul_mod(mul_mod(inv_total, ep, M), es, M);
  return d ? r : 0;
}

// ---- Newton interpolation on shared nodes (Introduction, the Newton formula) -----
//
// Every term of a step is interpolated on the same S nodes x_0..x_{S-1}, so
// the map from the S values to the S monomial coefficients is one S x S
// matrix W shared by all terms.  Column s of W is what Newton's method gives
// for the unit vector e_s: the divided-difference table, then the nested
// expansion of the Newton form into powers of z.  Applying W to a term's
// values is S^2 independent multiply-accumulates with one reduction per
// coefficient, instead of a chain of S^2 dependent modular products.

constexpr int kNewtonMax = 64;   // largest point count

// W for the nodes xs_g (device, S <= kNewtonMax) by one block of
// kNewtonThreads threads, all S columns at once: level by level, every
// (column, entry) pair of the divided-difference table and then of the nested
// expansion is updated by its own thread.  smem: newton_table_words(S) words.
// Equal nodes set ST_DUP_SAMPLE in *status (W is then meaningless).
constexpr int kNewtonThreads = 1024;
constexpr int kNewtonPairs = kNewtonMax * kNewtonMax / kNewtonThreads;   // pairs per thread
__host__ __device__ constexpr int newton_table_words(int S) { return 2 * S * S + S; }

__device__ inline void newton_table_block(int S, const uint64_t* __restrict__ xs_g, uint64_t* __restrict__ W,
                                          uint32_t* status, uint64_t* smem, const Mod& M) {
  uint64_t* xs = smem;
  uint64_t* A = smem + S;        // A[s * S + t]: column s's divided differences
  uint64_t* B = A + S * S;       // B[l * S + t] = 1 / (x_t - x_{t-l}), then the expansion cf[s * S + e]
  const int n2 = S * S, tid = threadIdx.x;
  for (int i = tid; i < S; i += kNewtonThreads) xs[i] = xs_g[i];
  __syncthreads();
  for (int idx = tid; idx < n2; idx += kNewtonThreads) {
    const int l = idx / S, t = idx - l * S;
    uint64_t r = 0;
    if (l >= 1 && t >= l) {
      const uint64_t d = sub_mod(xs[t], xs[t - l], M);
      if (d == 0) atomicOr(status, ST_DUP_SAMPLE);
      r = inv_mod(d, M);
    }
    B[idx] = r;
    A[idx] = l == t ? 1 : 0;     // column l is the unit vector e_l
  }
  __syncthreads();
  uint64_t nw[kNewtonPairs];
  // divided differences: level l replaces a_t by (a_t - a_{t-1}) / (x_t - x_{t-l}), t >= l
  for (int l = 1; l < S; l++) {
#pragma unroll
    for (int q = 0; q < kNewtonPairs; q++) {
      const int idx = tid + q * kNewtonThreads, t = idx % S;
      if (idx < n2 && t >= l) nw[q] = mul_mod(sub_mod(A[idx], A[idx - 1], M), B[l * S + t], M);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kNewtonPairs; q++) {
      const int idx = tid + q * kNewtonThreads, t = idx % S;
      if (idx < n2 && t >= l) A[idx] = nw[q];
    }
    __syncthreads();
  }
  // nested expansion, innermost bracket first: cf <- cf (z - x_l) + a_l
  for (int idx = tid; idx < n2; idx += kNewtonThreads) {
    const int s = idx / S, e = idx - s * S;
    B[idx] = e == 0 ? A[s * S + S - 1] : 0;
  }
  __syncthreads();
  for (int l = S - 2; l >= 0; l--) {
    const uint64_t xl = xs[l];
#pragma unroll
    for (int q = 0; q < kNewtonPairs; q++) {
      const int idx = tid + q * kNewtonThreads, s = idx / S, e = idx - s * S;
      if (idx < n2 && e <= S - 1 - l)
        nw[q] = sub_mod(e == 0 ? A[s * S + l] : B[idx - 1], mul_mod(xl, B[idx], M), M);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kNewtonPairs; q++) {
      const int idx = tid + q * kNewtonThreads, e = idx % S;
      if (idx < n2 && e <= S - 1 - l) B[idx] = nw[q];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < n2; idx += kNewtonThreads) {
    const int s = idx / S, e = idx - s * S;
    W[e * S + s] = B[idx];
  }
}

// out[e * ld] = scale * sum_s W[e][s] val[s * stride] for e < S (W and val in
// shared memory, val canonical); returns how many of them are nonzero.
__device__ inline int newton_apply(int S, const uint64_t* W, const uint64_t* val, int stride, uint64_t scale,
                                   uint64_t* out, int64_t ld, const Mod& M, int e_first = 0, int e_step = 1) {
  int cnt = 0;
  if (e_step != 1) {
    // the outputs e_first, e_first + e_step, ... only
    for (int e = e_first; e < S; e += e_step) {
      Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
      const uint64_t* w = W + (int64_t)e * S;
      for (int s = 0; s < S; s++) {
        const uint64_t x = val[s * stride], y = w[s];
        mac8(acc, lo32(x), hi32(x), lo32(y), hi32(y));
      }
      const uint64_t g = mul_mod(acc8_value(acc, M), scale, M);
      out[(int64_t)e * ld] = g;
      cnt += g != 0;
    }
    return cnt;
  }
  for (int e0 = 0; e0 < S; e0 += 4) {
    Acc8 acc[4];
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t* w0 = W + (e0 + 0 < S ? e0 + 0 : S - 1) * S;
    const uint64_t* w1 = W + (e0 + 1 < S ? e0 + 1 : S - 1) * S;
    const uint64_t* w2 = W + (e0 + 2 < S ? e0 + 2 : S - 1) * S;
    const uint64_t* w3 = W + (e0 + 3 < S ? e0 + 3 : S - 1) * S;
    for (int s = 0; s < S; s++) {
      const uint64_t x = val[s * stride];
      const uint32_t x0 = lo32(x), x1 = hi32(x);
      uint64_t w = w0[s];
      mac8(acc[0], x0, x1, lo32(w), hi32(w));
      w = w1[s];
      mac8(acc[1], x0, x1, lo32(w), hi32(w));
      w = w2[s];
      mac8(acc[2], x0, x1, lo32(w), hi32(w));
      w = w3[s];
      mac8(acc[3], x0, x1, lo32(w), hi32(w));
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (e0 + q < S) {
        const uint64_t g = mul_mod(acc8_value(acc[q], M), scale, M);
        out[(int64_t)(e0 + q) * ld] = g;
        cnt += g != 0;
      }
  }
  return cnt;
}

// Exclusive scan over a CTA (blockDim.x a multiple of 32, at most 1024);
// sh holds 33 words; every thread of the CTA must call it.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t* sh, int64_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int64_t s = lane < nw ? sh[lane] : 0;
    int64_t si = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, si, off);
      if (lane >= off) si += t;
    }
    sh[lane] = si - s;          // exclusive prefix of warp totals
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  total = sh[32];
  const int64_t r = incl - x + sh[w];
  __syncthreads();              // sh may be reused right after
  return r;
}

// Segment of a flattened index: the largest i < n with pre[i] <= x.
__device__ __forceinline__ int seg_of(const int64_t* __restrict__ pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace zr
