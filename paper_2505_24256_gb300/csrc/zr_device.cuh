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
struct Acc3 { uint64_t lo, hi, top; };
__device__ __forceinline__ void mac128(Acc3& a, uint64_t x, uint64_t y) {
  uint64_t h, l;
  mul128(x, y, h, l);
  a.lo += l;
  uint64_t hh = h + (a.lo < l);           // h <= 2^64 - 2: no overflow
  a.hi += hh;
  a.top += (a.hi < hh);
}
__device__ __forceinline__ uint64_t acc3_value(const Acc3& a, const Mod& M) {
  return reduce128(reduce128(a.top, a.hi, M), a.lo, M);   // top < p
}

// coefficient n of (A + z^a)(B + z^b), A at in[po..po+a), B at in[po+a..po+a+b)
__device__ __forceinline__ uint64_t conv_coef(const uint64_t* in, int po, int a, int b, int n, const Mod& M) {
  Acc3 acc = {0, 0, 0};
  int ilo = n - b > 0 ? n - b : 0, ihi = n < a ? n : a;
  for (int i = ilo; i <= ihi; i++) {
    uint64_t Ai = (i < a) ? in[po + i] : 1;
    int jj = n - i;
    uint64_t Bj = (jj < b) ? in[po + a + jj] : 1;
    mac128(acc, Ai, Bj);
  }
  return acc3_value(acc, M);
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

template <int SMAX>
__device__ __forceinline__ void newton_to_monomial(uint64_t (&a)[SMAX], int S, const uint64_t* __restrict__ xs,
                                                   const uint64_t* __restrict__ invd, const Mod& M) {
  // divided differences
#pragma unroll
  for (int l = 1; l < SMAX; l++) {
#pragma unroll
    for (int s = SMAX - 1; s >= l; s--) {
      if (l < S && s < S) a[s] = mul_mod(sub_mod(a[s], a[s - 1], M), __ldg(invd + l * S + s), M);
    }
  }
  // nested expansion, innermost bracket first: coef <- coef (z - x_l) + a_l
  uint64_t cf[SMAX];
#pragma unroll
  for (int e = 0; e < SMAX; e++) cf[e] = 0;
#pragma unroll
  for (int e = 0; e < SMAX; e++)
    if (e == S - 1) cf[0] = a[e];
#pragma unroll
  for (int l = SMAX - 2; l >= 0; l--) {
    if (l <= S - 2) {
      const uint64_t xl = __ldg(xs + l);
      // degree before this step: S - 2 - l
#pragma unroll
      for (int e = SMAX - 1; e >= 1; e--)
        if (e <= S - 1 - l) cf[e] = sub_mod(cf[e - 1], mul_mod(xl, cf[e], M), M);
      cf[0] = sub_mod(a[l], mul_mod(xl, cf[0], M), M);
    }
  }
#pragma unroll
  for (int e = 0; e < SMAX; e++) a[e] = cf[e];
}

// The same expansion with rolled loops (arrays in local memory) for the
// largest point count, to keep compile time bounded.
template <int SMAX>
__device__ __noinline__ void newton_to_monomial_rolled(uint64_t* a, int S, const uint64_t* __restrict__ xs,
                                                       const uint64_t* __restrict__ invd, const Mod& M) {
  for (int l = 1; l < S; l++)
    for (int s = S - 1; s >= l; s--) a[s] = mul_mod(sub_mod(a[s], a[s - 1], M), __ldg(invd + l * S + s), M);
  uint64_t cf[SMAX];
  for (int e = 0; e < S; e++) cf[e] = 0;
  cf[0] = a[S - 1];
  for (int l = S - 2; l >= 0; l--) {
    const uint64_t xl = __ldg(xs + l);
    for (int e = S - 1 - l; e >= 1; e--) cf[e] = sub_mod(cf[e - 1], mul_mod(xl, cf[e], M), M);
    cf[0] = sub_mod(a[l], mul_mod(xl, cf[0], M), M);
  }
  for (int e = 0; e < S; e++) a[e] = cf[e];
}

template <int SMAX>
__device__ __forceinline__ void newton_any(uint64_t (&a)[SMAX], int S, const uint64_t* __restrict__ xs,
                                           const uint64_t* __restrict__ invd, const Mod& M) {
  if constexpr (SMAX > 32) newton_to_monomial_rolled<SMAX>(a, S, xs, invd, M);
  else newton_to_monomial<SMAX>(a, S, xs, invd, M);
}

// Exclusive scan over a CTA of 1024 threads; sh holds 33 words.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t* sh, int64_t& total) {
  // blockDim.x == kScanB; sh holds 32 words
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t s = sh[lane];
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
  return incl - x + sh[w];
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
