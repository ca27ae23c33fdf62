// zr_fast.cu -- the transposed Vandermonde solve in O(T log^2 T).
//
// The step's systems sum_j c_j v_j^k = b_k (k < T) have the solution
// c_j = N(v_j) / M'(v_j) (Sec. 1; Sec. 2.2 writes it with the quotients
// q_j = M / (z - v_j): N(v_j) = <q_j, b>), where M = prod_j (z - v_j) and the
// generating function sum_k b_k z^(-k-1) = sum_j c_j / (z - v_j) = N / M.  The
// quadratic kernel forms every dot product <q_j, b>; this path evaluates N at
// all nodes with a subproduct tree instead (Bernstein's scaled remainder
// tree; the transposed multipoint evaluation of Bostan, Lecerf and Schost):
//
//   tree     M's factors are paired level by level: leaf blocks of 128 roots
//            (products in one CTA), then products of sibling polynomials by
//            transforms (zr_ntt.cuh).  The children's spectra are kept.
//   descent  b itself is the expansion of N / M to precision T.  A node P
//            with children L, R passes to L the expansion of (N mod P) R / P
//            truncated to deg L terms: X_L[m] = sum_{i <= deg R} r_i X_P[m+i],
//            a middle product computed as a cyclic convolution of size 2^l of
//            the reversed X_P with R, read backwards; likewise for R.
//   leaves   at a block P of 128 roots, X_P is the expansion of a
//            generating function whose numerator is N(v_j) / (M/P)(v_j) at
//            the block's roots; <q^P_j, X_P> with q^P_j = P / (z - v_j) gives
//            N(v_j) directly (the quadratic method on 128 roots).
//   denominators   M'(v_j) is the same evaluation with N = M', whose
//            expansion M'/M = sum_k (sum_j v_j^k) z^(-k-1) holds the power
//            sums of the nodes: summed directly (T^2 Shoup steps beside the
//            tree, up to kDirectPsMaxT unknowns; their row then joins the
//            right-hand sides' descent), else rev(M') / rev(M) mod z^T by
//            Newton's iteration for the power-series inverse (with a final
//            division step in one cluster up to 2^14).
//
// The results are the unique solution, bit-identical to the quadratic path.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "zr_device.cuh"
#include "zr_internal.h"
#include "zr_launch.cuh"
#include "zr_ntt.cuh"

namespace zr {

namespace {

inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
// Launches in this file are programmatic dependent launches (launch_k, every
// kernel starting with pdl_enter: zr_launch.cuh).

inline int ilog2(int64_t x) {
  int l = 0;
  while ((1ll << l) < x) l++;
  return l;
}

// ---- tables ----------------------------------------------------------------------

__device__ uint32_t pow32(uint32_t a, uint32_t e, uint32_t q) {
  uint64_t r = 1, x = a;
  while (e) {
    if (e & 1) r = r * x % q;
    x = x * x % q;
    e >>= 1;
  }
  return (uint32_t)r;
}

// tw[i N + k] = w_{2m}^brev(k - m), itw the inverse, m the largest power of
// two <= k (w_{2m} a primitive 2m-th root of unity mod q_i), with Shoup
// quotients.
__global__ void k_ntt_tables(int logN, NttConsts C, uint2* __restrict__ tw, uint2* __restrict__ itw) {
  pdl_enter();
  const int64_t N = 1ll << logN;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kNP * N) return;
  const int i = (int)(idx >> logN);
  const uint32_t k = (uint32_t)(idx & (N - 1));
  const uint32_t q = C.q[i];
  uint32_t w = 1, wi = 1;
  if (k >= 1) {
    const int lm = 31 - __clz(k);
    const uint32_t m = 1u << lm, j = k - m;
    const uint32_t e = lm ? (__brev(j) >> (32 - lm)) : 0;
    const uint32_t root = pow32(C.g[i], (q - 1) >> (lm + 1), q);
    w = pow32(root, e, q);
    wi = pow32(root, (2 * m - e) & (2 * m - 1), q);
  }
  tw[idx] = make_uint2(w, (uint32_t)(((uint64_t)w << 32) / q));
  itw[idx] = make_uint2(wi, (uint32_t)(((uint64_t)wi << 32) / q));
}

// ---- transforms --------------------------------------------------------------------
//
// Data: planes of 2^plane_log residues, plane k holding prime k mod 5; each
// plane is a run of transforms of size n = 2^logn.  Forward stage s (m = 2^s
// groups of distance t = n / 2^(s+1)) pairs j and j + t of group j / 2t with
// twiddle tw[m + group]; the inverse runs the stages in reverse order.
// Stages with t < kNttTile / 2 act within contiguous tiles of kNttTile
// elements (k_ntt_local); the first logn - 13 forward stages (last inverse
// ones) act within columns of stride 2^13 (k_ntt_cols).

// Shared-memory layout of the transform kernels: logical word x lives at
// sw(x), its bank bits XORed with bits of its 32-word row (a permutation
// within each row).  The register passes below touch words at strides 1, 8
// and multiples of 32; with this swizzle each of those warp accesses, and
// every run of 32 consecutive row-aligned words, hits 32 distinct banks.
__device__ __forceinline__ int sw(int x) { return x ^ (((x >> 5) & 7) | ((x >> 3) & 24)); }

// One pass of R <= 3 butterfly stages over groups of 2^R words held in
// registers (a radix-2^R pass).  Forward (Cooley-Tukey) stages s .. s+R-1:
// a group is the words a + i 2^u (u = lt - R + 1, lt = logn - 1 - s) of one
// block of 2^(lt+1); stage s+j pairs words 2^(R-1-j) apart with the twiddle
// of block (k 2^j + (i >> (R-j))) of that stage, k the group's block index.
// Inverse (Gentleman-Sande) stages s .. s-R+1: the words a + i 2^lt of one
// block of 2^(lt+R); stage s-j pairs words 2^j apart with the twiddle of
// block (K 2^(R-1-j) + (i >> (j+1))).  Logical word x (from off) sits at
// transform position (boff + x) mod 2^logn; prime_of(x) gives its prime.
// COLS: the buffer holds 2^cwl columns side by side instead (word x of
// column c at x 2^cwl + c, no swizzle), one transform each; consecutive
// threads take consecutive columns.
template <bool INV, int R, bool COLS, class PrimeOf>
__device__ __forceinline__ void radix_pass(uint32_t* sm, int off, int len, int logn, int s, uint32_t boff,
                                           const uint2* __restrict__ tw, int logN, const NttConsts& C,
                                           PrimeOf prime_of, int cwl) {
  constexpr int NR = 1 << R;
  const int lt = logn - 1 - s;
  const int u = INV ? lt : lt - R + 1;           // log2 of the stride within a group
  const int blog = INV ? lt + R : lt + 1;        // log2 of the group's block
  const uint32_t pmask = (1u << logn) - 1;
  const uint32_t m = 1u << s;
  for (int g0 = threadIdx.x; g0 < (len >> R); g0 += blockDim.x) {
    const int col = COLS ? (g0 & ((1 << cwl) - 1)) : 0;
    const int g = COLS ? (g0 >> cwl) : g0;
    const int a = ((g >> u) << blog) + (g & ((1 << u) - 1));
    const int prime = prime_of(a);
    const uint32_t q = C.q[prime];
    const uint32_t kb = ((boff + (uint32_t)a) & pmask) >> blog;
    const uint2* __restrict__ twp = tw + ((int64_t)prime << logN);
    uint2 w[NR - 1];
    int wo = 0;
#pragma unroll
    for (int j = 0; j < R; j++) {
      const int cnt = INV ? (1 << (R - 1 - j)) : (1 << j);
      const uint32_t base = INV ? (m >> j) + (kb << (R - 1 - j)) : (m << j) + (kb << j);
      // a stage's twiddles are contiguous and start at a multiple of their
      // count: pairs load as 16 bytes
      if (cnt == 1) {
        w[wo] = __ldg(&twp[base]);
      } else {
#pragma unroll
        for (int c = 0; c < cnt; c += 2) {
          const uint4 t2 = __ldg(reinterpret_cast<const uint4*>(twp + base + c));
          w[wo + c] = make_uint2(t2.x, t2.y);
          w[wo + c + 1] = make_uint2(t2.z, t2.w);
        }
      }
      wo += cnt;
    }
    // word addresses: for stride 1 the group lies in one row (sw(base) ^ i),
    // for strides of 256 and more the row bits of the swizzle are the
    // base's (sw(base) + (i << u)); strides 8 and 64 swizzle each word
    int at[NR];
    const int sb = sw(off + a);
#pragma unroll
    for (int i = 0; i < NR; i++)
      at[i] = COLS ? (((a + (i << u)) << cwl) + col)
                   : (u == 0 ? (sb ^ i) : (u >= 8 ? sb + (i << u) : sw(off + a + (i << u))));
    uint32_t x[NR];
#pragma unroll
    for (int i = 0; i < NR; i++) x[i] = sm[at[i]];
    wo = 0;
#pragma unroll
    for (int j = 0; j < R; j++) {
      const int hs = INV ? (1 << j) : (1 << (R - 1 - j));
#pragma unroll
      for (int i = 0; i < NR; i++)
        if (!(i & hs)) butterfly<INV>(x[i], x[i + hs], w[wo + (INV ? (i >> (j + 1)) : (i >> (R - j)))], q);
      wo += INV ? (1 << (R - 1 - j)) : (1 << j);
    }
#pragma unroll
    for (int i = 0; i < NR; i++) sm[at[i]] = x[i];
  }
}

// Stages s_lo .. logn-1 of the transforms in sm (logical words off ..
// off + len), forward in increasing or inverse in decreasing stage order:
// radix-8 passes, the leftover one or two stages as one pass on the
// largest strides.  Callers synchronise before; the last pass is followed
// by a barrier.
template <bool INV, bool COLS = false, class PrimeOf>
__device__ __forceinline__ void smem_stages(uint32_t* sm, int off, int len, int logn, int s_lo, uint32_t boff,
                                            const uint2* __restrict__ tw, int logN, const NttConsts& C,
                                            PrimeOf prime_of, int cwl = 0) {
  const int rem = (logn - s_lo) % 3;
  if (!INV) {
    int s = s_lo;
    if (rem == 1) {
      radix_pass<false, 1, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    } else if (rem == 2) {
      radix_pass<false, 2, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    }
    for (s += rem; s < logn; s += 3) {
      radix_pass<false, 3, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    }
  } else {
    int s = logn - 1;
    for (; s - 2 >= s_lo; s -= 3) {
      radix_pass<true, 3, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    }
    if (rem == 2) {
      radix_pass<true, 2, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    } else if (rem == 1) {
      radix_pass<true, 1, COLS>(sm, off, len, logn, s, boff, tw, logN, C, prime_of, cwl);
      __syncthreads();
    }
  }
}

// A tile of kNttTile elements starting at `base` (a multiple of kNttTile):
// the transform of an element is prime (base >> plane_log) + (pos >>
// plane_log) mod 5 (planes are powers of two, at most or at least a tile);
// the tile runs the stages s_lo .. logn-1 that stay inside it.
template <bool INV>
__global__ void __launch_bounds__(kNttThreads) k_ntt_local(uint32_t* __restrict__ data, int64_t total, int logn,
                                                           int plane_log, int s_lo, const uint2* __restrict__ tw,
                                                           int logN, NttConsts C) {
  pdl_enter();
  __shared__ __align__(16) uint32_t sm[kNttTile];
  const int64_t base = (int64_t)blockIdx.x * kNttTile;
  const int len = (int)((total - base) < kNttTile ? (total - base) : kNttTile);
  if ((len & 3) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(data + base);
    for (int e = threadIdx.x; e < (len >> 2); e += kNttThreads) {
      const uint4 v = src[e];
      sm[sw(4 * e)] = v.x;
      sm[sw(4 * e + 1)] = v.y;
      sm[sw(4 * e + 2)] = v.z;
      sm[sw(4 * e + 3)] = v.w;
    }
  } else {
    for (int e = threadIdx.x; e < len; e += kNttThreads) sm[sw(e)] = data[base + e];
  }
  __syncthreads();
  const int pb5 = (int)((base >> plane_log) % kNP);   // the tile's first plane, modulo 5
  const uint32_t boff = (uint32_t)(base & ((1ll << logn) - 1));   // the tile's offset within its transform
  if (plane_log >= kNttTileLog)
    smem_stages<INV>(sm, 0, len, logn, s_lo, boff, tw, logN, C, [=](int) { return pb5; });
  else
    smem_stages<INV>(sm, 0, len, logn, s_lo, boff, tw, logN, C,
                     [=](int x) { return (pb5 + (x >> plane_log)) % kNP; });
  if ((len & 3) == 0) {
    uint4* dst = reinterpret_cast<uint4*>(data + base);
    for (int e = threadIdx.x; e < (len >> 2); e += kNttThreads)
      dst[e] = make_uint4(sm[sw(4 * e)], sm[sw(4 * e + 1)], sm[sw(4 * e + 2)], sm[sw(4 * e + 3)]);
  } else {
    for (int e = threadIdx.x; e < len; e += kNttThreads) data[base + e] = sm[sw(e)];
  }
}

// The first L1 = logn - 13 forward stages (the last inverse ones) of a
// transform larger than a tile pair words 2^13 or more apart.  A CTA takes
// 2^(13 - L1) adjacent columns of the transform's 2^L1 rows of 2^13 words:
// stage s of the whole transform acts on each column as stage s of a
// transform of size 2^L1, twiddles included, run as radix passes with
// consecutive threads on consecutive columns.
template <bool INV>
__global__ void __launch_bounds__(kNttThreads) k_ntt_cols(uint32_t* __restrict__ data, int logn, int plane_log, int L1,
                                                          const uint2* __restrict__ tw, int logN, NttConsts C) {
  pdl_enter();
  __shared__ uint32_t sm[kNttTile];
  const int cwl = kNttTileLog - L1, CW = 1 << cwl;
  const int64_t tbase = (int64_t)(blockIdx.x >> L1) << logn;
  const int jlo0 = (blockIdx.x & ((1 << L1) - 1)) * CW;
  for (int e = threadIdx.x; e < kNttTile; e += kNttThreads) {
    const int h = e >> cwl, c = e & (CW - 1);
    sm[e] = data[tbase + ((int64_t)h << kNttTileLog) + jlo0 + c];
  }
  __syncthreads();
  const int prime = (int)((tbase >> plane_log) % kNP);
  smem_stages<INV, true>(sm, 0, kNttTile, L1, 0, 0u, tw, logN, C, [=](int) { return prime; }, cwl);
  for (int e = threadIdx.x; e < kNttTile; e += kNttThreads) {
    const int h = e >> cwl, c = e & (CW - 1);
    data[tbase + ((int64_t)h << kNttTileLog) + jlo0 + c] = sm[e];
  }
}

// ---- loads, products, Chinese remaindering ---------------------------------------

// Tree level l (nodes of size n = 2^l, children of size h = n/2): every child
// c of node P as a full monic polynomial of its degree d_c (coefficients from
// the level below, then 1, then zeros up to n), as residues:
//   spec[i][P][c][k], plane of 2T' per prime.
__global__ void k_tree_load(const uint64_t* __restrict__ below, int64_t T, int64_t Tp, int logn, NttConsts C,
                            uint32_t* __restrict__ spec) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over kNP * 2T'
  if (idx >= kNP * 2 * Tp) return;
  const int i = (int)(idx / (2 * Tp));
  const int64_t r = idx - (int64_t)i * 2 * Tp;
  const int64_t n = 1ll << logn, h = n >> 1;
  const int64_t child = r >> logn;          // 2P + c
  const int64_t k = r & (n - 1);
  int64_t d = T - child * h;
  d = d < 0 ? 0 : (d > h ? h : d);
  uint32_t x = 0;
  if (k < d) x = residue64(below[child * h + k], C, i);
  else if (k == d) x = 1;
  spec[idx] = x;
}

// Z[i][P][k] = spec_L[k] spec_R[k] (Montgomery), per prime plane of T'.
__global__ void k_tree_mul(const uint32_t* __restrict__ spec, int64_t Tp, int logn, NttConsts C,
                           uint32_t* __restrict__ Z) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over kNP * T'
  if (idx >= kNP * Tp) return;
  const int i = (int)(idx / Tp);
  const int64_t r = idx - (int64_t)i * Tp;
  const int64_t P = r >> logn, k = r & ((1ll << logn) - 1);
  const uint32_t q = C.q[i];
  const uint32_t* s = spec + (int64_t)i * 2 * Tp + (2 * P << logn);
  Z[idx] = mont32(sub_if(s[k], 2 * q), sub_if(s[(1ll << logn) + k], 2 * q), q, C.qinv[i]);
}

// coef[P n + k] = (L R)[k] for k < d_P, from the inverse transforms; when
// d_P = n the leading z^n wrapped onto z^0 and is taken off.
__global__ void k_tree_crt(const uint32_t* __restrict__ Z, int64_t T, int64_t Tp, int logn, NttConsts C, CrtScale sc,
                           Mod M, uint64_t* __restrict__ coef) {
  pdl_enter();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Tp) return;
  const int64_t n = 1ll << logn;
  const int64_t P = r >> logn, k = r & (n - 1);
  int64_t d = T - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  if (k >= d) return;
  uint32_t res[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++) res[i] = shoup32(Z[(int64_t)i * Tp + r], sc.s[i], sc.sp[i], C.q[i]);
  uint64_t x = crt_to_p(res, C, M);
  if (k == 0 && d == n) x = sub_mod(x, 1, M);
  coef[r] = x;
}

// Descent load: XH[r][i][P n + k] = X_P[d_P - 1 - k] (k < d_P), else 0; one
// thread per (r, P n + k) writes all five primes' residues.
__global__ void k_desc_load(const uint64_t* __restrict__ X, int R, int64_t T, int64_t Tp, int logn, NttConsts C,
                            uint32_t* __restrict__ XH) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over R * T'
  if (idx >= (int64_t)R * Tp) return;
  const int rr = (int)(idx / Tp);
  const int64_t e = idx - (int64_t)rr * Tp;
  const int64_t n = 1ll << logn;
  const int64_t P = e >> logn, k = e & (n - 1);
  int64_t d = T - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  const uint64_t x = k < d ? X[(int64_t)rr * Tp + P * n + d - 1 - k] : 0;
  uint32_t* out = XH + (int64_t)rr * kNP * Tp + e;
#pragma unroll
  for (int i = 0; i < kNP; i++) out[(int64_t)i * Tp] = k < d ? residue64(x, C, i) : 0u;
}

// Descent products: Y[c][r][i][P n + k] = XH[r][i][P n + k] spec[i][P][1 - c][k];
// one thread per (i, P n + k) loads the two spectra once for all R rows.
__global__ void k_desc_mul(const uint32_t* __restrict__ XH, const uint32_t* __restrict__ spec, int R, int64_t Tp,
                           int logn, NttConsts C, uint32_t* __restrict__ Y) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over kNP * T'
  if (idx >= (int64_t)kNP * Tp) return;
  const int i = (int)(idx / Tp);
  const int64_t e = idx - (int64_t)i * Tp;
  const uint32_t q = C.q[i], qi = C.qinv[i];
  const int64_t P = e >> logn, k = e & ((1ll << logn) - 1);
  const uint32_t* s = spec + (int64_t)i * 2 * Tp + (2 * P << logn) + k;
  const uint32_t sL = sub_if(s[0], 2 * q), sR = sub_if(s[1ll << logn], 2 * q);
  const int64_t all = (int64_t)R * kNP * Tp;
  for (int r = 0; r < R; r++) {
    const int64_t at = ((int64_t)r * kNP + i) * Tp + e;
    const uint32_t x = sub_if(XH[at], 2 * q);
    Y[at] = mont32(x, sR, q, qi);                   // child L: times R
    Y[all + at] = mont32(x, sL, q, qi);             // child R: times L
  }
}

// Descent Chinese remaindering: X'[r][(2P + c) h + m] = y_c[d_P - 1 - m], m < d_c.
__global__ void k_desc_crt(const uint32_t* __restrict__ Y, int R, int64_t T, int64_t Tp, int logn, NttConsts C,
                           CrtScale sc, Mod M, uint64_t* __restrict__ Xn) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over R * T' (child slots)
  if (idx >= (int64_t)R * Tp) return;
  const int rr = (int)(idx / Tp);
  const int64_t slot = idx - (int64_t)rr * Tp;             // (2P + c) h + m
  const int64_t n = 1ll << logn, h = n >> 1;
  const int64_t child = slot / h, m = slot - child * h;
  const int64_t P = child >> 1;
  const int c = (int)(child & 1);
  int64_t d = T - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  const int64_t dl = d < h ? d : h;
  const int64_t dc = c ? d - dl : dl;
  if (m >= dc) return;
  const int64_t all = (int64_t)R * kNP * Tp;
  const uint32_t* y = Y + c * all + (int64_t)rr * kNP * Tp + P * n + (d - 1 - m);
  uint32_t res[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++) res[i] = shoup32(y[(int64_t)i * Tp], sc.s[i], sc.sp[i], C.q[i]);
  Xn[idx] = crt_to_p(res, C, M);
}

// ---- general cyclic products (Newton's iteration) ----------------------------------

// A[i][k] = a[k] mod q_i for k < na, else 0 (planes of N)
__global__ void k_cyc_load(const uint64_t* __restrict__ a, int64_t na, int logN, NttConsts C, uint32_t* __restrict__ A) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ((int64_t)kNP << logN)) return;
  const int i = (int)(idx >> logN);
  const int64_t k = idx & ((1ll << logN) - 1);
  A[idx] = k < na ? residue64(a[k], C, i) : 0;
}
__global__ void k_cyc_mul(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B, int logN, NttConsts C,
                          uint32_t* __restrict__ Z) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ((int64_t)kNP << logN)) return;
  const int i = (int)(idx >> logN);
  const uint32_t q = C.q[i];
  Z[idx] = mont32(sub_if(A[idx], 2 * q), sub_if(B[idx], 2 * q), q, C.qinv[i]);
}
// out[t] = +-(a * b)[lo + t], t < cnt
__global__ void k_cyc_crt(const uint32_t* __restrict__ Z, int logN, int64_t lo, int64_t cnt, int neg, NttConsts C,
                          CrtScale sc, Mod M, uint64_t* __restrict__ out) {
  pdl_enter();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  uint32_t res[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++) res[i] = shoup32(Z[((int64_t)i << logN) + lo + t], sc.s[i], sc.sp[i], C.q[i]);
  const uint64_t x = crt_to_p(res, C, M);
  out[t] = neg ? (x ? M.p - x : 0) : x;
}

// f_t = coefficient t of rev(M) (f_0 = 1, f_t = m_{T-t}); rd_t = (T - t) m_{T-t}
// (rev(M'), degree T - 1; skipped when rd is null); g_0 = 1.
__global__ void k_rev_poly(const uint64_t* __restrict__ m, int64_t T, Mod M, uint64_t* __restrict__ f,
                           uint64_t* __restrict__ rd, uint64_t* __restrict__ g) {
  pdl_enter();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > T) return;
  const uint64_t mt = t == 0 ? 1 : m[T - t];
  f[t] = mt;
  if (rd && t < T) rd[t] = mul_mod((uint64_t)(T - t) % M.p, mt, M);
  if (t == 0) g[0] = 1;
}

// ---- levels small enough for one CTA ------------------------------------------------
//
// For transforms of n <= kFusedMax, one CTA holds the five primes' transforms
// of a node in shared memory and runs a whole level's work for it in one
// launch: residues, forward transforms, products, inverse transforms and the
// Chinese remaindering, with no trip through global memory in between.

constexpr int kFusedLog = 12;
constexpr int kFusedMax = 1 << kFusedLog;
constexpr int kFusedThreads = 512;
constexpr int kNewtonThreadsF = 1024;   // the single-CTA Newton kernel
constexpr int kClusterThreadsMax = 1024; // cluster levels of 2^13 and 2^14

// ntr transforms of size 2^logn at logical words off + t 2^logn of sm (the
// swizzled layout), transform t modulo prime t mod 5; forward (CT) or
// inverse (GS) stages.
template <bool INV>
__device__ __forceinline__ void smem_ntt(uint32_t* sm, int off, int ntr, int logn, const uint2* __restrict__ tw,
                                         int logN, const NttConsts& C) {
  smem_stages<INV>(sm, off, ntr << logn, logn, 0, 0u, tw, logN, C, [=](int x) { return (x >> logn) % kNP; });
}

// Nodes a fused CTA takes at transform size 2^logn.  One: packing several
// small nodes into a CTA measured slower than one node per CTA.
__host__ __device__ inline int fused_npc(int) { return 1; }

// Tree level l <= kFusedLog, npc nodes P per CTA: the two children as full
// monic polynomials -> spectra (kept in spec for the descent) -> product ->
// coefficients of P (coef, the wrapped z^n taken off when deg P = n).
__global__ void __launch_bounds__(kFusedThreads) k_tree_fused(const uint64_t* __restrict__ below, int64_t T,
                                                              int64_t Tp, int logn, NttConsts C, CrtScale sc, Mod M,
                                                              const uint2* __restrict__ tw, int logN,
                                                              uint32_t* __restrict__ spec, uint64_t* __restrict__ coef,
                                                              int64_t nodes) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // [c][node][prime][n]
  const int npc = fused_npc(logn);
  const int64_t P0 = (int64_t)blockIdx.x * npc;
  const int n = 1 << logn, h = n >> 1;
  const int half = (npc * kNP) << logn;         // the right children's transforms start here
  for (int e = threadIdx.x; e < 2 * npc * n; e += blockDim.x) {
    const int c = e / (npc * n), rest = e - c * npc * n;
    const int a = rest >> logn, k = rest & (n - 1);
    const int64_t child = 2 * (P0 + a) + c;
    int64_t d = T - child * h;
    d = d < 0 ? 0 : (d > h ? h : d);
    const uint64_t x = k < d ? below[child * h + k] : 0;
#pragma unroll
    for (int i = 0; i < kNP; i++)
      fsm[sw((((c * npc + a) * kNP + i) << logn) + k)] = k < d ? residue64(x, C, i) : (k == d ? 1u : 0u);
  }
  __syncthreads();
  smem_ntt<false>(fsm, 0, 2 * kNP * npc, logn, tw, logN, C);
  for (int e = threadIdx.x; e < half; e += blockDim.x) {
    const int t = e >> logn, k = e & (n - 1);    // t = a kNP + i
    const int a = t / kNP, i = t - a * kNP;
    const int64_t P = P0 + a;
    const uint32_t q = C.q[i];
    const uint32_t x = fsm[sw(e)], y = fsm[sw(half + e)];
    if (P < nodes) {
      uint32_t* sp = spec + (int64_t)i * 2 * Tp + (2 * P << logn) + k;
      sp[0] = x;
      sp[n] = y;
    }
    fsm[sw(e)] = mont32(sub_if(x, 2 * q), sub_if(y, 2 * q), q, C.qinv[i]);
  }
  __syncthreads();
  smem_ntt<true>(fsm, 0, npc * kNP, logn, tw + ((size_t)kNP << logN), logN, C);
  for (int e = threadIdx.x; e < npc * n; e += blockDim.x) {
    const int a = e >> logn, k = e & (n - 1);
    const int64_t P = P0 + a;
    int64_t d = T - P * n;
    d = d < 0 ? 0 : (d > n ? n : d);
    if (k >= d) continue;
    uint32_t res[kNP];
#pragma unroll
    for (int i = 0; i < kNP; i++) res[i] = shoup32(fsm[sw(((a * kNP + i) << logn) + k)], sc.s[i], sc.sp[i], C.q[i]);
    uint64_t x = crt_to_p(res, C, M);
    if (k == 0 && d == n) x = sub_mod(x, 1, M);
    coef[P * n + k] = x;
  }
}

// Descent level l <= kFusedLog, npc nodes P of one right-hand side r per
// CTA: X_P reversed -> spectrum -> times each child's sibling spectrum ->
// inverse -> Chinese remaindering into the children's expansions.
__global__ void __launch_bounds__(kFusedThreads) k_desc_fused(const uint64_t* __restrict__ X, int64_t T, int64_t Tp,
                                                              int logn, NttConsts C, CrtScale sc, Mod M,
                                                              const uint2* __restrict__ tw, int logN,
                                                              const uint32_t* __restrict__ spec,
                                                              uint64_t* __restrict__ Xn, int64_t nodes) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // XH [node][prime][n], then Y [node][prime][n] (logical words)
  const int npc = fused_npc(logn);
  const int64_t ctas = (nodes + npc - 1) / npc;
  const int64_t P0 = (int64_t)(blockIdx.x % ctas) * npc;
  const int r = (int)(blockIdx.x / ctas);
  const int n = 1 << logn, h = n >> 1;
  const int span = (npc * kNP) << logn;
  const uint64_t* x = X + (int64_t)r * Tp;
  for (int e = threadIdx.x; e < npc * n; e += blockDim.x) {
    const int a = e >> logn, k = e & (n - 1);
    const int64_t P = P0 + a;
    int64_t d = T - P * n;
    d = d < 0 ? 0 : (d > n ? n : d);
    const uint64_t v = k < d ? x[P * n + d - 1 - k] : 0;
#pragma unroll
    for (int i = 0; i < kNP; i++) fsm[sw(((a * kNP + i) << logn) + k)] = k < d ? residue64(v, C, i) : 0u;
  }
  __syncthreads();
  smem_ntt<false>(fsm, 0, npc * kNP, logn, tw, logN, C);
  for (int c = 0; c < 2; c++) {
    for (int e = threadIdx.x; e < span; e += blockDim.x) {
      const int t = e >> logn, k = e & (n - 1);
      const int a = t / kNP, i = t - a * kNP;
      const int64_t P = P0 + a;
      const uint32_t q = C.q[i];
      const uint32_t s = P < nodes ? spec[(int64_t)i * 2 * Tp + ((2 * P + (1 - c)) << logn) + k] : 0u;
      fsm[sw(span + e)] = mont32(sub_if(fsm[sw(e)], 2 * q), sub_if(s, 2 * q), q, C.qinv[i]);
    }
    __syncthreads();
    smem_ntt<true>(fsm, span, npc * kNP, logn, tw + ((size_t)kNP << logN), logN, C);
    for (int e = threadIdx.x; e < npc * h; e += blockDim.x) {
      const int a = e / h, m = e - a * h;
      const int64_t P = P0 + a;
      int64_t d = T - P * n;
      d = d < 0 ? 0 : (d > n ? n : d);
      const int64_t dl = d < h ? d : h;
      const int64_t dc = c ? d - dl : dl;
      if (m >= dc) continue;
      uint32_t res[kNP];
#pragma unroll
      for (int i = 0; i < kNP; i++)
        res[i] = shoup32(fsm[sw(span + ((a * kNP + i) << logn) + (int)(d - 1 - m))], sc.s[i], sc.sp[i], C.q[i]);
      Xn[(int64_t)r * Tp + (2 * P + c) * h + m] = crt_to_p(res, C, M);
    }
    __syncthreads();
  }
}

// Newton's iteration for g = 1 / f mod z^K (K a power of two <= kFusedMax),
// f_0 = 1, all in one CTA: for k = 1, 2, .., K/2, e = f g_k (its coefficients
// k..2k-1, a cyclic product of size 2k), then g_{k..2k} = -(g_k e_hi mod z^k).
// g (2K words) and e (K words) live in global memory; f has nf coefficients.
__global__ void __launch_bounds__(kNewtonThreadsF) k_newton_fused(const uint64_t* __restrict__ f, int64_t nf, int logK,
                                                                NttConsts C, Mod M, const uint2* __restrict__ tw,
                                                                int logN, uint64_t* __restrict__ g,
                                                                uint64_t* __restrict__ e) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // A [prime][2k], then B [prime][2k] (logical words)
  if (threadIdx.x == 0) g[0] = 1;
  __syncthreads();
  for (int lk = 0; lk < logK; lk++) {
    const int k = 1 << lk, logn = lk + 1, n = 2 * k;
    const int bo = kNP << logn;                  // B's first logical word
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const uint64_t fv = t < nf ? f[t] : 0;
      const uint64_t gv = t < k ? g[t] : 0;
#pragma unroll
      for (int i = 0; i < kNP; i++) {
        fsm[sw((i << logn) + t)] = t < nf ? residue64(fv, C, i) : 0u;
        fsm[sw(bo + (i << logn) + t)] = t < k ? residue64(gv, C, i) : 0u;
      }
    }
    __syncthreads();
    smem_ntt<false>(fsm, 0, 2 * kNP, logn, tw, logN, C);  // A and B are contiguous: ten transforms
    for (int x = threadIdx.x; x < kNP * n; x += blockDim.x) {
      const int i = x >> logn;
      const uint32_t q = C.q[i];
      fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(bo + x)], 2 * q), q, C.qinv[i]);
    }
    __syncthreads();
    smem_ntt<true>(fsm, 0, kNP, logn, tw + ((size_t)kNP << logN), logN, C);
    // scale 2^32 / n per prime, computed here (n varies by step)
    uint32_t s[kNP], sp[kNP];
#pragma unroll
    for (int i = 0; i < kNP; i++) {
      const uint32_t q = C.q[i];
      // 2^32 / 2^logn mod q: 2^(32 - logn) when logn <= 32 is exact
      const uint32_t x = (uint32_t)(((uint64_t)1 << (32 - logn)) % q);
      s[i] = x;
      sp[i] = (uint32_t)(((uint64_t)x << 32) / q);
    }
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      uint32_t res[kNP];
#pragma unroll
      for (int i = 0; i < kNP; i++) res[i] = shoup32(fsm[sw((i << logn) + k + t)], s[i], sp[i], C.q[i]);
      e[t] = crt_to_p(res, C, M);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const uint64_t ev = t < k ? e[t] : 0;
#pragma unroll
      for (int i = 0; i < kNP; i++) fsm[sw((i << logn) + t)] = t < k ? residue64(ev, C, i) : 0u;
    }
    __syncthreads();
    smem_ntt<false>(fsm, 0, kNP, logn, tw, logN, C);
    for (int x = threadIdx.x; x < kNP * n; x += blockDim.x) {
      const int i = x >> logn;
      const uint32_t q = C.q[i];
      fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(bo + x)], 2 * q), q, C.qinv[i]);
    }
    __syncthreads();
    smem_ntt<true>(fsm, 0, kNP, logn, tw + ((size_t)kNP << logN), logN, C);
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      uint32_t res[kNP];
#pragma unroll
      for (int i = 0; i < kNP; i++) res[i] = shoup32(fsm[sw((i << logn) + t)], s[i], sp[i], C.q[i]);
      const uint64_t x = crt_to_p(res, C, M);
      g[k + t] = x ? M.p - x : 0;
    }
    __syncthreads();
  }
}

// Thread-block cluster primitives (PTX): the CTA's rank in its cluster, a
// cluster-wide barrier (arrive has release, wait acquire semantics at
// cluster scope), and 32-bit loads from another CTA's shared memory.
__device__ __forceinline__ int cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive;\n\tbarrier.cluster.wait;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_cluster(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Precision up to which k_newton_cluster runs schoolbook steps, and the
// largest number of coefficients a thread holds in registers (precision up
// to 2^14 = kNewtonPer x 1024 threads).
constexpr int kNewtonSchool = 256;
constexpr int kNewtonPer = 16;
__device__ __forceinline__ int ilog2_dev(int x) { return 31 - __clz(x); }   // x a power of two

// The division step of k_newton_cluster's quotient mode: g mod q_me in
// Gq[0, k), k = n / 2; writes h = rd / f mod z^T (k < T <= n) to ps.  The
// residues a CTA needs of a remaindered product wait in v across the barrier
// that frees the buffer they go to.
__device__ __forceinline__ void newton_cluster_divide(uint32_t* fsm, int me, const uint32_t* peer, int logn,
                                                      const uint64_t* __restrict__ f, int64_t nf, const uint32_t* Gq,
                                                      const uint64_t* __restrict__ rd, int64_t T, const NttConsts& C,
                                                      const Mod& M, const uint2* __restrict__ tw,
                                                      const uint2* __restrict__ itw, int logN,
                                                      uint64_t* __restrict__ ps) {
  const int n = 1 << logn, k = n / 2;
  const int hi = (int)(T - k);                   // the coefficients the last product gives: 1 .. k
  const uint32_t q = C.q[me], qi = C.qinv[me];
  auto prime = [=](int) { return me; };
  uint32_t s[kNP], sp[kNP];                      // 2^(32 - logn) mod q_j
#pragma unroll
  for (int j = 0; j < kNP; j++) {
    s[j] = (uint32_t)(((uint64_t)1 << (32 - logn)) % C.q[j]);
    sp[j] = (uint32_t)(((uint64_t)s[j] << 32) / C.q[j]);
  }
  uint32_t v[kNewtonPer];
  // g's region (at 2n) into the transform layout, B := rd mod z^k
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    v[r] = t < k ? Gq[t] : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    if (t < n) fsm[sw(2 * n + t)] = v[r];
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) fsm[sw(n + t)] = t < k ? residue64(rd[t], C, me) : 0u;
  __syncthreads();
  smem_stages<false>(fsm, n, 2 * n, logn, 0, 0u, tw, logN, C, prime);   // B and g
  for (int x = threadIdx.x; x < n; x += blockDim.x)
    fsm[sw(n + x)] = mont32(sub_if(fsm[sw(n + x)], 2 * q), sub_if(fsm[sw(2 * n + x)], 2 * q), q, qi);
  __syncthreads();
  smem_stages<true>(fsm, n, n, logn, 0, 0u, itw, logN, C, prime);
  cluster_sync();                                // every CTA's B holds rd g mod its prime
  // q0 = h mod z^k: every CTA remainders all k coefficients, CTA 0 writes them
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    uint32_t val = 0;
    if (t < k) {
      uint32_t res[kNP];
#pragma unroll
      for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(n + t)), s[j], sp[j], C.q[j]);
      const uint64_t x = crt_to_p(res, C, M);
      if (me == 0) ps[t] = x;
      val = residue64(x, C, me);
    }
    v[r] = val;
  }
  cluster_sync();                                // B is no longer read
  // A := f mod z^T, B := q0; their product's coefficients k .. T-1
  for (int t = threadIdx.x; t < n; t += blockDim.x) fsm[sw(t)] = (t < T && t < nf) ? residue64(f[t], C, me) : 0u;
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    if (t < n) fsm[sw(n + t)] = v[r];
  }
  __syncthreads();
  smem_stages<false>(fsm, 0, 2 * n, logn, 0, 0u, tw, logN, C, prime);   // A and B
  for (int x = threadIdx.x; x < n; x += blockDim.x)
    fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(n + x)], 2 * q), q, qi);
  __syncthreads();
  smem_stages<true>(fsm, 0, n, logn, 0, 0u, itw, logN, C, prime);
  cluster_sync();                                // every CTA's A holds f q0 mod its prime
  // r_t = rd_{k+t} - (f q0)_{k+t}, t < T - k
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    uint32_t val = 0;
    if (t < hi) {
      uint32_t res[kNP];
#pragma unroll
      for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(k + t)), s[j], sp[j], C.q[j]);
      const uint64_t fq = crt_to_p(res, C, M), a = rd[k + t];
      val = residue64(a >= fq ? a - fq : a + (M.p - fq), C, me);
    }
    v[r] = val;
  }
  cluster_sync();                                // A is no longer read
#pragma unroll
  for (int r = 0; r < kNewtonPer; r++) {
    const int t = threadIdx.x + r * (int)blockDim.x;
    if (t < n) fsm[sw(t)] = v[r];
  }
  __syncthreads();
  smem_stages<false>(fsm, 0, n, logn, 0, 0u, tw, logN, C, prime);
  for (int x = threadIdx.x; x < n; x += blockDim.x)
    fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(2 * n + x)], 2 * q), q, qi);
  __syncthreads();
  smem_stages<true>(fsm, 0, n, logn, 0, 0u, itw, logN, C, prime);
  cluster_sync();                                // every CTA's A holds g r mod its prime
  // h_{k+t} = (g r)_t: each CTA remainders and writes a fifth
  const int chunk = (hi + kNP - 1) / kNP, t0 = me * chunk, t1 = t0 + chunk < hi ? t0 + chunk : hi;
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    uint32_t res[kNP];
#pragma unroll
    for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(t)), s[j], sp[j], C.q[j]);
    ps[k + t] = crt_to_p(res, C, M);
  }
}

// k_newton_fused spread over a cluster of kNP CTAs, CTA i holding prime i's
// transforms in its shared memory: A (f, then f g, then e_hi and g e_hi: the
// second product takes A's place once every CTA has read it), B (g's
// spectrum) in the swizzled layout, and g mod q_i.  Each Chinese
// remaindering reads the five CTAs' residues through distributed shared
// memory, and every CTA remainders all k coefficients, so that each has e
// (and the new g) for its own prime without a trip through global memory;
// CTA 0 writes g.  A cluster barrier separates a product's last writes from
// its remote reads, and another those reads from the buffer's next writes
// (the remaindered values wait in registers meanwhile); the last one keeps
// every CTA resident until the others are done reading it.
//
// With ps non-null the kernel returns the quotient h = rd / f mod z^T
// instead (rd: T coefficients, 2^(logK-1) < T <= 2^logK, T > kNewtonSchool):
// Newton's iteration stops at g = 1/f mod z^k, k = 2^(logK-1), and one
// division step in the manner of Karp and Markstein finishes with three
// products of n = 2k points: q0 = rd g mod z^k (= h mod z^k); r = (rd - f q0)
// div z^k mod z^(T-k); h_{k+t} = (g r)_t for t < T - k.  (f h = rd mod z^T
// and f q0 = rd mod z^k give f (h - q0) / z^k = r, so (h - q0) / z^k = g r
// mod z^(T-k), T - k <= k.)  The cyclic products are exact where read: rd g
// and g r have fewer than n coefficients, and f q0 (f mod z^T) wraps only
// onto coefficients below T + k - n <= k.  Shared memory: A at 0, B at n
// and g's region at 2n, each of n words.
__global__ void __launch_bounds__(kNewtonThreadsF) k_newton_cluster(const uint64_t* __restrict__ f, int64_t nf,
                                                                  int logK, NttConsts C, Mod M,
                                                                  const uint2* __restrict__ tw, int logN,
                                                                  uint64_t* __restrict__ g,
                                                                  const uint64_t* __restrict__ rd, int64_t T,
                                                                  uint64_t* __restrict__ ps) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // A (= C) [n] at 0, B [n] at n (logical); then g mod q
  const int me = cluster_rank();
  const int K = 1 << logK;
  uint32_t* Gq = fsm + ((2 * K + 31) & ~31);
  const uint32_t q = C.q[me], qi = C.qinv[me];
  const uint2* __restrict__ itw = tw + ((size_t)kNP << logN);
  uint32_t peer[kNP];
#pragma unroll
  for (int j = 0; j < kNP; j++) peer[j] = cluster_addr(fsm, j);
  auto prime = [=](int) { return me; };
  const int logG = ps ? logK - 1 : logK;         // Newton's iteration runs to precision 2^logG
  const int KG = 1 << logG;
  // the first steps, to precision K1, by schoolbook products in 64-bit
  // residues, every CTA computing the same g (no transforms, no exchange):
  // e_t = (f g)_{k+t} = sum_{i<k} f_{k+t-i} g_i, then g_{k+t} = -sum_{i<=t} g_i e_{t-i}
  const int K1 = KG < kNewtonSchool ? KG : kNewtonSchool;
  uint64_t* g64 = reinterpret_cast<uint64_t*>(fsm);            // K1 words
  uint64_t* e64 = g64 + K1;                                     // K1 / 2 words
  if (threadIdx.x == 0) g64[0] = 1;
  __syncthreads();
  for (int k = 1; k < K1; k *= 2) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int i = 0; i < k; i++) {
        const int64_t fi = k + t - i;
        if (fi < nf) {
          const uint64_t x = f[fi], y = g64[i];
          mac8(acc, lo32(x), hi32(x), lo32(y), hi32(y));
        }
      }
      e64[t] = acc8_value(acc, M);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int i = 0; i <= t; i++) {
        const uint64_t x = g64[i], y = e64[t - i];
        mac8(acc, lo32(x), hi32(x), lo32(y), hi32(y));
      }
      const uint64_t v = acc8_value(acc, M);
      g64[k + t] = v ? M.p - v : 0;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < K1; t += blockDim.x) {
    Gq[t] = residue64(g64[t], C, me);
    if (me == 0) g[t] = g64[t];
  }
  __syncthreads();
  for (int lk = ilog2_dev(K1); lk < logG; lk++) {
    const int k = 1 << lk, logn = lk + 1, n = 2 * k;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      fsm[sw(t)] = t < nf ? residue64(f[t], C, me) : 0u;
      fsm[sw(n + t)] = t < k ? Gq[t] : 0u;
    }
    __syncthreads();
    smem_stages<false>(fsm, 0, 2 * n, logn, 0, 0u, tw, logN, C, prime);   // A and B
    for (int x = threadIdx.x; x < n; x += blockDim.x)
      fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(n + x)], 2 * q), q, qi);
    __syncthreads();
    smem_stages<true>(fsm, 0, n, logn, 0, 0u, itw, logN, C, prime);
    uint32_t s[kNP], sp[kNP];                    // 2^32 / n mod q_j: 2^(32 - logn) mod q_j
#pragma unroll
    for (int j = 0; j < kNP; j++) {
      s[j] = (uint32_t)(((uint64_t)1 << (32 - logn)) % C.q[j]);
      sp[j] = (uint32_t)(((uint64_t)s[j] << 32) / C.q[j]);
    }
    cluster_sync();                              // every CTA's A holds f g mod its prime
    // e_hi mod this prime, held in registers until every CTA has read A
    uint32_t ev[kNewtonPer];
#pragma unroll
    for (int r = 0; r < kNewtonPer; r++) {
      const int t = threadIdx.x + r * (int)blockDim.x;
      uint32_t v = 0;
      if (t < k) {
        uint32_t res[kNP];
#pragma unroll
        for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(k + t)), s[j], sp[j], C.q[j]);
        v = residue64(crt_to_p(res, C, M), C, me);
      }
      ev[r] = v;
    }
    cluster_sync();                              // A is no longer read: C takes its place
#pragma unroll
    for (int r = 0; r < kNewtonPer; r++) {
      const int t = threadIdx.x + r * (int)blockDim.x;
      if (t < n) fsm[sw(t)] = ev[r];
    }
    __syncthreads();
    smem_stages<false>(fsm, 0, n, logn, 0, 0u, tw, logN, C, prime);
    for (int x = threadIdx.x; x < n; x += blockDim.x)
      fsm[sw(x)] = mont32(sub_if(fsm[sw(x)], 2 * q), sub_if(fsm[sw(n + x)], 2 * q), q, qi);
    __syncthreads();
    smem_stages<true>(fsm, 0, n, logn, 0, 0u, itw, logN, C, prime);
    cluster_sync();                              // every CTA's C holds g e_hi mod its prime
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      uint32_t res[kNP];
#pragma unroll
      for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(t)), s[j], sp[j], C.q[j]);
      const uint64_t x = crt_to_p(res, C, M);
      const uint64_t gv = x ? M.p - x : 0;
      Gq[k + t] = residue64(gv, C, me);
      if (me == 0) g[k + t] = gv;
    }
    cluster_sync();                              // C is no longer read: the next step may write A
  }
  if (ps) newton_cluster_divide(fsm, me, peer, logK, f, nf, Gq, rd, T, C, M, tw, itw, logN, ps);
  cluster_sync();
}

// ---- levels small enough for one CTA per prime: clusters of kNP CTAs ---------------
//
// The same levels as k_tree_fused / k_desc_fused / k_up_fused with a node's
// five transforms spread over a cluster, CTA i holding prime i's: a fifth of
// the shared memory and five times the CTAs of the one-CTA form.  After the
// inverse transforms a cluster barrier makes every CTA's residues visible,
// each CTA remainders a fifth of the node's outputs reading the five
// residues of a coefficient through distributed shared memory, and a last
// barrier keeps the CTAs resident until the others are done reading.

// Threads of a cluster CTA at transform size 2^logn.
inline int cluster_threads(int logn) {
  return logn >= 13 ? kClusterThreadsMax : std::min(kFusedThreads, std::max(64, (1 << logn) >> 2));
}

// Cluster levels go up to transforms of 2^14 (a descent CTA then holds
// 192 KB); Newton's cluster runs to precision 2^14.  Above 2^12 a level
// takes the cluster form only when its CTAs fit in two waves: with many
// nodes the tile kernels' higher occupancy wins.
constexpr int kClusterMaxLog = 14;
constexpr int kNewtonClusterLog = 14;

// Tree level l <= kFusedLog: the children of node P as full monic
// polynomials (modulo prime `me`) -> spectra (kept in spec for the descent)
// -> product -> inverse -> coefficients of P (the wrapped z^n taken off).
__global__ void __launch_bounds__(kClusterThreadsMax) k_tree_cluster(const uint64_t* __restrict__ below, int64_t T,
                                                                int64_t Tp, int logn, NttConsts C, CrtScale sc, Mod M,
                                                                const uint2* __restrict__ tw, int logN,
                                                                uint32_t* __restrict__ spec,
                                                                uint64_t* __restrict__ coef) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // L [n], R [n] (logical words)
  const int me = cluster_rank();
  const int64_t P = blockIdx.x / kNP;
  const int n = 1 << logn, h = n >> 1;
  const uint32_t q = C.q[me], qi = C.qinv[me];
  auto prime = [=](int) { return me; };
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    const int c = e >> logn, k = e & (n - 1);
    const int64_t child = 2 * P + c;
    int64_t d = T - child * h;
    d = d < 0 ? 0 : (d > h ? h : d);
    fsm[sw(e)] = k < d ? residue64(below[child * h + k], C, me) : (k == d ? 1u : 0u);
  }
  __syncthreads();
  smem_stages<false>(fsm, 0, 2 * n, logn, 0, 0u, tw, logN, C, prime);
  uint32_t* sp = spec + (int64_t)me * 2 * Tp + (2 * P << logn);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t x = fsm[sw(k)], y = fsm[sw(n + k)];
    sp[k] = x;
    sp[n + k] = y;
    fsm[sw(k)] = mont32(sub_if(x, 2 * q), sub_if(y, 2 * q), q, qi);
  }
  if (coef == nullptr) return;                   // the children's spectra only (every CTA alike)
  __syncthreads();
  smem_stages<true>(fsm, 0, n, logn, 0, 0u, tw + ((size_t)kNP << logN), logN, C, prime);
  cluster_sync();
  int64_t d = T - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  const int per = (int)((d + kNP - 1) / kNP);
  const int lo = me * per, hi = (int)(d < (int64_t)lo + per ? d : (int64_t)lo + per);
  uint32_t peer[kNP];
#pragma unroll
  for (int j = 0; j < kNP; j++) peer[j] = cluster_addr(fsm, j);
  for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    uint32_t res[kNP];
#pragma unroll
    for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(k)), sc.s[j], sc.sp[j], C.q[j]);
    uint64_t x = crt_to_p(res, C, M);
    if (k == 0 && d == n) x = sub_mod(x, 1, M);
    coef[P * n + k] = x;
  }
  cluster_sync();
}

// Descent level l <= kFusedLog, node P and right-hand side r per cluster:
// X_P reversed (modulo prime `me`) -> spectrum -> times each child's sibling
// spectrum -> inverse -> the children's expansions.
__global__ void __launch_bounds__(kClusterThreadsMax) k_desc_cluster(const uint64_t* __restrict__ X, int64_t T, int64_t Tp,
                                                                int logn, NttConsts C, CrtScale sc, Mod M,
                                                                const uint2* __restrict__ tw, int logN,
                                                                const uint32_t* __restrict__ spec,
                                                                uint64_t* __restrict__ Xn, int64_t nodes) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // XH [n], Y [2][n] at n (logical words)
  const int me = cluster_rank();
  const int64_t cl = blockIdx.x / kNP;
  const int64_t P = cl % nodes;
  const int r = (int)(cl / nodes);
  const int n = 1 << logn, h = n >> 1;
  const uint32_t q = C.q[me], qi = C.qinv[me];
  auto prime = [=](int) { return me; };
  int64_t d = T - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  const uint64_t* x = X + (int64_t)r * Tp + P * n;
  if (d <= h) {
    // the right child holds no roots (R = 1): the left child's expansion is
    // the node's, X_L[m] = X_P[m], at the same offset; the five CTAs copy a
    // fifth each and leave together (no cluster barrier on this branch)
    const int per = (int)((d + kNP - 1) / kNP);
    const int lo = me * per, hi = (int)(d < (int64_t)lo + per ? d : (int64_t)lo + per);
    for (int o = lo + threadIdx.x; o < hi; o += blockDim.x) Xn[(int64_t)r * Tp + P * n + o] = x[o];
    return;
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) fsm[sw(k)] = k < d ? residue64(x[d - 1 - k], C, me) : 0u;
  __syncthreads();
  smem_stages<false>(fsm, 0, n, logn, 0, 0u, tw, logN, C, prime);
  const uint32_t* sp = spec + (int64_t)me * 2 * Tp + (2 * P << logn);
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    const int c = e >> logn, k = e & (n - 1);
    const uint32_t sib = sp[((1 - c) << logn) + k];       // child c times its sibling
    fsm[sw(n + e)] = mont32(sub_if(fsm[sw(k)], 2 * q), sub_if(sib, 2 * q), q, qi);
  }
  __syncthreads();
  smem_stages<true>(fsm, n, 2 * n, logn, 0, 0u, tw + ((size_t)kNP << logN), logN, C, prime);
  cluster_sync();
  const int dl = (int)(d < h ? d : h);
  const int per = (int)((d + kNP - 1) / kNP);
  const int lo = me * per, hi = (int)(d < (int64_t)lo + per ? d : (int64_t)lo + per);
  uint32_t peer[kNP];
#pragma unroll
  for (int j = 0; j < kNP; j++) peer[j] = cluster_addr(fsm, j);
  for (int o = lo + threadIdx.x; o < hi; o += blockDim.x) {
    const int c = o < dl ? 0 : 1;
    const int m = c ? o - dl : o;
    const int at = n + (c << logn) + (int)(d - 1 - m);
    uint32_t res[kNP];
#pragma unroll
    for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(at)), sc.s[j], sc.sp[j], C.q[j]);
    Xn[(int64_t)r * Tp + (2 * P + c) * h + m] = crt_to_p(res, C, M);
  }
  cluster_sync();
}

// ---- leaves --------------------------------------------------------------------------

constexpr int kLeaf = 128;                     // roots per leaf block (tree level 7)
constexpr int kLeafLog = 7;

// Block polynomials prod_{j in block} (z - v_j), monic, degree d <= 128:
// levels 0..6 of pairwise products in shared memory.
__global__ void __launch_bounds__(kLeaf) k_fast_leafpoly(const uint64_t* __restrict__ v, int64_t T, Mod M,
                                                         uint64_t* __restrict__ coef) {
  pdl_enter();
  __shared__ uint64_t buf[2][kLeaf];
  const int64_t base = (int64_t)blockIdx.x * kLeaf;
  const int cnt = (int)((T - base) < kLeaf ? (T - base) : kLeaf);
  const int t = threadIdx.x;
  if (t < cnt) {
    const uint64_t x = v[base + t];
    buf[0][t] = x ? M.p - x : 0;
  }
  __syncthreads();
  int cur = 0;
  for (int l = 0; l < kLeafLog; l++) {
    const int size = 1 << l, pair = 2 << l;
    if (t < cnt) {
      const int po = t & ~(pair - 1);
      uint64_t r;
      if (cnt - po <= size) r = buf[cur][t];
      else r = conv_coef(buf[cur], po, size, min(size, cnt - po - size), t - po, M);
      buf[cur ^ 1][t] = r;
    }
    __syncthreads();
    cur ^= 1;
  }
  if (t < cnt) coef[base + t] = buf[cur][t];
}

// Leaf values: for root j of block P (degree d), val_r = <q^P_j, X_P^(r)>,
// q^P_{j,d-1} = 1, q^P_{j,k-1} = p_k + v_j q^P_{j,k}.  Rows r < R - 1 are the
// right-hand sides (written to part[r ldp + j]), row R - 1 the power sums
// (M'(v_j), written to den[j]).  A CTA takes one block and one group of
// kLeafCols rows (blockIdx.y), each thread one root, rerunning the chain per
// group so that the groups run in parallel.
constexpr int kLeafCols = 4;

__global__ void __launch_bounds__(kLeaf) k_fast_leafval(const uint64_t* __restrict__ coef7,
                                                        const uint64_t* __restrict__ X, int R, int64_t T, int64_t Tp,
                                                        const uint64_t* __restrict__ v, const uint64_t* __restrict__ vp,
                                                        Mod M, uint64_t* __restrict__ part, int64_t ldp,
                                                        uint64_t* __restrict__ den) {
  pdl_enter();
  __shared__ uint64_t pc[kLeaf];                 // block polynomial
  __shared__ uint64_t xs[kLeafCols][kLeaf];      // this group's X rows
  const int64_t base = (int64_t)blockIdx.x * kLeaf;
  const int r0 = blockIdx.y * kLeafCols;
  const int d = (int)((T - base) < kLeaf ? (T - base) : kLeaf);
  const int t = threadIdx.x;
  if (t < d) pc[t] = coef7[base + t];
#pragma unroll
  for (int c = 0; c < kLeafCols; c++)
    if (t < d && r0 + c < R) xs[c][t] = X[(int64_t)(r0 + c) * Tp + base + t];
  __syncthreads();
  if (t >= d) return;
  const int64_t j = base + t;
  const uint64_t vj = v[j], vpj = vp[j];
  Acc8 acc[kLeafCols];
#pragma unroll
  for (int c = 0; c < kLeafCols; c++) acc[c] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t q = 1;
  for (int k = d - 1; k >= 0; k--) {
    const uint64_t qc = canon(q, M);
    const uint32_t x0 = lo32(qc), x1 = hi32(qc);
#pragma unroll
    for (int c = 0; c < kLeafCols; c++)
      if (r0 + c < R) {
        const uint64_t w = xs[c][k];
        mac8(acc[c], x0, x1, lo32(w), hi32(w));
      }
    q = canon(shoup_lazy(qc, vj, vpj, M), M) + pc[k];
  }
#pragma unroll
  for (int c = 0; c < kLeafCols; c++) {
    const int r = r0 + c;
    if (r < R - 1) part[(int64_t)r * ldp + j] = acc8_value(acc[c], M);
    else if (r == R - 1) den[j] = acc8_value(acc[c], M);
  }
}

// X0[r][k] = b[r ldb + k] (r < S), X0[S][k] = power sums (k < T), rows r0 .. r0 + nr - 1
__global__ void k_stage_rhs(const uint64_t* __restrict__ b, int64_t ldb, int S, const uint64_t* __restrict__ ps,
                            int r0, int nr, int64_t T, int64_t Tp, uint64_t* __restrict__ X0) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nr * T) return;
  const int r = r0 + (int)(idx / T);
  const int64_t k = idx - (int64_t)(r - r0) * T;
  X0[(int64_t)r * Tp + k] = r < S ? b[(int64_t)r * ldb + k] : ps[k];
}

// ---- power sums directly: p_k = sum_j v_j^k ------------------------------------------
//
// T^2 Shoup steps over every SM, from the nodes alone, so that they run beside
// the tree and the power sums' row joins the right-hand sides' descent.  Block
// (kb, jb) takes the exponents [kb kr, (kb + 1) kr) and the nodes
// [jb kPsNodes, (jb + 1) kPsNodes); each thread carries kPsJ powers v_j^k
// (lazily in [0, 2p)) along the exponents, one Shoup product per step, and
// adds them over a window of kPsWin exponents into 128-bit sums; the block
// then adds its threads' windows through shared memory (one warp per
// exponent: 8 partial sums a lane, then 5 shuffles) and reduces each sum
// once, into part[jb T + k].  The starting powers v_j^(kb kr) come from
// k_ps_start.
constexpr int kPsThreads = 256;
constexpr int kPsJ = 8;
constexpr int kPsWin = 8;                     // kPsThreads = kPsWin warps
constexpr int kPsNodes = kPsThreads * kPsJ;
constexpr int kPsWaves = 8;

// start[kb T + j] = v_j^(kb kr) (lazily, in [0, 2p)), kb < nkb
__global__ void k_ps_start(const uint64_t* __restrict__ v, int64_t T, int kr, int nkb, Mod M,
                           uint64_t* __restrict__ start) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  const uint64_t w = pow_mod(v[j], (uint64_t)kr, M), wq = shoup_pre(w, M);
  uint64_t x = 1;
  for (int kb = 0; kb < nkb; kb++) {
    start[(int64_t)kb * T + j] = x;
    x = shoup_lazy(x, w, wq, M);
  }
}

__global__ void __launch_bounds__(kPsThreads) k_power_sums(const uint64_t* __restrict__ v,
                                                           const uint64_t* __restrict__ vp, int64_t T, int kr,
                                                           const uint64_t* __restrict__ start, Mod M,
                                                           uint64_t* __restrict__ part) {
  pdl_enter();
  __shared__ uint64_t red_lo[kPsThreads][kPsWin + 1];
  __shared__ uint32_t red_hi[kPsThreads][kPsWin + 1];
  const int64_t k0 = (int64_t)blockIdx.x * kr;
  const int64_t k1 = k0 + kr < T ? k0 + kr : T;
  const int64_t j0 = (int64_t)blockIdx.y * kPsNodes;
  uint64_t x[kPsJ], w[kPsJ], wq[kPsJ];         // nodes past T carry 0
#pragma unroll
  for (int m = 0; m < kPsJ; m++) {
    const int64_t j = j0 + m * kPsThreads + threadIdx.x;
    const bool in = j < T;
    w[m] = in ? v[j] : 0;
    wq[m] = in ? vp[j] : 0;
    x[m] = in ? start[(int64_t)blockIdx.x * T + j] : 0;
  }
  const int kk = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t kw = k0; kw < k1; kw += kPsWin) {
    uint64_t lo[kPsWin];
    uint32_t hi[kPsWin];
#pragma unroll
    for (int i = 0; i < kPsWin; i++) lo[i] = 0, hi[i] = 0;
#pragma unroll
    for (int m = 0; m < kPsJ; m++) {
#pragma unroll
      for (int i = 0; i < kPsWin; i++) {
        lo[i] += x[m];
        hi[i] += lo[i] < x[m];
        x[m] = shoup_lazy(x[m], w[m], wq[m], M);
      }
    }
#pragma unroll
    for (int i = 0; i < kPsWin; i++) red_lo[threadIdx.x][i] = lo[i], red_hi[threadIdx.x][i] = hi[i];
    __syncthreads();
    uint64_t sl = 0;
    uint32_t sh = 0;
#pragma unroll
    for (int i = 0; i < kPsThreads / 32; i++) {
      const uint64_t a = red_lo[lane + 32 * i][kk];
      sl += a;
      sh += red_hi[lane + 32 * i][kk] + (sl < a);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const uint64_t a = __shfl_xor_sync(0xffffffffu, sl, o);
      const uint32_t b = __shfl_xor_sync(0xffffffffu, sh, o);
      sl += a;
      sh += b + (sl < a);
    }
    if (lane == 0 && kw + kk < k1) part[(int64_t)blockIdx.y * T + kw + kk] = reduce128(sh, sl, M);
    __syncthreads();
  }
}

// ps[k] = sum over the nb node blocks of part[jb T + k]
__global__ void k_power_sums_add(const uint64_t* __restrict__ part, int64_t T, int nb, Mod M,
                                 uint64_t* __restrict__ ps) {
  pdl_enter();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T) return;
  uint64_t sum = 0;
  for (int jb = 0; jb < nb; jb++) sum = add_mod(sum, part[(int64_t)jb * T + k], M);
  ps[k] = sum;
}

// The launch shape of k_power_sums: nb node blocks, nkb exponent blocks of kr
// (a multiple of kPsWin) exponents, about kPsWaves blocks per SM in all (two
// resident at a time): short blocks, so that the SMs they free go to the
// tree's clusters beside them.
struct PsShape {
  int nb, nkb, kr;
};
PsShape ps_shape(int64_t T, int sms) {
  PsShape s;
  s.nb = (int)((T + kPsNodes - 1) / kPsNodes);
  int want = kPsWaves * sms / s.nb;
  if (want < 1) want = 1;
  int64_t kr = (T + want - 1) / want;
  kr = (kr + kPsWin - 1) / kPsWin * kPsWin;
  s.kr = (int)kr;
  s.nkb = (int)((T + kr - 1) / kr);
  return s;
}

// ---- the transposed problem: weighted power sums (the probe evaluator) ----------------
//
// out[s][i] = sum_g w_{g,s} u_g^i, i < T, is the expansion of
// sum_g w_{g,s} / (z - u_g) = N_s / M, M = prod_g (z - u_g): the transpose of
// the descent.  N_s is built bottom-up on the same subproduct tree,
// N_P = N_L M_R + N_R M_L (degree < deg P), and the expansion is
// rev(N_s) / rev(M) mod z^T.

// N_blk for every column s at a leaf block (the 128 roots of the block),
// by the pairwise levels of the block polynomial.
__device__ __forceinline__ uint64_t up_coef(const uint64_t* Nb, const uint64_t* Mb, int po, int a, int b, int kk,
                                            const Mod& M) {
  Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
  // N_L[i] (i < a) times the full right polynomial (degree b) at kk - i
  for (int i = (kk - b > 0 ? kk - b : 0); i <= (kk < a - 1 ? kk : a - 1); i++) {
    const int j = kk - i;
    const uint64_t x = Nb[po + i], y = j < b ? Mb[po + a + j] : 1;
    mac8(acc, lo32(x), hi32(x), lo32(y), hi32(y));
  }
  // N_R[i] (i < b) times the full left polynomial (degree a) at kk - i
  for (int i = (kk - a > 0 ? kk - a : 0); i <= (kk < b - 1 ? kk : b - 1); i++) {
    const int j = kk - i;
    const uint64_t x = Nb[po + a + i], y = j < a ? Mb[po + j] : 1;
    mac8(acc, lo32(x), hi32(x), lo32(y), hi32(y));
  }
  return acc8_value(acc, M);
}

__global__ void __launch_bounds__(kLeaf) k_up_leaf(const uint64_t* __restrict__ U, int64_t G,
                                                   const uint64_t* __restrict__ W, int64_t ldw, int S, Mod M,
                                                   uint64_t* __restrict__ N7, int64_t Gp) {
  pdl_enter();
  extern __shared__ uint64_t usm[];              // M [2][128], then N [S][2][128]
  uint64_t* Mb = usm;
  uint64_t* Nb = usm + 2 * kLeaf;
  const int64_t base = (int64_t)blockIdx.x * kLeaf;
  const int cnt = (int)((G - base) < kLeaf ? (G - base) : kLeaf);
  const int t = threadIdx.x;
  if (t < cnt) {
    const uint64_t x = U[base + t];
    Mb[t] = x ? M.p - x : 0;                     // z - u
    for (int c = 0; c < S; c++) Nb[c * 2 * kLeaf + t] = W[(int64_t)c * ldw + base + t];
  }
  __syncthreads();
  int cur = 0;
  for (int l = 0; l < kLeafLog; l++) {
    const int size = 1 << l, pair = 2 << l;
    if (t < cnt) {
      const int po = t & ~(pair - 1), kk = t - po;
      const uint64_t* Mc = Mb + cur * kLeaf;
      if (cnt - po <= size) {
        Mb[(cur ^ 1) * kLeaf + t] = Mc[t];
        for (int c = 0; c < S; c++) Nb[(c * 2 + (cur ^ 1)) * kLeaf + t] = Nb[(c * 2 + cur) * kLeaf + t];
      } else {
        const int a = size, b = min(size, cnt - po - size);
        Mb[(cur ^ 1) * kLeaf + t] = conv_coef(Mc, po, a, b, kk, M);
        for (int c = 0; c < S; c++)
          Nb[(c * 2 + (cur ^ 1)) * kLeaf + t] = up_coef(Nb + (c * 2 + cur) * kLeaf, Mc, po, a, b, kk, M);
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  if (t < cnt)
    for (int c = 0; c < S; c++) N7[(int64_t)c * Gp + base + t] = Nb[(c * 2 + cur) * kLeaf + t];
}

// Up level l <= kFusedLog, npc nodes of one column s per CTA: the children's
// numerators -> spectra -> N_L M_R + N_R M_L with the tree's spectra ->
// inverse -> N_P.
__global__ void __launch_bounds__(kFusedThreads) k_up_fused(const uint64_t* __restrict__ Nprev, int64_t G, int64_t Gp,
                                                            int logn, NttConsts C, CrtScale sc, Mod M,
                                                            const uint2* __restrict__ tw, int logN,
                                                            const uint32_t* __restrict__ spec,
                                                            uint64_t* __restrict__ Nout, int64_t nodes) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // [c][node][prime][n]
  const int npc = fused_npc(logn);
  const int64_t ctas = (nodes + npc - 1) / npc;
  const int64_t P0 = (int64_t)(blockIdx.x % ctas) * npc;
  const int col = (int)(blockIdx.x / ctas);
  const int n = 1 << logn, h = n >> 1;
  const int half = (npc * kNP) << logn;
  const uint64_t* src = Nprev + (int64_t)col * Gp;
  for (int e = threadIdx.x; e < 2 * npc * n; e += blockDim.x) {
    const int c = e / (npc * n), rest = e - c * npc * n;
    const int a = rest >> logn, k = rest & (n - 1);
    const int64_t child = 2 * (P0 + a) + c;
    int64_t d = G - child * h;
    d = d < 0 ? 0 : (d > h ? h : d);
    const uint64_t x = k < d ? src[child * h + k] : 0;
#pragma unroll
    for (int i = 0; i < kNP; i++) fsm[sw((((c * npc + a) * kNP + i) << logn) + k)] = k < d ? residue64(x, C, i) : 0u;
  }
  __syncthreads();
  smem_ntt<false>(fsm, 0, 2 * kNP * npc, logn, tw, logN, C);
  for (int e = threadIdx.x; e < half; e += blockDim.x) {
    const int t = e >> logn, k = e & (n - 1);
    const int a = t / kNP, i = t - a * kNP;
    const int64_t P = P0 + a;
    const uint32_t q = C.q[i], qi = C.qinv[i];
    uint32_t sL = 0, sR = 0;
    if (P < nodes) {
      const uint32_t* sp = spec + (int64_t)i * 2 * Gp + (2 * P << logn) + k;
      sL = sub_if(sp[0], 2 * q);
      sR = sub_if(sp[n], 2 * q);
    }
    const uint32_t z =
        mont32(sub_if(fsm[sw(e)], 2 * q), sR, q, qi) + mont32(sub_if(fsm[sw(half + e)], 2 * q), sL, q, qi);
    fsm[sw(e)] = z;                              // < 2q
  }
  __syncthreads();
  smem_ntt<true>(fsm, 0, npc * kNP, logn, tw + ((size_t)kNP << logN), logN, C);
  uint64_t* dst = Nout + (int64_t)col * Gp;
  for (int e = threadIdx.x; e < npc * n; e += blockDim.x) {
    const int a = e >> logn, k = e & (n - 1);
    const int64_t P = P0 + a;
    int64_t d = G - P * n;
    d = d < 0 ? 0 : (d > n ? n : d);
    if (k >= d) continue;
    uint32_t res[kNP];
#pragma unroll
    for (int i = 0; i < kNP; i++) res[i] = shoup32(fsm[sw(((a * kNP + i) << logn) + k)], sc.s[i], sc.sp[i], C.q[i]);
    dst[P * n + k] = crt_to_p(res, C, M);
  }
}

// Up level l <= kFusedLog on a cluster per (node P, column): the children's
// numerators (modulo prime `me`) -> spectra -> N_L M_R + N_R M_L with the
// tree's spectra -> inverse -> N_P (see the cluster levels of the solve).
__global__ void __launch_bounds__(kClusterThreadsMax) k_up_cluster(const uint64_t* __restrict__ Nprev, int64_t G,
                                                              int64_t Gp, int logn, NttConsts C, CrtScale sc, Mod M,
                                                              const uint2* __restrict__ tw, int logN,
                                                              const uint32_t* __restrict__ spec,
                                                              uint64_t* __restrict__ Nout, int64_t nodes) {
  pdl_enter();
  extern __shared__ uint32_t fsm[];              // N_L [n], N_R [n] (logical words)
  const int me = cluster_rank();
  const int64_t cl = blockIdx.x / kNP;
  const int64_t P = cl % nodes;
  const int col = (int)(cl / nodes);
  const int n = 1 << logn, h = n >> 1;
  const uint32_t q = C.q[me], qi = C.qinv[me];
  auto prime = [=](int) { return me; };
  const uint64_t* src = Nprev + (int64_t)col * Gp;
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    const int c = e >> logn, k = e & (n - 1);
    const int64_t child = 2 * P + c;
    int64_t d = G - child * h;
    d = d < 0 ? 0 : (d > h ? h : d);
    fsm[sw(e)] = k < d ? residue64(src[child * h + k], C, me) : 0u;
  }
  __syncthreads();
  smem_stages<false>(fsm, 0, 2 * n, logn, 0, 0u, tw, logN, C, prime);
  const uint32_t* sp = spec + (int64_t)me * 2 * Gp + (2 * P << logn);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t sL = sub_if(sp[k], 2 * q), sR = sub_if(sp[n + k], 2 * q);
    fsm[sw(k)] = mont32(sub_if(fsm[sw(k)], 2 * q), sR, q, qi) + mont32(sub_if(fsm[sw(n + k)], 2 * q), sL, q, qi);
  }
  __syncthreads();
  smem_stages<true>(fsm, 0, n, logn, 0, 0u, tw + ((size_t)kNP << logN), logN, C, prime);
  cluster_sync();
  int64_t d = G - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  const int per = (int)((d + kNP - 1) / kNP);
  const int lo = me * per, hi = (int)(d < (int64_t)lo + per ? d : (int64_t)lo + per);
  uint32_t peer[kNP];
#pragma unroll
  for (int j = 0; j < kNP; j++) peer[j] = cluster_addr(fsm, j);
  uint64_t* dst = Nout + (int64_t)col * Gp + P * n;
  for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    uint32_t res[kNP];
#pragma unroll
    for (int j = 0; j < kNP; j++) res[j] = shoup32(ld_cluster(peer[j] + 4u * sw(k)), sc.s[j], sc.sp[j], C.q[j]);
    dst[k] = crt_to_p(res, C, M);
  }
  cluster_sync();
}

// Up level l > kFusedLog in separate passes: A[s][i][(2P + c) n + k] (planes
// of 2 G'), forward transforms, Z[s][i][P n + k] = N_L M_R + N_R M_L (planes
// of G'), inverse transforms, then Chinese remaindering into N_P.
__global__ void k_up_load(const uint64_t* __restrict__ Nprev, int S, int64_t G, int64_t Gp, int logn, NttConsts C,
                          uint32_t* __restrict__ A) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over S * 2 G'
  if (idx >= (int64_t)S * 2 * Gp) return;
  const int col = (int)(idx / (2 * Gp));
  const int64_t e = idx - (int64_t)col * 2 * Gp;
  const int64_t n = 1ll << logn, h = n >> 1;
  const int64_t child = e >> logn, k = e & (n - 1);
  int64_t d = G - child * h;
  d = d < 0 ? 0 : (d > h ? h : d);
  const uint64_t x = k < d ? Nprev[(int64_t)col * Gp + child * h + k] : 0;
  uint32_t* out = A + (int64_t)col * kNP * 2 * Gp + e;
#pragma unroll
  for (int i = 0; i < kNP; i++) out[(int64_t)i * 2 * Gp] = k < d ? residue64(x, C, i) : 0u;
}
__global__ void k_up_mul(const uint32_t* __restrict__ A, const uint32_t* __restrict__ spec, int S, int64_t Gp, int logn,
                         NttConsts C, uint32_t* __restrict__ Z) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over kNP * G'
  if (idx >= (int64_t)kNP * Gp) return;
  const int i = (int)(idx / Gp);
  const int64_t e = idx - (int64_t)i * Gp;
  const uint32_t q = C.q[i], qi = C.qinv[i];
  const int64_t n = 1ll << logn;
  const int64_t P = e >> logn, k = e & (n - 1);
  const uint32_t* sp = spec + (int64_t)i * 2 * Gp + (2 * P << logn) + k;
  const uint32_t sL = sub_if(sp[0], 2 * q), sR = sub_if(sp[n], 2 * q);
  for (int col = 0; col < S; col++) {
    const uint32_t* a = A + ((int64_t)col * kNP + i) * 2 * Gp + (2 * P << logn) + k;
    const uint32_t z = mont32(sub_if(a[0], 2 * q), sR, q, qi) + mont32(sub_if(a[n], 2 * q), sL, q, qi);
    Z[((int64_t)col * kNP + i) * Gp + e] = z;
  }
}
__global__ void k_up_crt(const uint32_t* __restrict__ Z, int S, int64_t G, int64_t Gp, int logn, NttConsts C,
                         CrtScale sc, Mod M, uint64_t* __restrict__ Nout) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over S * G'
  if (idx >= (int64_t)S * Gp) return;
  const int col = (int)(idx / Gp);
  const int64_t e = idx - (int64_t)col * Gp;
  const int64_t n = 1ll << logn;
  const int64_t P = e >> logn, k = e & (n - 1);
  int64_t d = G - P * n;
  d = d < 0 ? 0 : (d > n ? n : d);
  if (k >= d) return;
  uint32_t res[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++)
    res[i] = shoup32(Z[((int64_t)col * kNP + i) * Gp + e], sc.s[i], sc.sp[i], C.q[i]);
  Nout[idx] = crt_to_p(res, C, M);
}

// The expansions: A[s][i][t] = N_s[G - 1 - t] (t < na), B = g (T terms), both
// transformed at size 2^logn; Z[s] = A[s] B; out[s][t] = Z[s][t], t < T.
__global__ void k_rows_load(const uint64_t* __restrict__ N, int S, int64_t G, int64_t Gp, int64_t na, int logn,
                            NttConsts C, uint32_t* __restrict__ A) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over S 2^logn
  if (idx >= ((int64_t)S << logn)) return;
  const int col = (int)(idx >> logn);
  const int64_t t = idx & ((1ll << logn) - 1);
  const uint64_t x = t < na ? N[(int64_t)col * Gp + G - 1 - t] : 0;
  uint32_t* out = A + ((int64_t)col * kNP << logn) + t;
#pragma unroll
  for (int i = 0; i < kNP; i++) out[(int64_t)i << logn] = t < na ? residue64(x, C, i) : 0u;
}
__global__ void k_rows_mul(uint32_t* __restrict__ A, const uint32_t* __restrict__ B, int S, int logn, NttConsts C) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over kNP 2^logn
  if (idx >= ((int64_t)kNP << logn)) return;
  const int i = (int)(idx >> logn);
  const uint32_t q = C.q[i], qi = C.qinv[i];
  const uint32_t b = sub_if(B[idx], 2 * q);
  for (int col = 0; col < S; col++) {
    uint32_t* a = A + ((int64_t)col * kNP << logn) + idx;
    *a = mont32(sub_if(*a, 2 * q), b, q, qi);
  }
}
__global__ void k_rows_crt(const uint32_t* __restrict__ Z, int S, int64_t T, int logn, NttConsts C, CrtScale sc,
                           Mod M, uint64_t* __restrict__ out, int64_t ldo) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over S T
  if (idx >= (int64_t)S * T) return;
  const int col = (int)(idx / T);
  const int64_t t = idx - (int64_t)col * T;
  uint32_t res[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++)
    res[i] = shoup32(Z[(((int64_t)col * kNP + i) << logn) + t], sc.s[i], sc.sp[i], C.q[i]);
  out[(int64_t)col * ldo + t] = crt_to_p(res, C, M);
}

// ---- host side ---------------------------------------------------------------------

uint32_t h_pow32(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  a %= q;
  while (e) {
    if (e & 1) r = r * a % q;
    a = a * a % q;
    e >>= 1;
  }
  return (uint32_t)r;
}
uint32_t h_shoup(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

constexpr uint32_t kPrimes[kNP] = {998244353u, 897581057u, 880803841u, 754974721u, 645922817u};
constexpr uint32_t kRoots[kNP] = {3u, 3u, 26u, 11u, 3u};

// 2^32 / n mod q_i (undoes one Montgomery factor and the inverse transform's n)
CrtScale crt_scale(int logn) {
  CrtScale s;
  for (int i = 0; i < kNP; i++) {
    const uint64_t q = kPrimes[i];
    const uint64_t ninv = h_pow32(h_pow32(2, (uint64_t)logn, q), q - 2, q);
    const uint32_t x = (uint32_t)(((uint64_t)1 << 32) % q * ninv % q);
    s.s[i] = x;
    s.sp[i] = h_shoup(x, (uint32_t)q);
  }
  return s;
}

// Transforms of count runs of 2^logn residues (see above).  With the
// context's profiler on, each tile launch is timed as phase PH_NTT with its
// butterflies (total / 2 per stage it runs) as the phase's work.
void launch_ntt(zr_ctx* ctx, uint32_t* data, int64_t count, int logn, int plane_log, bool inv, const uint2* tw,
                const uint2* itw, int logN, const NttConsts& C, cudaStream_t st) {
  if (logn <= 0 || count <= 0) return;
  const int64_t total = count << logn;
  const int L1 = logn > kNttTileLog ? logn - kNttTileLog : 0;
  const unsigned tiles = cdivu(total, kNttTile);
  const unsigned cols = (unsigned)(count << L1);
  auto local = [&](bool inverse) {
    cudaEvent_t a = prof_mark(ctx, st);
    if (inverse)
      launch_k(k_ntt_local<true>, tiles, kNttThreads, 0, st, data, total, logn, plane_log, L1, itw, logN, C);
    else
      launch_k(k_ntt_local<false>, tiles, kNttThreads, 0, st, data, total, logn, plane_log, L1, tw, logN, C);
    note_launch();
    cudaEvent_t b = prof_mark(ctx, st);
    prof_add(ctx, PH_NTT, a, b, (double)(total / 2) * (logn - L1));
  };
  if (!inv) {
    if (L1) {
      launch_k(k_ntt_cols<false>, cols, kNttThreads, 0, st, data, logn, plane_log, L1, tw, logN, C);
      note_launch();
    }
    local(false);
  } else {
    local(true);
    if (L1) {
      launch_k(k_ntt_cols<true>, cols, kNttThreads, 0, st, data, logn, plane_log, L1, itw, logN, C);
      note_launch();
    }
  }
}

// Workspace of one fast solve, carved in order.
struct FastWs {
  int64_t Tp = 0;
  int Lt = 0, R = 0;
  std::vector<uint64_t*> coef;     // levels 7 .. 7 + Lt, T' words each
  std::vector<uint32_t*> spec;     // levels 8 .. 7 + Lt, kNP * 2T' words each
  uint64_t *X0 = nullptr, *X1 = nullptr;   // R x T'
  uint32_t *XH = nullptr, *Y = nullptr;    // R kNP T', 2 R kNP T'
  uint64_t *f = nullptr, *rd = nullptr, *g = nullptr, *ps = nullptr, *e = nullptr;
  uint32_t *A = nullptr, *B = nullptr, *Z = nullptr;   // kNP * 2T' each
  uint64_t* psp = nullptr;         // k_power_sums' partial sums, T per node block (T <= kDirectPsMaxT)
  uint64_t* pss = nullptr;         // its starting powers, T per exponent block
};

// Up to this many unknowns the power sums come from k_power_sums (T^2 Shoup
// steps from the nodes alone, beside the tree) rather than from rev(M') /
// rev(M) after the tree.  Measured on GB300 (S = 21, whole solve): 0.31
// against 0.34 ms at T = 4096, 0.48 against 0.54 ms at T = 8192, 0.67
// against 0.81 ms at T = 10^4, but 0.95 against 0.86 ms at T = 16384, where
// the T^2 steps (0.33 ms alone) outgrow the cluster's Newton iteration.
constexpr int64_t kDirectPsMaxT = 12288;
// k_power_sums is shaped for at most this many SMs (its starting powers'
// workspace grows with the count)
constexpr int kPsSmsMax = 192;

FastWs carve_fast(Carver& cv, int64_t T, int R) {
  FastWs w;
  w.Lt = 0;
  while ((int64_t)kLeaf << w.Lt < T) w.Lt++;
  w.Tp = (int64_t)kLeaf << w.Lt;
  w.R = R;
  const int64_t Tp = w.Tp;
  for (int l = 0; l <= w.Lt; l++) w.coef.push_back(cv.take<uint64_t>(Tp));
  for (int l = 1; l <= w.Lt; l++) w.spec.push_back(cv.take<uint32_t>((size_t)kNP * 2 * Tp));
  w.X0 = cv.take<uint64_t>((size_t)R * Tp);
  w.X1 = cv.take<uint64_t>((size_t)R * Tp);
  w.XH = cv.take<uint32_t>((size_t)R * kNP * Tp);
  w.Y = cv.take<uint32_t>((size_t)2 * R * kNP * Tp);
  w.f = cv.take<uint64_t>(Tp + 1);
  w.rd = cv.take<uint64_t>(Tp);
  w.g = cv.take<uint64_t>(2 * Tp);
  w.ps = cv.take<uint64_t>(Tp);
  w.e = cv.take<uint64_t>(Tp);
  w.A = cv.take<uint32_t>((size_t)kNP * 2 * Tp);
  w.B = cv.take<uint32_t>((size_t)kNP * 2 * Tp);
  w.Z = cv.take<uint32_t>((size_t)kNP * 2 * Tp);
  if (T <= kDirectPsMaxT) w.psp = cv.take<uint64_t>((size_t)cdivu(T, kPsNodes) * T);
  if (T <= kDirectPsMaxT) w.pss = cv.take<uint64_t>((size_t)T * ps_shape(T, kPsSmsMax).nkb);
  return w;
}

void configure_fused();
bool newton_cluster_ok();
size_t newton_cluster_smem(int logK);
bool cluster_level(const zr_ctx* ctx, int logn, int64_t clusters);

struct FastRun {
  zr_ctx* ctx;
  const NttConsts& C;
  const Mod& M;
  const uint2 *tw, *itw;
  int logN;
  cudaStream_t st;
  // subproduct tree over the T roots v: coef[l] (levels 7 .. 7 + Lt, T' =
  // 128 2^Lt words each) and the children's spectra spec[l - 1] (kNP 2T'
  // words each); Z: kNP T' words of scratch.  Without `root` the top level
  // may stop at its children's spectra (coef[Lt], M itself, left unwritten
  // when that level runs on a cluster).
  void tree(const uint64_t* v, int64_t T, int64_t Tp, int Lt, const std::vector<uint64_t*>& coef,
            const std::vector<uint32_t*>& spec, uint32_t* Z, bool root = true);
  // g = 1 / f mod z^prec (f_0 = 1, nf coefficients): Newton's iteration, the
  // first steps in one CTA; g holds 2 prec words, e prec words, A, B, Z
  // kNP 2^ceil(log2(2 prec)) words each
  void inverse(const uint64_t* f, int64_t nf, int64_t prec, uint64_t* g, uint64_t* e, uint32_t* A, uint32_t* B,
               uint32_t* Z);
  // h = rd / f mod z^T (rd: T coefficients) in one cluster, when T fits it
  // (kNewtonSchool < T <= 2^kNewtonClusterLog); false: nothing was launched
  bool quotient(const uint64_t* f, int64_t nf, const uint64_t* rd, int64_t T, uint64_t* g, uint64_t* h);
  // out[t] = +-(a * b mod (z^N - 1))[lo + t], t < cnt; N = 2^logn
  void cyc(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int logn, int64_t lo, int64_t cnt, bool neg,
           uint32_t* A, uint32_t* B, uint32_t* Z, uint64_t* out) {
    const int64_t all = (int64_t)kNP << logn;
    launch_k(k_cyc_load, cdivu(all, 256), 256, 0, st, a, na, logn, C, A);
    launch_k(k_cyc_load, cdivu(all, 256), 256, 0, st, b, nb, logn, C, B);
    note_launches(2);
    launch_ntt(ctx, A, kNP, logn, logn, false, tw, itw, logN, C, st);
    launch_ntt(ctx, B, kNP, logn, logn, false, tw, itw, logN, C, st);
    launch_k(k_cyc_mul, cdivu(all, 256), 256, 0, st, A, B, logn, C, Z);
    note_launch();
    launch_ntt(ctx, Z, kNP, logn, logn, true, tw, itw, logN, C, st);
    launch_k(k_cyc_crt, cdivu(cnt, 256), 256, 0, st, Z, logn, lo, cnt, neg ? 1 : 0, C, crt_scale(logn), M, out);
    note_launch();
  }
};

// Launches `kernel` on `clusters` clusters of kNP CTAs.
template <class... P, class... A>
cudaError_t launch_cluster(void (*kernel)(P...), int64_t clusters, int threads, size_t smem, cudaStream_t st,
                           A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * kNP));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kNP;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
  note_launch();
  return e;
}

// Shared memory of k_newton_cluster for K = 2^logK: two swizzled buffers
// of up to K words (rounded to whole 32-word rows) and g mod q.
size_t newton_cluster_smem(int logK) {
  const size_t K = (size_t)1 << logK;
  return sizeof(uint32_t) * (((2 * K + 31) & ~(size_t)31) + K);
}

// Whether this device runs k_newton_cluster (a cluster of kNP CTAs with the
// largest shared memory it needs); else the single-CTA kernel runs.
bool newton_cluster_ok() {
  static DeviceValue ok;
  return ok.get([] {
           const size_t bytes = newton_cluster_smem(kNewtonClusterLog);
           if (cudaFuncSetAttribute(k_newton_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
               cudaSuccess) {
             (void)cudaGetLastError();
             return 2;
           }
           cudaLaunchConfig_t cfg = {};
           cfg.gridDim = dim3(kNP);
           cfg.blockDim = dim3(kNewtonThreadsF);
           cfg.dynamicSmemBytes = bytes;
           cudaLaunchAttribute attr[1];
           attr[0].id = cudaLaunchAttributeClusterDimension;
           attr[0].val.clusterDim.x = kNP;
           attr[0].val.clusterDim.y = 1;
           attr[0].val.clusterDim.z = 1;
           cfg.attrs = attr;
           cfg.numAttrs = 1;
           int clusters = 0;
           if (cudaOccupancyMaxActiveClusters(&clusters, k_newton_cluster, &cfg) != cudaSuccess) {
             (void)cudaGetLastError();
             return 2;
           }
           return clusters > 0 ? 1 : 2;
         }) == 1;
}

// Whether a level of `clusters` clusters at transform size 2^logn takes the
// cluster kernels.
bool cluster_level(const zr_ctx* ctx, int logn, int64_t clusters) {
  if (!newton_cluster_ok() || logn > kClusterMaxLog) return false;
  return logn <= kFusedLog || clusters * kNP <= 2 * (int64_t)ctx->sms;
}

void configure_fused() {
  static DeviceOnce fused_attr;
  fused_attr.run([] {
    const int bytes = (int)(sizeof(uint32_t) * 2 * kNP * kFusedMax);
    cudaFuncSetAttribute(k_tree_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_desc_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_up_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_newton_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    const int c2 = (int)(sizeof(uint32_t) * 2 << kClusterMaxLog), c3 = (int)(sizeof(uint32_t) * 3 << kClusterMaxLog);
    cudaFuncSetAttribute(k_tree_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, c2);
    cudaFuncSetAttribute(k_desc_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, c3);
    cudaFuncSetAttribute(k_up_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, c2);
    cudaFuncSetAttribute(k_up_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(uint64_t) * 2 * kLeaf * (1 + kFastProbeMaxS)));
  });
}

void FastRun::tree(const uint64_t* v, int64_t T, int64_t Tp, int Lt, const std::vector<uint64_t*>& coef,
                   const std::vector<uint32_t*>& spec, uint32_t* Z, bool root) {
  const int logT = kLeafLog + Lt;
  launch_k(k_fast_leafpoly, cdivu(T, kLeaf), kLeaf, 0, st, v, T, M, coef[0]);
  note_launch();
  for (int l = 1; l <= Lt; l++) {
    const int logn = kLeafLog + l;
    uint32_t* sp = spec[l - 1];
    const int64_t nodes = (T + (1ll << logn) - 1) >> logn;
    if (cluster_level(ctx, logn, nodes)) {
      const cudaError_t e = launch_cluster(k_tree_cluster, nodes, cluster_threads(logn), sizeof(uint32_t) * 2 << logn,
                                           st, coef[l - 1], T, Tp, logn, C, crt_scale(logn), M, tw, logN, sp,
                                           (l == Lt && !root) ? (uint64_t*)nullptr : coef[l]);
      if (e == cudaSuccess) continue;
      (void)cudaGetLastError();
    }
    if (logn <= kFusedLog) {
      const int npc = fused_npc(logn);
      launch_k(k_tree_fused, (unsigned)((nodes + npc - 1) / npc), kFusedThreads, sizeof(uint32_t) * 2 * kNP * npc << logn, st, coef[l - 1], T, Tp, logn, C, crt_scale(logn), M,
                                                                     tw, logN, sp, coef[l], nodes);
      note_launch();
      continue;
    }
    launch_k(k_tree_load, cdivu(kNP * 2 * Tp, 256), 256, 0, st, coef[l - 1], T, Tp, logn, C, sp);
    note_launch();
    launch_ntt(ctx, sp, (kNP * 2 * Tp) >> logn, logn, logT + 1, false, tw, itw, logN, C, st);
    launch_k(k_tree_mul, cdivu(kNP * Tp, 256), 256, 0, st, sp, Tp, logn, C, Z);
    note_launch();
    launch_ntt(ctx, Z, (kNP * Tp) >> logn, logn, logT, true, tw, itw, logN, C, st);
    launch_k(k_tree_crt, cdivu(Tp, 256), 256, 0, st, Z, T, Tp, logn, C, crt_scale(logn), M, coef[l]);
    note_launch();
  }
}

bool FastRun::quotient(const uint64_t* f, int64_t nf, const uint64_t* rd, int64_t T, uint64_t* g, uint64_t* h) {
  const int logK = ilog2(T);
  if (T <= kNewtonSchool || logK > kNewtonClusterLog || !newton_cluster_ok()) return false;
  if (launch_cluster(k_newton_cluster, 1, kNewtonThreadsF, newton_cluster_smem(logK), st, f, nf, logK, C, M, tw, logN,
                     g, rd, T, h) == cudaSuccess)
    return true;
  (void)cudaGetLastError();
  return false;
}

void FastRun::inverse(const uint64_t* f, int64_t nf, int64_t prec, uint64_t* g, uint64_t* e, uint32_t* A,
                      uint32_t* B, uint32_t* Z) {
  int logK0 = std::min(ilog2(prec), kNewtonClusterLog);
  bool done = false;
  if (newton_cluster_ok()) {
    done = launch_cluster(k_newton_cluster, 1, kNewtonThreadsF, newton_cluster_smem(logK0), st, f, nf, logK0, C, M,
                          tw, logN, g, (const uint64_t*)nullptr, (int64_t)0, (uint64_t*)nullptr) == cudaSuccess;
    if (!done) (void)cudaGetLastError();
  }
  if (!done) {
    logK0 = std::min(logK0, kFusedLog);
    launch_k(k_newton_fused, 1, kNewtonThreadsF, sizeof(uint32_t) * 2 * kNP << logK0, st, f, nf, logK0, C, M, tw, logN, g,
                                                                                  e);
    note_launch();
  }
  for (int64_t k = 1ll << logK0; k < prec; k *= 2) {
    const int logk2 = ilog2(2 * k);
    const int64_t fn = std::min<int64_t>(2 * k, nf);
    // e = f g: its coefficients k .. 2k-1 (the low ones are 1, 0, ..)
    cyc(f, fn, g, k, logk2, k, k, false, A, B, Z, e);
    // g_{k..2k} = -(g e_hi mod z^k)
    cyc(g, k, e, k, logk2, 0, k, true, A, B, Z, g + k);
  }
}

// Workspace of the fast evaluator, carved in order: the tree over the G'
// padded roots, the numerators (two ping-pong sets of S rows), the transform
// planes of the up levels and of the final products, Newton's buffers.
struct ProbeWs {
  int64_t Gp = 0, Pp = 0;
  int Lt = 0, logR = 0;
  std::vector<uint64_t*> coef;
  std::vector<uint32_t*> spec;
  uint64_t *N0 = nullptr, *N1 = nullptr, *f = nullptr, *g = nullptr, *e = nullptr;
  uint32_t *A = nullptr, *Z = nullptr, *Bg = nullptr, *A2 = nullptr, *B2 = nullptr, *Z2 = nullptr;
};

ProbeWs carve_probes(Carver& cv, int64_t G, int64_t T, int S) {
  ProbeWs w;
  while ((int64_t)kLeaf << w.Lt < G) w.Lt++;
  w.Gp = (int64_t)kLeaf << w.Lt;
  w.Pp = 1;
  while (w.Pp < T) w.Pp *= 2;
  w.logR = ilog2(2 * w.Pp);
  const int64_t Gp = w.Gp, R2 = 2 * w.Pp;
  for (int l = 0; l <= w.Lt; l++) w.coef.push_back(cv.take<uint64_t>(Gp));
  for (int l = 1; l <= w.Lt; l++) w.spec.push_back(cv.take<uint32_t>((size_t)kNP * 2 * Gp));
  w.N0 = cv.take<uint64_t>((size_t)S * Gp);
  w.N1 = cv.take<uint64_t>((size_t)S * Gp);
  // up levels: S kNP 2G' (children) and S kNP G' (products); the final
  // products reuse A (S kNP 2P' words)
  w.A = cv.take<uint32_t>((size_t)S * kNP * std::max(2 * Gp, R2));
  w.Z = cv.take<uint32_t>((size_t)std::max<int64_t>(S, 1) * kNP * Gp);
  w.Bg = cv.take<uint32_t>((size_t)kNP * R2);
  w.f = cv.take<uint64_t>(Gp + 1);
  w.g = cv.take<uint64_t>(R2);
  w.e = cv.take<uint64_t>(w.Pp);
  w.A2 = cv.take<uint32_t>((size_t)kNP * R2);
  w.B2 = cv.take<uint32_t>((size_t)kNP * R2);
  w.Z2 = cv.take<uint32_t>((size_t)kNP * std::max(R2, Gp));
  return w;
}

}  // namespace

// ---- entry points used by the batch ------------------------------------------------

size_t fast_ws_need(int64_t T, int R) {
  Carver m0(nullptr);
  carve_fast(m0, T, R);
  return m0.off + 256;
}

int fast_ntt_log(int64_t T) {
  int Lt = 0;
  while ((int64_t)kLeaf << Lt < T) Lt++;
  return kLeafLog + Lt + 1;           // the final power-sum product has size 2T'
}

NttConsts make_ntt_consts(uint64_t p) {
  NttConsts C;
  memset(&C, 0, sizeof(C));
  typedef unsigned __int128 u128;
  for (int i = 0; i < kNP; i++) {
    const uint32_t q = kPrimes[i];
    C.q[i] = q;
    C.g[i] = kRoots[i];
    uint32_t inv = 1;   // q^-1 mod 2^32 by Newton's iteration on 2-adic digits
    for (int it = 0; it < 5; it++) inv *= 2u - q * inv;
    C.qinv[i] = inv;
    C.r32[i] = (uint32_t)((((uint64_t)1) << 32) % q);
    C.r32p[i] = h_shoup(C.r32[i], q);
    C.onep[i] = h_shoup(1, q);
    for (int j = 0; j < i; j++) {
      C.gc[i][j] = h_pow32(kPrimes[j], q - 2, q);
      C.gcp[i][j] = h_shoup(C.gc[i][j], q);
    }
    u128 pre = 1;
    for (int j = 0; j < i; j++) pre = pre * kPrimes[j] % p;
    C.pre[i] = (uint64_t)pre;
  }
  return C;
}

// The tables for transforms up to 2^logN, grown on demand (context-owned).
zr_status ensure_ntt_tables(zr_ctx* ctx, int logN, cudaStream_t st) {
  if (ctx->ntt_logN >= logN) return ZR_OK;
  if (logN > kNttMaxLog) return set_err(ctx, ZR_ERR_INVALID_ARG, "fast solve: transform too large");
  if (ctx->ntt_tw) {
    // the old tables may be in use on any stream of the context (probe
    // lanes, fast streams): wait for the whole device before freeing them
    cudaDeviceSynchronize();
    cudaFree(ctx->ntt_tw);
    ctx->ntt_tw = nullptr;
    ctx->ntt_logN = 0;
  }
  const size_t words = (size_t)kNP << logN;
  cudaError_t e = cudaMalloc(&ctx->ntt_tw, 2 * words * sizeof(uint2));
  if (e != cudaSuccess) {
    ctx->ntt_tw = nullptr;
    return cuda_err(ctx, e, "transform tables");
  }
  uint2* tw = reinterpret_cast<uint2*>(ctx->ntt_tw);
  launch_k(k_ntt_tables, cdivu((int64_t)words, 256), 256, 0, st, logN, ctx->ntt, tw, tw + words);
  note_launch();
  ctx->ntt_logN = logN;
  return cuda_err(ctx, cudaGetLastError(), "transform tables");
}

// The transform tables for fast solves of up to T unknowns (grown here, on
// st, so that solves enqueued on other streams afterwards never grow them).
zr_status fast_tables_for(zr_ctx* ctx, int64_t T, cudaStream_t st) {
  int Lt = 0;
  while ((int64_t)kLeaf << Lt < T) Lt++;
  return ensure_ntt_tables(ctx, kLeafLog + Lt + 1, st);
}

// One system (or step entry) solved by the fast path: writes the numerators
// <q_j, b_s> to part[s T + j] (s < S) and M'(v_j) to den[j], the layout the
// finish kernels read for a single k-block.  v and vp (Shoup quotients of v)
// are on the device already; ws holds fast_ws_need(T, S + 1) bytes.
zr_status fast_solve_enqueue(zr_ctx* ctx, int64_t T, int S, const uint64_t* v, const uint64_t* vp,
                             const uint64_t* b, int64_t ldb, uint64_t* part, uint64_t* den, char* ws,
                             cudaStream_t st, cudaStream_t aux, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  const int R = S + 1;
  Carver cv(ws);
  FastWs w = carve_fast(cv, T, R);
  const int64_t Tp = w.Tp;
  const int Lt = w.Lt;
  const int logT = kLeafLog + Lt;
  zr_status r = ensure_ntt_tables(ctx, logT + 1, st);
  if (r) return r;
  const NttConsts& C = ctx->ntt;
  const Mod& M = ctx->M;
  const uint2* tw = reinterpret_cast<const uint2*>(ctx->ntt_tw);
  const uint2* itw = tw + ((size_t)kNP << ctx->ntt_logN);
  const int logN = ctx->ntt_logN;
  FastRun F{ctx, C, M, tw, itw, logN, st};

  configure_fused();
  // The right-hand sides' descent needs only the tree; the power sums' row
  // needs the power sums.  Up to kDirectPsMaxT unknowns they come from the
  // nodes alone: with an auxiliary stream (of the greatest priority) the tree
  // runs there and k_power_sums on st beside it, and one descent takes all
  // S + 1 rows.  Above, they need the tree's
  // root: with an auxiliary stream they and their row's descent run there,
  // beside the other rows' descent (each branch in its own rows of X and of
  // the scratch), joined at the leaves.  (With the context's profiler on,
  // everything runs on st, so that each timed launch has the GPU to itself.)
  const bool fork = aux != nullptr && ev_fork != nullptr && ev_join != nullptr && !ctx->prof.on;
  const bool direct_ps = w.psp != nullptr;
  cudaStream_t sa = fork ? aux : st;
  FastRun Fa{ctx, C, M, tw, itw, logN, sa};
  if (direct_ps) {
    if (fork) {
      cudaEventRecord(ev_fork, st);
      cudaStreamWaitEvent(sa, ev_fork, 0);
    }
    const PsShape ps = ps_shape(T, ctx->sms < kPsSmsMax ? ctx->sms : kPsSmsMax);
    launch_k(k_ps_start, cdivu(T, 256), 256, 0, st, v, T, ps.kr, ps.nkb, M, w.pss);
    cudaEvent_t pa = prof_mark(ctx, st);
    launch_k(k_power_sums, dim3((unsigned)ps.nkb, (unsigned)ps.nb), kPsThreads, 0, st, v, vp, T, ps.kr,
             (const uint64_t*)w.pss, M, w.psp);
    cudaEvent_t pb = prof_mark(ctx, st);
    prof_add(ctx, PH_PSUM, pa, pb, (double)T * (double)T);
    launch_k(k_power_sums_add, cdivu(T, 256), 256, 0, st, (const uint64_t*)w.psp, T, ps.nb, M, w.ps);
    note_launches(3);
    Fa.tree(v, T, Tp, Lt, w.coef, w.spec, w.Z, false);   // M itself is not needed: the descent takes its children
    if (fork) cudaEventRecord(ev_join, sa);
  } else {
    F.tree(v, T, Tp, Lt, w.coef, w.spec, w.Z);
  }
  const uint64_t* m = w.coef[Lt];   // M without its leading 1 (written on the Newton path only)
  // descent from the root (node size T') to the leaf blocks of nr rows from
  // row r0: every branch swaps X0 and X1 once per level
  auto descend = [&](int r0, int nr, cudaStream_t s) {
    uint64_t* X = w.X0 + (size_t)r0 * Tp;
    uint64_t* Xn = w.X1 + (size_t)r0 * Tp;
    uint32_t* XH = w.XH + (size_t)r0 * kNP * Tp;
    uint32_t* Y = w.Y + (size_t)2 * r0 * kNP * Tp;
    for (int l = Lt; l >= 1; l--) {
      const int logn = kLeafLog + l;
      const int64_t nodes = (T + (1ll << logn) - 1) >> logn;
      bool done = false;
      if (cluster_level(ctx, logn, nodes * nr)) {
        cudaEvent_t a = prof_mark(ctx, s);
        done = launch_cluster(k_desc_cluster, nodes * nr, cluster_threads(logn), sizeof(uint32_t) * 3 << logn, s, X,
                              T, Tp, logn, C, crt_scale(logn), M, tw, logN, w.spec[l - 1], Xn, nodes) == cudaSuccess;
        if (!done) (void)cudaGetLastError();
        cudaEvent_t b2 = prof_mark(ctx, s);
        // one forward and two inverse transforms of 2^logn per prime of each
        // cluster, but for a last node whose right child holds no roots (copied)
        const int64_t tx = nodes - ((T - (nodes - 1) * (1ll << logn)) <= (1ll << (logn - 1)) ? 1 : 0);
        if (done) prof_add(ctx, PH_DESC, a, b2, (double)(tx * nr) * kNP * 3 * (double)((1ll << logn) / 2) * logn);
      }
      if (!done && logn <= kFusedLog) {
        const int npc = fused_npc(logn);
        launch_k(k_desc_fused, (unsigned)((nodes + npc - 1) / npc * nr), kFusedThreads,
                 sizeof(uint32_t) * 2 * kNP * npc << logn, s, X, T, Tp, logn, C, crt_scale(logn), M, tw, logN,
                 w.spec[l - 1], Xn, nodes);
        note_launch();
        done = true;
      }
      if (!done) {
        const int64_t all = (int64_t)nr * kNP * Tp;
        launch_k(k_desc_load, cdivu((int64_t)nr * Tp, 256), 256, 0, s, X, nr, T, Tp, logn, C, XH);
        note_launch();
        launch_ntt(ctx, XH, all >> logn, logn, logT, false, tw, itw, logN, C, s);
        launch_k(k_desc_mul, cdivu((int64_t)kNP * Tp, 256), 256, 0, s, XH, w.spec[l - 1], nr, Tp, logn, C, Y);
        note_launch();
        launch_ntt(ctx, Y, (2 * all) >> logn, logn, logT, true, tw, itw, logN, C, s);
        launch_k(k_desc_crt, cdivu((int64_t)nr * Tp, 256), 256, 0, s, Y, nr, T, Tp, logn, C, crt_scale(logn), M,
                 Xn);
        note_launch();
      }
      std::swap(X, Xn);
    }
  };
  if (direct_ps) {
    // all R rows in one descent on the call's stream, once the power sums are in
    if (fork) cudaStreamWaitEvent(st, ev_join, 0);
    launch_k(k_stage_rhs, cdivu((int64_t)R * T, 256), 256, 0, st, b, ldb, S, (const uint64_t*)w.ps, 0, R, T, Tp,
             w.X0);
    note_launch();
    descend(0, R, st);
  } else {
    if (fork) {                     // the tree (spectra, M) before the auxiliary branch goes on
      cudaEventRecord(ev_fork, st);
      cudaStreamWaitEvent(sa, ev_fork, 0);
    }
    // the right-hand sides (rows 0 .. S-1) on the call's stream
    if (S > 0) {
      launch_k(k_stage_rhs, cdivu((int64_t)S * T, 256), 256, 0, st, b, ldb, S, (const uint64_t*)nullptr, 0, S, T,
               Tp, w.X0);
      note_launch();
      descend(0, S, st);
    }
    // power sums: ps = rev(M') / rev(M) mod z^T, up to 2^14 in one cluster
    // (Newton's iteration to half the precision, then a division step), else
    // g = 1 / rev(M) by Newton's iteration and ps = rev(M') g; then their row S
    launch_k(k_rev_poly, cdivu(T + 1, 256), 256, 0, sa, m, T, M, w.f, w.rd, w.g);
    note_launch();
    if (!Fa.quotient(w.f, T + 1, w.rd, T, w.g, w.ps)) {
      Fa.inverse(w.f, T + 1, T, w.g, w.e, w.A, w.B, w.Z);
      Fa.cyc(w.rd, T, w.g, T, logT + 1, 0, T, false, w.A, w.B, w.Z, w.ps);
    }
    launch_k(k_stage_rhs, cdivu(T, 256), 256, 0, sa, b, ldb, S, (const uint64_t*)w.ps, S, 1, T, Tp, w.X0);
    note_launch();
    descend(S, 1, sa);
    if (fork) {
      cudaEventRecord(ev_join, sa);
      cudaStreamWaitEvent(st, ev_join, 0);
    }
  }
  uint64_t* X = (Lt & 1) ? w.X1 : w.X0;     // where Lt swaps leave the rows
  // leaves
  launch_k(k_fast_leafval, dim3(cdivu(T, kLeaf), (unsigned)((R + kLeafCols - 1) / kLeafCols)), kLeaf, 0, st, 
      w.coef[0], X, R, T, Tp, v, vp, M, part, T, den);
  note_launch();
  return cuda_err(ctx, cudaGetLastError(), "fast solve");
}

size_t fast_probes_ws_need(int64_t G, int64_t T, int S) {
  Carver m0(nullptr);
  carve_probes(m0, G, T, S);
  return m0.off + 256;
}

// out[s ldo + i] = sum_{g < G} W[s ldw + g] U[g]^i, i < T (1 <= G, T <= 2^21,
// S <= 256): the tree over U, the numerators N_s bottom-up, Newton's inverse
// of rev(M) to precision T, and the S products rev(N_s) / rev(M) mod z^T.
zr_status fast_probes_enqueue(zr_ctx* ctx, int64_t G, const uint64_t* U, const uint64_t* W, int64_t ldw, int S,
                              int64_t T, uint64_t* out, int64_t ldo, char* ws, cudaStream_t st) {
  Carver cv(ws);
  ProbeWs w = carve_probes(cv, G, T, S);
  const int64_t Gp = w.Gp;
  const int Lt = w.Lt;
  const int logG = kLeafLog + Lt;
  zr_status r = ensure_ntt_tables(ctx, std::max(logG + 1, w.logR), st);
  if (r) return r;
  const NttConsts& C = ctx->ntt;
  const Mod& M = ctx->M;
  const uint2* tw = reinterpret_cast<const uint2*>(ctx->ntt_tw);
  const uint2* itw = tw + ((size_t)kNP << ctx->ntt_logN);
  const int logN = ctx->ntt_logN;
  FastRun F{ctx, C, M, tw, itw, logN, st};
  configure_fused();
  F.tree(U, G, Gp, Lt, w.coef, w.spec, w.Z2);

  // numerators: leaf blocks, then the levels up to the root
  launch_k(k_up_leaf, cdivu(G, kLeaf), kLeaf, sizeof(uint64_t) * 2 * kLeaf * (1 + S), st, U, G, W, ldw, S, M, w.N0, Gp);
  note_launch();
  uint64_t* Nc = w.N0;
  uint64_t* Nn = w.N1;
  for (int l = 1; l <= Lt; l++) {
    const int logn = kLeafLog + l;
    const int64_t nodes = (G + (1ll << logn) - 1) >> logn;
    bool done = false;
    if (cluster_level(ctx, logn, nodes * S)) {
      done = launch_cluster(k_up_cluster, nodes * S, cluster_threads(logn), sizeof(uint32_t) * 2 << logn, st, Nc, G,
                            Gp, logn, C, crt_scale(logn), M, tw, logN, w.spec[l - 1], Nn, nodes) == cudaSuccess;
      if (!done) (void)cudaGetLastError();
    }
    if (!done && logn <= kFusedLog) {
      const int npc = fused_npc(logn);
      launch_k(k_up_fused, (unsigned)((nodes + npc - 1) / npc * S), kFusedThreads, sizeof(uint32_t) * 2 * kNP * npc << logn, st, Nc, G, Gp, logn, C, crt_scale(logn), M, tw, logN,
                                                                   w.spec[l - 1], Nn, nodes);
      note_launch();
      done = true;
    }
    if (!done) {
      launch_k(k_up_load, cdivu((int64_t)S * 2 * Gp, 256), 256, 0, st, Nc, S, G, Gp, logn, C, w.A);
      note_launch();
      launch_ntt(ctx, w.A, ((int64_t)S * kNP * 2 * Gp) >> logn, logn, logG + 1, false, tw, itw, logN, C, st);
      launch_k(k_up_mul, cdivu((int64_t)kNP * Gp, 256), 256, 0, st, w.A, w.spec[l - 1], S, Gp, logn, C, w.Z);
      note_launch();
      launch_ntt(ctx, w.Z, ((int64_t)S * kNP * Gp) >> logn, logn, logG, true, tw, itw, logN, C, st);
      launch_k(k_up_crt, cdivu((int64_t)S * Gp, 256), 256, 0, st, w.Z, S, G, Gp, logn, C, crt_scale(logn), M, Nn);
      note_launch();
    }
    std::swap(Nc, Nn);
  }

  // 1 / rev(M) to precision T, then rev(N_s) times it, the first T terms
  launch_k(k_rev_poly, cdivu(G + 1, 256), 256, 0, st, w.coef[Lt], G, M, w.f, nullptr, w.g);
  note_launch();
  F.inverse(w.f, G + 1, T, w.g, w.e, w.A2, w.B2, w.Z2);
  const int logR = w.logR;
  const int64_t na = std::min(G, T);
  launch_k(k_rows_load, cdivu((int64_t)S << logR, 256), 256, 0, st, Nc, S, G, Gp, na, logR, C, w.A);
  note_launch();
  launch_k(k_cyc_load, cdivu((int64_t)kNP << logR, 256), 256, 0, st, w.g, T, logR, C, w.Bg);
  note_launch();
  launch_ntt(ctx, w.A, (int64_t)S * kNP, logR, logR, false, tw, itw, logN, C, st);
  launch_ntt(ctx, w.Bg, kNP, logR, logR, false, tw, itw, logN, C, st);
  launch_k(k_rows_mul, cdivu((int64_t)kNP << logR, 256), 256, 0, st, w.A, w.Bg, S, logR, C);
  note_launch();
  launch_ntt(ctx, w.A, (int64_t)S * kNP, logR, logR, true, tw, itw, logN, C, st);
  launch_k(k_rows_crt, cdivu((int64_t)S * T, 256), 256, 0, st, w.A, S, T, logR, C, crt_scale(logR), M, out, ldo);
  note_launch();
  return cuda_err(ctx, cudaGetLastError(), "fast probes");
}

}  // namespace zr
