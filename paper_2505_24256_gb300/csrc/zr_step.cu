// zr_step.cu -- kernels of the Zippel step (Sec. 1, Sec. 2.2).
//
//   anchor values + node check   v_j = prod_{m<k} y_m^{e_{j,m}}, distinct   (a2)
//   master polynomial            M(z) = prod_j (z - v_j)                    (a3)
//   synthetic division + dots    acc[s][j] = sum_k q_{j,k} b[s][k],
//                                q_{j,k-1} = m_k + v_j q_{j,k}, den_j = q_j(v_j)   (a4, a5)
//   finish                       c[s][j] = acc[s][j] / den_j (batch inverse)
//   Newton in the new variable   divided differences, monomial form, compaction (a6)
#include <cuda_runtime.h>

#include "zr_kernels.cuh"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
static constexpr uint64_t kEmpty = ~0ull;

// ---------------------------------------------------------------------------
// a2: per-variable power tables y_m^e (the paper's power table, Sec. 2.2) and
// anchor values.
// ---------------------------------------------------------------------------

__global__ void k_powtab(const uint64_t* __restrict__ y, int k, Mod M, uint64_t* __restrict__ tab) {
  int m = blockIdx.x, e = threadIdx.x;
  if (m < k && e < kPowTab) tab[m * kPowTab + e] = pow_mod(y[m], (uint64_t)e, M);
}

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
    unsigned long long prev = atomicCAS((unsigned long long*)&htab[idx], (unsigned long long)kEmpty,
                                        (unsigned long long)x);
    if (prev == kEmpty) return;
    if (prev == x) { atomicOr(status, ST_DUP_NODE); return; }
    idx = (idx + 1) & hmask;
  }
  atomicOr(status, ST_HASH_FULL);
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
// a3: master polynomial by a product tree.  Level l holds monic polynomials
// of degree 2^l (the last one may be shorter) without their leading 1; the
// polynomial covering leaves [g 2^l, ...) keeps its coefficients at the same
// offset, so every level is an array of T words.
// ---------------------------------------------------------------------------

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

constexpr int kTreeL1 = 10;  // levels 0..9 inside one CTA (1024 leaves)

__global__ void __launch_bounds__(512) k_tree_leaf(int64_t T, const uint64_t* __restrict__ v, Mod M,
                                                   uint64_t* __restrict__ out) {
  __shared__ uint64_t buf[2][1 << kTreeL1];
  const int64_t base = (int64_t)blockIdx.x << kTreeL1;
  const int n = (int)((T - base) < (1 << kTreeL1) ? (T - base) : (1 << kTreeL1));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    uint64_t x = v[base + i];
    buf[0][i] = x ? M.p - x : 0;           // z - v_j
  }
  __syncthreads();
  int cur = 0;
  for (int l = 0; l < kTreeL1; l++) {
    const int size = 1 << l, pair = 2 << l;
    for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
      int po = pos & ~(pair - 1), nn = pos - po;
      uint64_t r;
      if (n - po <= size) r = buf[cur][pos];                         // no right child
      else r = conv_coef(buf[cur], po, size, min(size, n - po - size), nn, M);
      buf[cur ^ 1][pos] = r;
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[base + i] = buf[cur][i];
}

// One level l >= kTreeL1: a CTA computes NO consecutive outputs with NS
// slices of the inner index each, staging the factors in shared memory.
constexpr int kNO = 64, kNS = 4, kIC = 256;
__global__ void __launch_bounds__(kNO* kNS) k_tree_level(int64_t T, int l, const uint64_t* __restrict__ in, Mod M,
                                                         uint64_t* __restrict__ out) {
  __shared__ uint64_t As[kIC];
  __shared__ uint64_t Bw[kIC + kNO];
  __shared__ uint64_t red[kNS][kNO];
  const int64_t t0 = (int64_t)blockIdx.x * kNO;
  if (t0 >= T) return;
  const int64_t size = 1ll << l, pair = 2ll << l;
  const int64_t po = t0 & ~(pair - 1);
  const int tid = threadIdx.x, o = tid % kNO, sl = tid / kNO;
  if (T - po <= size) {                                              // no right child: copy
    if (sl == 0 && t0 + o < T) out[t0 + o] = in[t0 + o];
    return;
  }
  const int64_t a = size, b = (T - po - size) < size ? (T - po - size) : size;
  const int64_t n0 = t0 - po;
  const int64_t nmax = a + b;                                        // outputs n < a + b
  const int64_t ilo = n0 - b > 0 ? n0 - b : 0;
  const int64_t ihi = (n0 + kNO - 1) < a ? (n0 + kNO - 1) : a;      // inclusive
  Acc3 acc = {0, 0, 0};
  for (int64_t i0 = ilo; i0 <= ihi; i0 += kIC) {
    __syncthreads();
    for (int t = tid; t < kIC; t += blockDim.x) {
      int64_t i = i0 + t;
      As[t] = (i < a) ? in[po + i] : (i == a ? 1 : 0);
    }
    // window: j = n0 + o - i for o in [0, NO), i in [i0, i0 + IC): j in [n0 - i0 - IC + 1, n0 - i0 + NO - 1]
    const int64_t jlo = n0 - i0 - kIC + 1;
    for (int t = tid; t < kIC + kNO - 1; t += blockDim.x) {
      int64_t jj = jlo + t;
      Bw[t] = (jj < 0 || jj > b) ? 0 : (jj == b ? 1 : in[po + a + jj]);
    }
    __syncthreads();
    for (int t = sl; t < kIC; t += kNS) {
      // i = i0 + t, j = n0 + o - i  ->  window index o - t + IC - 1
      mac128(acc, As[t], Bw[o - t + kIC - 1]);
    }
  }
  __syncthreads();
  uint64_t r = acc3_value(acc, M);
  red[sl][o] = r;
  __syncthreads();
  if (sl == 0 && n0 + o < nmax && t0 + o < T) {
    uint64_t s = red[0][o];
    for (int q = 1; q < kNS; q++) s = add_mod(s, red[q][o], M);
    out[t0 + o] = s;
  }
}

void launch_master_poly(int64_t T, const uint64_t* v, const Mod& M, uint64_t* m, uint64_t* tmp, cudaStream_t st) {
  if (T <= 0) return;
  int64_t levels = 0;
  while ((1ll << levels) < T) levels++;
  uint64_t* bufs[2] = {tmp, tmp + T};
  int cur = 0;
  uint64_t* dst = levels <= kTreeL1 ? m : bufs[cur];
  { k_tree_leaf<<<cdiv(T, 1 << kTreeL1), 512, 0, st>>>(T, v, M, dst); note_launch(); }
  const uint64_t* src = dst;
  for (int l = kTreeL1; l < levels; l++) {
    uint64_t* o = (l == levels - 1) ? m : bufs[cur ^ 1];
    { k_tree_level<<<cdiv(T, kNO), kNO * kNS, 0, st>>>(T, l, src, M, o); note_launch(); }
    src = o;
    cur ^= 1;
  }
}

// ---------------------------------------------------------------------------
// Right-hand sides in MAC form: bx[k S + s] = make_bx(b[s][k]).
// ---------------------------------------------------------------------------

__global__ void k_expand_b(int64_t T, int S, const uint64_t* __restrict__ b, int64_t ldb, Mod M,
                           BX* __restrict__ bx) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * S) return;
  int64_t k = idx / S;
  int s = (int)(idx - k * S);
  uint64_t x = b[s * ldb + k];
  if (x >= M.p) x -= M.p;   // tolerate one extra p: inputs are documented canonical
  bx[idx] = make_bx(x, M);
}

void launch_expand_b(int64_t T, int S, const uint64_t* b, int64_t ldb, const Mod& M, BX* bx, cudaStream_t st) {
  if (T > 0 && S > 0) { k_expand_b<<<cdiv(T * S, 256), 256, 0, st>>>(T, S, b, ldb, M, bx); note_launch(); }
}

// ---------------------------------------------------------------------------
// Finish: combine the k-block partials, invert the denominators of a warp
// with one inversion (Montgomery's trick, prefix/suffix products by shuffle),
// scale.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t combine_den(int64_t j, int64_t T, int NB, int64_t BK, int offset, uint64_t vj,
                                                const uint64_t* __restrict__ denp, const Mod& M) {
  // den = sum_kb U_kb v^{kb BK}
  uint64_t den = 0, pw = 1;
  const uint64_t vBK = NB > 1 ? pow_mod(vj, (uint64_t)BK, M) : 1;
  for (int kb = 0; kb < NB; kb++) {
    den = add_mod(den, mul_mod(denp[(int64_t)kb * T + j], pw, M), M);
    pw = mul_mod(pw, vBK, M);
  }
  if (offset == 1) den = mul_mod(den, vj, M);
  return den;
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

__global__ void __launch_bounds__(256) k_finish_solve(int64_t T, int S, int NB, int64_t BK, int offset,
                                                      const uint64_t* __restrict__ v,
                                                      const uint64_t* __restrict__ part,
                                                      const uint64_t* __restrict__ denp, Mod M,
                                                      uint64_t* __restrict__ c, int64_t ldc, uint32_t* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < T;
  uint64_t den = 1;
  if (active) {
    den = combine_den(j, T, NB, BK, offset, v[j], denp, M);
    if (den == 0) atomicOr(status, ST_ZERO_DEN);
  }
  const uint64_t inv = warp_batch_inverse(den, M);
  if (!active) return;
  for (int s = 0; s < S; s++) {
    uint64_t num = 0;
    for (int kb = 0; kb < NB; kb++) num = add_mod(num, part[((int64_t)kb * S + s) * T + j], M);
    c[s * ldc + j] = mul_mod(num, inv, M);
  }
}

void launch_finish_solve(const StepDims& D, int offset, const uint64_t* v, const uint64_t* part,
                         const uint64_t* denp, const Mod& M, uint64_t* c, int64_t ldc, uint32_t* status,
                         cudaStream_t st) {
  if (D.T > 0) { k_finish_solve<<<cdiv(D.T, 256), 256, 0, st>>>(D.T, D.S, D.NB, D.BK, offset, v, part, denp, M, c, ldc, status); note_launch(); }
}

// ---------------------------------------------------------------------------
// a6: Newton in the new variable, Eq. (newton).
//   invd[l S + s] = 1 / (x_s - x_{s-l}),  1 <= l <= s < S   (shared by all terms)
//   a_s: divided differences; then the nested form a_0 + (z-x_0)[a_1 + ...]
//   expanded to monomial coefficients.
// ---------------------------------------------------------------------------

__global__ void k_newton_table(int S, const uint64_t* __restrict__ xs, Mod M, uint64_t* __restrict__ invd,
                               uint32_t* status) {
  for (int idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
    int l = idx / S, s = idx - l * S;
    if (l >= 1 && s >= l) {
      uint64_t d = sub_mod(xs[s], xs[s - l], M);
      if (d == 0) atomicOr(status, ST_DUP_SAMPLE);
      invd[idx] = inv_mod(d, M);
    }
  }
}

void launch_newton_table(int S, const uint64_t* xs, const Mod& M, uint64_t* invd, uint32_t* status, cudaStream_t st) {
  { k_newton_table<<<1, 256, 0, st>>>(S, xs, M, invd, status); note_launch(); }
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

template <int SMAX>
__global__ void __launch_bounds__(128) k_finish_newton(int64_t T, int S, int NB, int64_t BK, int offset,
                                                       const uint64_t* __restrict__ v,
                                                       const uint64_t* __restrict__ part,
                                                       const uint64_t* __restrict__ denp,
                                                       const uint64_t* __restrict__ xs,
                                                       const uint64_t* __restrict__ invd, Mod M,
                                                       uint64_t* __restrict__ g, int32_t* __restrict__ cnt,
                                                       uint32_t* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j < T;
  uint64_t den = 1;
  if (active) {
    den = combine_den(j, T, NB, BK, offset, v[j], denp, M);
    if (den == 0) atomicOr(status, ST_ZERO_DEN);
  }
  const uint64_t inv = warp_batch_inverse(den, M);
  if (!active) return;
  uint64_t a[SMAX];
#pragma unroll
  for (int s = 0; s < SMAX; s++) {
    a[s] = 0;
    if (s < S) {
      uint64_t num = 0;
      for (int kb = 0; kb < NB; kb++) num = add_mod(num, part[((int64_t)kb * S + s) * T + j], M);
      a[s] = mul_mod(num, inv, M);
    }
  }
  newton_any<SMAX>(a, S, xs, invd, M);
  int n = 0;
#pragma unroll
  for (int e = 0; e < SMAX; e++)
    if (e < S) {
      g[(int64_t)e * T + j] = a[e];
      n += a[e] != 0;
    }
  cnt[j] = n;
}

void launch_finish_newton(const StepDims& D, int offset, const uint64_t* v, const uint64_t* part,
                          const uint64_t* denp, const uint64_t* xs, const uint64_t* invd, const Mod& M,
                          uint64_t* g, int32_t* cnt, uint32_t* status, cudaStream_t st) {
  if (D.T <= 0) return;
  const unsigned grid = cdiv(D.T, 128);
  if (D.S <= 8) { k_finish_newton<8><<<grid, 128, 0, st>>>(D.T, D.S, D.NB, D.BK, offset, v, part, denp, xs, invd, M, g, cnt, status); note_launch(); }
  else if (D.S <= 16) { k_finish_newton<16><<<grid, 128, 0, st>>>(D.T, D.S, D.NB, D.BK, offset, v, part, denp, xs, invd, M, g, cnt, status); note_launch(); }
  else if (D.S <= 32) { k_finish_newton<32><<<grid, 128, 0, st>>>(D.T, D.S, D.NB, D.BK, offset, v, part, denp, xs, invd, M, g, cnt, status); note_launch(); }
  else { k_finish_newton<64><<<grid, 128, 0, st>>>(D.T, D.S, D.NB, D.BK, offset, v, part, denp, xs, invd, M, g, cnt, status); note_launch(); }
}

template <int SMAX>
__global__ void __launch_bounds__(128) k_newton(int64_t nterms, int S, const uint64_t* __restrict__ xs,
                                                const uint64_t* __restrict__ invd,
                                                const uint64_t* __restrict__ vals, int64_t ld, Mod M,
                                                uint64_t* __restrict__ coef) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nterms) return;
  uint64_t a[SMAX];
#pragma unroll
  for (int s = 0; s < SMAX; s++) {
    a[s] = 0;
    if (s < S) {
      uint64_t x = vals[(int64_t)s * ld + j];
      a[s] = x >= M.p ? x - M.p : x;
    }
  }
  newton_any<SMAX>(a, S, xs, invd, M);
#pragma unroll
  for (int e = 0; e < SMAX; e++)
    if (e < S) coef[(int64_t)e * ld + j] = a[e];
}

void launch_newton(int64_t nterms, int npts, const uint64_t* xs, const uint64_t* invd, const uint64_t* vals,
                   int64_t ld, const Mod& M, uint64_t* coef, cudaStream_t st) {
  if (nterms <= 0) return;
  const unsigned grid = cdiv(nterms, 128);
  if (npts <= 8) { k_newton<8><<<grid, 128, 0, st>>>(nterms, npts, xs, invd, vals, ld, M, coef); note_launch(); }
  else if (npts <= 16) { k_newton<16><<<grid, 128, 0, st>>>(nterms, npts, xs, invd, vals, ld, M, coef); note_launch(); }
  else if (npts <= 32) { k_newton<32><<<grid, 128, 0, st>>>(nterms, npts, xs, invd, vals, ld, M, coef); note_launch(); }
  else { k_newton<64><<<grid, 128, 0, st>>>(nterms, npts, xs, invd, vals, ld, M, coef); note_launch(); }
}

// ---------------------------------------------------------------------------
// Compaction of the new skeleton: terms (exps_j with column k = e, g_{j,e})
// for g != 0, ordered by j then e.
// ---------------------------------------------------------------------------

constexpr int kScanB = 1024;
int64_t scan_blocks(int64_t n) { return (n + kScanB - 1) / kScanB; }

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

__global__ void __launch_bounds__(kScanB) k_block_sums(int64_t T, const int32_t* __restrict__ cnt,
                                                       int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[33];
  int64_t j = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  int64_t x = j < T ? cnt[j] : 0, total;
  block_exclusive_scan(x, sh, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanB) k_scan_bsum(int64_t nb, int64_t* __restrict__ bsum,
                                                      int64_t* __restrict__ out_count) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanB) {
    int64_t i = base + threadIdx.x;
    int64_t x = i < nb ? bsum[i] : 0, total;
    int64_t ex = block_exclusive_scan(x, sh, total);
    __syncthreads();
    if (i < nb) bsum[i] = ex + carry;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_count = carry;
}

__global__ void __launch_bounds__(kScanB) k_scatter(int64_t T, int S, int nv, int k,
                                                    const uint8_t* __restrict__ exps,
                                                    const uint64_t* __restrict__ g, const int32_t* __restrict__ cnt,
                                                    const int64_t* __restrict__ bsum, int64_t cap,
                                                    uint8_t* __restrict__ out_exps, uint64_t* __restrict__ out_coef) {
  __shared__ int64_t sh[33];
  int64_t j = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  int64_t x = j < T ? cnt[j] : 0, total;
  int64_t o = block_exclusive_scan(x, sh, total) + bsum[blockIdx.x];
  if (j >= T || x == 0) return;
  const uint8_t* e = exps + j * nv;
  for (int s = 0; s < S; s++) {
    uint64_t val = g[(int64_t)s * T + j];
    if (val == 0) continue;
    if (o < cap) {
      uint8_t* oe = out_exps + o * nv;
      for (int m = 0; m < nv; m++) oe[m] = m < k ? e[m] : 0;
      oe[k] = (uint8_t)s;
      out_coef[o] = val;
    }
    o++;
  }
}

void launch_compact(int64_t T, int S, int nv, int k, const uint8_t* exps, const uint64_t* g, const int32_t* cnt,
                    int64_t* bsum, int64_t cap, uint8_t* out_exps, uint64_t* out_coef, int64_t* out_count,
                    cudaStream_t st) {
  const int64_t nb = scan_blocks(T);
  if (T <= 0) {
    cudaMemsetAsync(out_count, 0, sizeof(int64_t), st);
    return;
  }
  { k_block_sums<<<(unsigned)nb, kScanB, 0, st>>>(T, cnt, bsum); note_launch(); }
  { k_scan_bsum<<<1, kScanB, 0, st>>>(nb, bsum, out_count); note_launch(); }
  { k_scatter<<<(unsigned)nb, kScanB, 0, st>>>(T, S, nv, k, exps, g, cnt, bsum, cap, out_exps, out_coef); note_launch(); }
}

}  // namespace zr
