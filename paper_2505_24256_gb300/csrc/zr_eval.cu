// zr_eval.cu -- sparse black-box evaluator (Sec. 2.2, balanced coefficient
// preparation: base values raised to powers and substituted into the
// polynomial; one value per thread, terms split over threads, partial sums
// added).
//
// The Zippel probes of f for new variable k are the values
//     out[s][i] = f(y^(i+off), c_s, z_{k+1..})
//               = sum_t w_{t,s} u_t^(i+off),
//     u_t = prod_{m<k} y_m^{e_{t,m}},  w_{t,s} = coef_t c_s^{e_{t,k}} prod_{m>k} z_m^{e_{t,m}}.
// Terms with equal u are merged first (their w are added), which turns the
// evaluation into a transposed Vandermonde product over the G distinct u.
// The kernel tiles it: a CTA owns a range of consecutive i and walks the
// groups in chunks; for each chunk it builds the table X[g][t] = u_g^(I0+off+t)
// in shared memory by doubling (the paper's stride-k power table, Sec. 2.2)
// and its thread groups accumulate sum_g w_{g,s} X[g][t] for their columns
// with the deferred multiply-accumulate.
#include <cuda_runtime.h>

#include "zr_internal.h"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
static constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ uint64_t ehash(uint64_t x) {
  x ^= x >> 31;
  x *= 0x9E3779B97F4A7C15ull;
  return x ^ (x >> 29);
}

// rows of power tables: base[r]^e for e < 256
__global__ void k_powrows(const uint64_t* __restrict__ base, int nrows, Mod M, uint64_t* __restrict__ tab) {
  int r = blockIdx.x, e = threadIdx.x;
  if (r < nrows) tab[(int64_t)r * kPowTab + e] = pow_mod(base[r] >= M.p ? base[r] - M.p : base[r], (uint64_t)e, M);
}

__global__ void k_eval_terms(int64_t Tf, int nv, const uint8_t* __restrict__ exps, const uint64_t* __restrict__ coef,
                             int k, const uint64_t* __restrict__ tabY, const uint64_t* __restrict__ tabZ,
                             const uint64_t* __restrict__ tabC, int S, Mod M, uint64_t* __restrict__ u,
                             uint64_t* __restrict__ w, uint64_t* htab, uint64_t hmask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tf) return;
  const uint8_t* e = exps + t * nv;
  uint64_t uu = 1;
  for (int m = 0; m < k; m++) uu = mul_mod(uu, tabY[m * kPowTab + e[m]], M);
  uint64_t c = coef[t];
  if (c >= M.p) c -= M.p;
  for (int m = k + 1; m < nv; m++) c = mul_mod(c, tabZ[m * kPowTab + e[m]], M);
  u[t] = uu;
  for (int s = 0; s < S; s++) w[t * S + s] = mul_mod(c, tabC[s * kPowTab + e[k]], M);
  // insert the key; equal keys share a slot
  uint64_t idx = ehash(uu) & hmask;
  for (uint64_t probe = 0; probe <= hmask; probe++) {
    unsigned long long prev = atomicCAS((unsigned long long*)&htab[idx], (unsigned long long)kEmpty,
                                        (unsigned long long)uu);
    if (prev == kEmpty || prev == uu) return;
    idx = (idx + 1) & hmask;
  }
}

__device__ __forceinline__ int64_t find_slot(uint64_t key, const uint64_t* htab, uint64_t hmask) {
  uint64_t idx = ehash(key) & hmask;
  for (uint64_t probe = 0; probe <= hmask; probe++) {
    uint64_t x = htab[idx];
    if (x == key) return (int64_t)idx;
    if (x == kEmpty) return -1;
    idx = (idx + 1) & hmask;
  }
  return -1;
}

// slot -> group id: exclusive scan of "slot used" flags
constexpr int kB = 1024;
__device__ __forceinline__ int64_t blk_scan(int64_t x, int64_t* sh, int64_t& total) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int64_t incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[wi] = incl;
  __syncthreads();
  if (wi == 0) {
    int64_t s = sh[lane], si = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, si, off);
      if (lane >= off) si += t;
    }
    sh[lane] = si - s;
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  total = sh[32];
  return incl - x + sh[wi];
}

__global__ void __launch_bounds__(kB) k_slot_sums(int64_t H, const uint64_t* __restrict__ htab,
                                                  int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[33];
  int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x, total;
  blk_scan(i < H && htab[i] != kEmpty, sh, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}
__global__ void __launch_bounds__(kB) k_scan_small(int64_t n, int64_t* __restrict__ a, int64_t* __restrict__ total_out) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += kB) {
    int64_t i = base + threadIdx.x, total;
    int64_t ex = blk_scan(i < n ? a[i] : 0, sh, total);
    __syncthreads();
    if (i < n) a[i] = ex + carry;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}
__global__ void __launch_bounds__(kB) k_slot_ids(int64_t H, const uint64_t* __restrict__ htab,
                                                 const int64_t* __restrict__ bsum, int32_t* __restrict__ gid) {
  __shared__ int64_t sh[33];
  int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x, total;
  bool used = i < H && htab[i] != kEmpty;
  int64_t o = blk_scan(used, sh, total) + bsum[blockIdx.x];
  if (i < H) gid[i] = used ? (int32_t)o : -1;
}

// W[g][s] accumulated as sums of 32-bit halves (no overflow below 2^32 terms)
__global__ void k_eval_accum(int64_t Tf, int S, const uint64_t* __restrict__ u, const uint64_t* __restrict__ w,
                             const uint64_t* __restrict__ htab, uint64_t hmask, const int32_t* __restrict__ gid,
                             uint64_t* __restrict__ U, unsigned long long* __restrict__ Wacc, uint32_t* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tf) return;
  const uint64_t uu = u[t];
  int64_t slot = find_slot(uu, htab, hmask);
  if (slot < 0) { atomicOr(status, ST_HASH_FULL); return; }
  const int g = gid[slot];
  U[g] = uu;
  for (int s = 0; s < S; s++) {
    uint64_t x = w[t * S + s];
    atomicAdd(&Wacc[((int64_t)g * S + s) * 2 + 0], (unsigned long long)lo32(x));
    atomicAdd(&Wacc[((int64_t)g * S + s) * 2 + 1], (unsigned long long)hi32(x));
  }
}

// finalize: the merged weights as residues and the squares table
// UP[g][a] = u_g^(2^a), a < 32
__global__ void k_eval_finalize(int64_t G, int S, const unsigned long long* __restrict__ Wacc,
                                const uint64_t* __restrict__ U, Mod M, uint64_t* __restrict__ Wp,
                                uint64_t* __restrict__ UP) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < G * S) {
    uint64_t lo = Wacc[idx * 2], hi = Wacc[idx * 2 + 1];
    // value = hi 2^32 + lo, as a 128-bit number
    uint64_t vlo = lo + (hi << 32);
    uint64_t vhi = (hi >> 32) + (vlo < lo);
    Wp[idx] = reduce128(vhi, vlo, M);
  }
  if (idx < G) {
    uint64_t x = U[idx];
    for (int a = 0; a < 32; a++) {
      UP[idx * 32 + a] = x;
      x = mul_mod(x, x, M);
    }
  }
}

constexpr int kGC = 32;   // groups per staged chunk

// The matrix-vector product out[s][i] = sum_g W[g][s] u_g^(i+off): a CTA owns
// NI consecutive i and NG thread groups of NI threads; group q accumulates
// the ST columns q ST .. q ST + ST - 1 for its thread's i.  Per chunk of kGC
// groups the CTA stages the weights and builds X[g][t] = u_g^(I0+off+t) by
// doubling (the paper's power table), shared by all NG groups; every thread
// then runs ST deferred multiply-accumulates per group, X[g][t] times a
// broadcast pair of weights.
template <int ST, int NG, int NI>
struct EvalCfg {
  static constexpr int STP = (ST + 1) & ~1;
  static constexpr int NT = NI * NG;
  static constexpr int WW = NG * STP;
  static constexpr int MINB = NT <= 448 ? 2 : 1;   // two CTAs per SM where the registers allow
};

template <int ST, int NG, int NI>
struct EvalSmem {
  uint64_t X[kGC][NI];
  uint64_t W[kGC][EvalCfg<ST, NG, NI>::WW];
  uint64_t part[kGC][8];
  uint64_t sq[kGC][8], sqp[kGC][8];   // u_g^(2^a) and its Shoup quotient, a < log2(NI)
};

template <int ST, int NG, int NI>
__global__ void __launch_bounds__(NI* NG, EvalCfg<ST, NG, NI>::MINB) k_eval_matvec(int64_t T, int S, int offset, int64_t G, int gsplit,
                                                           const uint64_t* __restrict__ UP,
                                                           const uint64_t* __restrict__ Wp, Mod M,
                                                           uint64_t* __restrict__ out, int64_t ldo,
                                                           uint64_t* __restrict__ partial) {
  using C = EvalCfg<ST, NG, NI>;
  extern __shared__ __align__(16) unsigned char smraw[];
  EvalSmem<ST, NG, NI>& sm = *reinterpret_cast<EvalSmem<ST, NG, NI>*>(smraw);
  const int tid = threadIdx.x, li = tid % NI, grp = tid / NI;
  const int64_t I0 = (int64_t)blockIdx.x * NI;
  const int split = blockIdx.y;
  const int64_t glo = G * split / gsplit, ghi = G * (split + 1) / gsplit;
  const uint64_t E = (uint64_t)(I0 + offset);
  Acc8 acc[ST];
#pragma unroll
  for (int c = 0; c < ST; c++) acc[c] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t gc = glo; gc < ghi; gc += kGC) {
    const int gn = (ghi - gc) < kGC ? (int)(ghi - gc) : kGC;
    __syncthreads();
    // base_g = u_g^E = prod over the set bits of E of UP[g][a]; 8 parts per group
    for (int t = tid; t < kGC * 8; t += C::NT) {
      const int g = t >> 3, pt = t & 7;
      uint64_t prod = 1;
      if (g < gn)
        for (int a = pt; a < 32; a += 8)
          if ((E >> a) & 1) prod = mul_mod(prod, UP[(gc + g) * 32 + a], M);
      sm.part[g][pt] = prod;
    }
    // weights of the chunk, [g][group][column], zero padded
    for (int t = tid; t < kGC * C::WW; t += C::NT) {
      const int g = t / C::WW, r = t - g * C::WW, q = r / C::STP, c = r - q * C::STP, sidx = q * ST + c;
      sm.W[g][r] = (g < gn && c < ST && sidx < S) ? Wp[(gc + g) * S + sidx] : 0;
    }
    __syncthreads();
    for (int g = tid; g < kGC; g += C::NT) {
      uint64_t b = 1;
      for (int q = 0; q < 8; q++) b = mul_mod(b, sm.part[g][q], M);
      sm.X[g][0] = b;
    }
    constexpr int LA = NI >= 256 ? 8 : (NI >= 128 ? 7 : (NI >= 64 ? 6 : 5));   // doubling levels
    for (int t = tid; t < kGC * LA; t += C::NT) {
      const int g = t / LA, a = t - g * LA;
      const uint64_t q = g < gn ? UP[(gc + g) * 32 + a] : 0;
      sm.sq[g][a] = q;
      sm.sqp[g][a] = shoup_pre(q, M);
    }
    __syncthreads();
    // doubling: X[g][t + 2^a] = X[g][t] u_g^(2^a), a Shoup multiply by a constant of the level
    for (int a = 0; a < LA; a++) {
      const int half = 1 << a;
      for (int idx = tid; idx < kGC * half; idx += C::NT) {
        const int g = idx / half, t = idx - g * half;
        if (g < gn) sm.X[g][t + half] = canon(shoup_lazy(sm.X[g][t], sm.sq[g][a], sm.sqp[g][a], M), M);
      }
      __syncthreads();
    }
    for (int g = 0; g < gn; g++) {
      const uint64_t x = sm.X[g][li];
      const uint32_t x0 = lo32(x), x1 = hi32(x);
      const uint64_t* row = &sm.W[g][grp * C::STP];
#pragma unroll
      for (int c = 0; c + 1 < ST; c += 2) {
        const uint4 w = *reinterpret_cast<const uint4*>(row + c);
        mac8(acc[c], x0, x1, w.x, w.y);
        mac8(acc[c + 1], x0, x1, w.z, w.w);
      }
      if (ST & 1) {
        const uint2 w = *reinterpret_cast<const uint2*>(row + ST - 1);
        mac8(acc[ST - 1], x0, x1, w.x, w.y);
      }
    }
  }
  const int64_t i = I0 + li;
  if (i >= T) return;
#pragma unroll
  for (int c = 0; c < ST; c++) {
    const int sidx = grp * ST + c;
    if (sidx >= S) continue;
    const uint64_t r = acc8_value(acc[c], M);
    if (gsplit == 1) out[(int64_t)sidx * ldo + i] = r;
    else partial[((int64_t)split * S + sidx) * T + i] = r;
  }
}

__global__ void k_eval_combine(int64_t T, int S, int gsplit, const uint64_t* __restrict__ partial, Mod M,
                               uint64_t* __restrict__ out, int64_t ldo) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * S) return;
  int s = (int)(idx / T);
  int64_t i = idx - (int64_t)s * T;
  uint64_t r = 0;
  for (int q = 0; q < gsplit; q++) r = add_mod(r, partial[((int64_t)q * S + s) * T + i], M);
  out[(int64_t)s * ldo + i] = r;
}

template <int ST, int NG, int NI>
static void launch_matvec_t(int64_t T, int S, int offset, int64_t G, int gsplit, const uint64_t* UP,
                            const uint64_t* Wp, const Mod& M, uint64_t* out, int64_t ldo, uint64_t* partial,
                            cudaStream_t st) {
  const size_t smem = sizeof(EvalSmem<ST, NG, NI>);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_eval_matvec<ST, NG, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  dim3 grid(cdiv(T, NI), gsplit);
  {
    k_eval_matvec<ST, NG, NI><<<grid, NI * NG, smem, st>>>(T, S, offset, G, gsplit, UP, Wp, M, out, ldo, partial);
    note_launch();
  }
}

// Launch shape by S: (columns per thread, thread groups, i per CTA).
struct EvalShape {
  int st, ng, ni;
};
static EvalShape eval_shape(int S) {
  // three columns per thread (four beyond 48 columns) keep a thread within
  // ~80 registers; as many i per CTA as keep two CTAs (<= 448 threads) per SM
  const int st = S <= 48 ? 3 : 4;
  const int ng = (S + st - 1) / st;
  int ni = 256;
  while (ni > 32 && ni * ng > 448) ni >>= 1;
  return {st, ng, ni};
}

template <int NG>
static void launch_matvec_g(int st, int ni, int64_t T, int S, int offset, int64_t G, int gsplit, const uint64_t* UP,
                            const uint64_t* Wp, const Mod& M, uint64_t* out, int64_t ldo, uint64_t* partial,
                            cudaStream_t s) {
  if (st == 4) {
    if constexpr (NG >= 13) launch_matvec_t<4, NG, 32>(T, S, offset, G, gsplit, UP, Wp, M, out, ldo, partial, s);
    return;
  }
  if constexpr (NG <= 16) {
    constexpr int NI1 = NG == 1 ? 256 : (NG <= 3 ? 128 : (NG <= 7 ? 64 : 32));
    (void)ni;
    launch_matvec_t<3, NG, NI1>(T, S, offset, G, gsplit, UP, Wp, M, out, ldo, partial, s);
  }
}

static void launch_matvec(const EvalShape& sh, int64_t T, int S, int offset, int64_t G, int gsplit,
                          const uint64_t* UP, const uint64_t* Wp, const Mod& M, uint64_t* out, int64_t ldo,
                          uint64_t* partial, cudaStream_t st) {
#define ZR_MV(NGV) \
  case NGV: launch_matvec_g<NGV>(sh.st, sh.ni, T, S, offset, G, gsplit, UP, Wp, M, out, ldo, partial, st); break;
  switch (sh.ng) {
    ZR_MV(1) ZR_MV(2) ZR_MV(3) ZR_MV(4) ZR_MV(5) ZR_MV(6) ZR_MV(7) ZR_MV(8)
    ZR_MV(9) ZR_MV(10) ZR_MV(11) ZR_MV(12) ZR_MV(13) ZR_MV(14) ZR_MV(15) ZR_MV(16)
    default: break;
  }
#undef ZR_MV
}

// Group splits so that the launch has at least eight CTAs per SM (about four
// waves of two: the last wave's imbalance stays small).
static int eval_gsplit(const zr_ctx* ctx, int64_t T, int S, int64_t Tf) {
  const EvalShape sh = eval_shape(S);
  const int64_t ctas = (int64_t)cdiv(T, sh.ni);
  int gsplit = 1;
  const int64_t want = 8ll * (ctx && ctx->sms ? ctx->sms : 152);
  while (ctas * gsplit < want && gsplit < 64 && Tf / (gsplit * 2) >= 2 * kGC) gsplit *= 2;
  return gsplit;
}

// Workspace bytes the evaluator needs for (f, S, T).
size_t probes_ws_need(const zr_ctx* ctx, const zr_poly* f, int k, int S, int64_t T);

zr_status probes_impl(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                      const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                      cudaStream_t st) {
  zr_status r = ensure_ws(ctx, probes_ws_need(ctx, f, k, S, T), st);
  if (r) return r;
  return probes_enqueue(ctx, f, k, y, S, samples, z, T, offset, out, ldo, status, ctx->ws, st);
}

// The evaluation itself, with its scratch at `base` (capacity checked by the caller).
zr_status probes_enqueue(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                         const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                         char* base, cudaStream_t st) {
  const Mod& M = ctx->M;
  const int64_t Tf = f->T;
  const int nv = f->nv;
  const uint64_t H = hash_slots(Tf > 0 ? Tf : 1);
  const int64_t nbH = (int64_t)((H + kB - 1) / kB);
  const int gsplit = eval_gsplit(ctx, T, S, Tf);
  auto layout = [&](Carver& cv, uint64_t** tabY, uint64_t** tabZ, uint64_t** tabC, uint64_t** u, uint64_t** w,
                    uint64_t** htab, int64_t** bsum, int32_t** gid, uint64_t** U, unsigned long long** Wacc,
                    uint64_t** Wp, uint64_t** UP, uint64_t** partial, int64_t** Gdev) {
    const int64_t Tn = Tf > 0 ? Tf : 1;
    *tabY = cv.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
    *tabZ = cv.take<uint64_t>((size_t)nv * kPowTab);
    *tabC = cv.take<uint64_t>((size_t)S * kPowTab);
    *u = cv.take<uint64_t>(Tn);
    *w = cv.take<uint64_t>((size_t)Tn * S);
    *htab = cv.take<uint64_t>(H);
    *bsum = cv.take<int64_t>(nbH + 1);
    *gid = cv.take<int32_t>(H);
    *U = cv.take<uint64_t>(Tn);
    *Wacc = cv.take<unsigned long long>((size_t)Tn * S * 2);
    *Wp = cv.take<uint64_t>((size_t)Tn * S);
    *UP = cv.take<uint64_t>((size_t)Tn * 32);
    *partial = cv.take<uint64_t>(gsplit > 1 ? (size_t)gsplit * S * (T > 0 ? T : 1) : 1);
    *Gdev = cv.take<int64_t>(1);
  };
  uint64_t *tabY, *tabZ, *tabC, *u, *w, *htab, *U, *UP, *partial;
  int64_t *bsum, *Gdev;
  int32_t* gid;
  unsigned long long* Wacc;
  uint64_t* Wp;
  Carver cv(base);
  layout(cv, &tabY, &tabZ, &tabC, &u, &w, &htab, &bsum, &gid, &U, &Wacc, &Wp, &UP, &partial, &Gdev);

  if (T <= 0) return ZR_OK;
  if (Tf == 0) {
    for (int s = 0; s < S; s++) cudaMemsetAsync(out + (int64_t)s * ldo, 0, sizeof(uint64_t) * T, st);
    return cuda_err(ctx, cudaGetLastError(), "zr_zippel_probes");
  }
  cudaMemsetAsync(htab, 0xFF, H * sizeof(uint64_t), st);
  cudaMemsetAsync(Wacc, 0, (size_t)Tf * S * 2 * sizeof(unsigned long long), st);
  if (k > 0) { k_powrows<<<k, kPowTab, 0, st>>>(y, k, M, tabY); note_launch(); }
  if (z && nv > k + 1) { k_powrows<<<nv, kPowTab, 0, st>>>(z, nv, M, tabZ); note_launch(); }
  else cudaMemsetAsync(tabZ, 0, (size_t)nv * kPowTab * sizeof(uint64_t), st);
  { k_powrows<<<S, kPowTab, 0, st>>>(samples, S, M, tabC); note_launch(); }
  { k_eval_terms<<<cdiv(Tf, 256), 256, 0, st>>>(Tf, nv, f->exps, f->coef, k, tabY, tabZ, tabC, S, M, u, w, htab, H - 1); note_launch(); }
  { k_slot_sums<<<(unsigned)nbH, kB, 0, st>>>((int64_t)H, htab, bsum); note_launch(); }
  { k_scan_small<<<1, kB, 0, st>>>(nbH, bsum, Gdev); note_launch(); }
  { k_slot_ids<<<(unsigned)nbH, kB, 0, st>>>((int64_t)H, htab, bsum, gid); note_launch(); }
  { k_eval_accum<<<cdiv(Tf, 256), 256, 0, st>>>(Tf, S, u, w, htab, H - 1, gid, U, Wacc, status); note_launch(); }
  // the group count is needed on the host to size the launch
  int64_t G = 0;
  cudaError_t e = cudaMemcpyAsync(ctx->h_count + 1, Gdev, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_probes: group count");
  G = ctx->h_count[1];
  { k_eval_finalize<<<cdiv(G * S > G ? G * S : G, 256), 256, 0, st>>>(G, S, Wacc, U, M, Wp, UP); note_launch(); }
  launch_matvec(eval_shape(S), T, S, offset, G, gsplit, UP, Wp, M, out, ldo, partial, st);
  if (gsplit > 1) { k_eval_combine<<<cdiv(T * S, 256), 256, 0, st>>>(T, S, gsplit, partial, M, out, ldo); note_launch(); }
  return cuda_err(ctx, cudaGetLastError(), "zr_zippel_probes");
}

size_t probes_ws_need(const zr_ctx* ctx, const zr_poly* f, int k, int S, int64_t T) {
  const int64_t Tf = f->T;
  const int nv = f->nv;
  const uint64_t H = hash_slots(Tf > 0 ? Tf : 1);
  const int64_t nbH = (int64_t)((H + kB - 1) / kB);
  const int gsplit = eval_gsplit(ctx, T, S, Tf);
  const int64_t Tn = Tf > 0 ? Tf : 1;
  Carver cv(nullptr);
  cv.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
  cv.take<uint64_t>((size_t)nv * kPowTab);
  cv.take<uint64_t>((size_t)S * kPowTab);
  cv.take<uint64_t>(Tn);
  cv.take<uint64_t>((size_t)Tn * S);
  cv.take<uint64_t>(H);
  cv.take<int64_t>(nbH + 1);
  cv.take<int32_t>(H);
  cv.take<uint64_t>(Tn);
  cv.take<unsigned long long>((size_t)Tn * S * 2);
  cv.take<uint64_t>((size_t)Tn * S);
  cv.take<uint64_t>((size_t)Tn * 32);
  cv.take<uint64_t>(gsplit > 1 ? (size_t)gsplit * S * (T > 0 ? T : 1) : 1);
  cv.take<int64_t>(1);
  return cv.off;
}

// ---------------------------------------------------------------------------
// f at arbitrary points: one CTA per point, terms split over the threads,
// partial sums reduced with shuffles (Sec. 2.2's warp sum, full-warp mask).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_eval_points(int64_t Tf, int nv, const uint8_t* __restrict__ exps,
                                                     const uint64_t* __restrict__ coef, const uint64_t* __restrict__ pts,
                                                     Mod M, uint64_t* __restrict__ out) {
  __shared__ uint64_t red[8];
  const int64_t pt = blockIdx.x;
  uint64_t sum = 0;
  for (int64_t t = threadIdx.x; t < Tf; t += blockDim.x) {
    uint64_t c = coef[t];
    if (c >= M.p) c -= M.p;
    for (int m = 0; m < nv; m++) {
      uint64_t x = pts[pt * nv + m];
      if (x >= M.p) x -= M.p;
      c = mul_mod(c, pow_mod(x, exps[t * nv + m], M), M);
    }
    sum = add_mod(sum, c, M);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum = add_mod(sum, __shfl_down_sync(0xffffffffu, sum, off), M);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int q = 0; q < 8; q++) s = add_mod(s, red[q], M);
    out[pt] = s;
  }
}

// The probe points of a Zippel step: thread i computes y_m^(i+off) once per
// variable and writes it into the S points of probe i.
__global__ void k_probe_points(int64_t T, int S, int nv, int k, int offset, const uint64_t* __restrict__ y,
                               const uint64_t* __restrict__ cs, const uint64_t* __restrict__ z, Mod M,
                               uint64_t* __restrict__ pts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T) return;
  for (int m = 0; m < nv; m++) {
    if (m == k) {
      for (int s = 0; s < S; s++) pts[((int64_t)s * T + i) * nv + m] = canon(cs[s], M);
    } else {
      const uint64_t val = m < k ? pow_mod(canon(y[m], M), (uint64_t)(i + offset), M) : canon(z[m], M);
      for (int s = 0; s < S; s++) pts[((int64_t)s * T + i) * nv + m] = val;
    }
  }
}

void launch_probe_points(int64_t T, int S, int nv, int k, int offset, const uint64_t* y, const uint64_t* cs,
                         const uint64_t* z, const Mod& M, uint64_t* pts, cudaStream_t st) {
  if (T > 0 && S > 0) { k_probe_points<<<cdiv(T, 128), 128, 0, st>>>(T, S, nv, k, offset, y, cs, z, M, pts); note_launch(); }
}

void launch_eval_points(const zr_poly* f, int64_t npts, const uint64_t* pts, const Mod& M, uint64_t* out,
                        cudaStream_t st) {
  if (npts > 0) { k_eval_points<<<(unsigned)npts, 256, 0, st>>>(f->T, f->nv, f->exps, f->coef, pts, M, out); note_launch(); }
}

}  // namespace zr

using namespace zr;

extern "C" zr_status zr_zippel_probes(zr_ctx* ctx, const zr_poly* f, int32_t k, const uint64_t* y, int32_t S,
                                      const uint64_t* samples, const uint64_t* z, int64_t T, int32_t offset,
                                      uint64_t* out, int64_t ldo, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (!f || f->nv < 1 || f->nv > kMaxVars || k < 0 || k >= f->nv || S < 1 || S > 256 || T < 0 || ldo < T ||
      f->T < 0 || (offset != 0 && offset != 1))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_probes: arguments out of range");
  if ((f->T > 0 && (!f->exps || !f->coef)) || !samples || (k > 0 && !y) || (T > 0 && !out) ||
      (k < f->nv - 1 && !z))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_probes: null pointer");
  if (T >= (1ll << 32)) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_probes: T must be below 2^32");
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  zr_status r = probes_impl(ctx, f, k, y, S, samples, z, T, offset, out, ldo, ctx->d_status_call, st);
  if (r) return r;
  cudaError_t e = cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_probes");
  return status_from_flags(ctx, ctx->h_status[1]);
}

extern "C" zr_status zr_eval_points(zr_ctx* ctx, const zr_poly* f, int64_t npts, const uint64_t* pts, uint64_t* out,
                                    void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (!f || f->nv < 1 || f->nv > kMaxVars || f->T < 0 || npts < 0 || (npts > 0 && (!pts || !out)) ||
      (f->T > 0 && (!f->exps || !f->coef)))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_eval_points: arguments out of range");
  cudaStream_t st = (cudaStream_t)stream;
  if (npts > 0) { k_eval_points<<<(unsigned)npts, 256, 0, st>>>(f->T, f->nv, f->exps, f->coef, pts, ctx->M, out); note_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_err(ctx, e, "zr_eval_points");
}

extern "C" zr_status zr_probe_points(zr_ctx* ctx, int32_t nv, int32_t k, const uint64_t* y, int32_t S,
                                     const uint64_t* samples, const uint64_t* z, int64_t T, int32_t offset,
                                     uint64_t* pts, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (nv < 1 || nv > kMaxVars || k < 0 || k >= nv || S < 1 || T < 0 || (offset != 0 && offset != 1) ||
      (T > 0 && (!pts || !samples || (k > 0 && !y) || (k + 1 < nv && !z))))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_probe_points: arguments out of range");
  launch_probe_points(T, S, nv, k, offset, y, samples, z, ctx->M, pts, (cudaStream_t)stream);
  return cuda_err(ctx, cudaGetLastError(), "zr_probe_points");
}
