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
// The kernel (k_eval_ring) tiles it: a CTA owns 32 consecutive i and walks a
// range of groups in chunks of 32; for each chunk a producer warp fills the
// power table X[t][g] = u_g^(I0+off+t) in shared memory (the paper's power
// table, Sec. 2.2: a starting power, then one multiply by u_g per entry) and
// consumer warps accumulate sum_g w_{g,s} X[t][g] for their columns with the
// deferred multiply-accumulate.
#include <cuda_runtime.h>

#include <cmath>

#include "zr_internal.h"
#include "zr_ring.cuh"

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

// per term: its anchor value u_t and its weight without the new variable,
// a_t = coef_t prod_{m>k} z_m^{e_{t,m}}; u_t goes into the hash table
__global__ void k_eval_terms(int64_t Tf, int nv, const uint8_t* __restrict__ exps, const uint64_t* __restrict__ coef,
                             int k, const uint64_t* __restrict__ tabY, const uint64_t* __restrict__ tabZ, Mod M,
                             uint64_t* __restrict__ u, uint64_t* __restrict__ a, uint64_t* htab, uint64_t hmask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tf) return;
  const uint8_t* e = exps + t * nv;
  uint64_t uu = 1;
  for (int m = 0; m < k; m++) uu = mul_mod(uu, tabY[m * kPowTab + e[m]], M);
  uint64_t c = coef[t];
  if (c >= M.p) c -= M.p;
  for (int m = k + 1; m < nv; m++) c = mul_mod(c, tabZ[m * kPowTab + e[m]], M);
  u[t] = uu;
  a[t] = c;
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

// The terms of every group, listed by a counting sort: tg[t] = the term's
// group, tp[t] = its place in the group, cnt[g] = the group's size.
__global__ void k_eval_count(int64_t Tf, const uint64_t* __restrict__ u, const uint64_t* __restrict__ htab,
                             uint64_t hmask, const int32_t* __restrict__ gid, uint64_t* __restrict__ U,
                             int32_t* __restrict__ cnt, int32_t* __restrict__ tg, int32_t* __restrict__ tp,
                             uint32_t* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tf) return;
  const uint64_t uu = u[t];
  int64_t slot = find_slot(uu, htab, hmask);
  if (slot < 0) {
    atomicOr(status, ST_HASH_FULL);
    tg[t] = -1;
    return;
  }
  const int g = gid[slot];
  U[g] = uu;
  tg[t] = g;
  tp[t] = atomicAdd(&cnt[g], 1);
}
// block sums of the group sizes, then each group's first place
__global__ void __launch_bounds__(kB) k_cnt_sums(int64_t n, const int32_t* __restrict__ cnt, int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[33];
  int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x, total;
  blk_scan(i < n ? cnt[i] : 0, sh, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}
__global__ void __launch_bounds__(kB) k_cnt_start(int64_t n, const int32_t* __restrict__ cnt,
                                                  const int64_t* __restrict__ bsum, int64_t* __restrict__ start) {
  __shared__ int64_t sh[33];
  int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x, total;
  const int64_t o = blk_scan(i < n ? cnt[i] : 0, sh, total) + bsum[blockIdx.x];
  if (i < n) start[i] = o;
}
__global__ void k_eval_scatter(int64_t Tf, const int32_t* __restrict__ tg, const int32_t* __restrict__ tp,
                               const int64_t* __restrict__ start, int64_t* __restrict__ order) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tf || tg[t] < 0) return;
  order[start[tg[t]] + tp[t]] = t;
}

// Where the weights of the matrix-vector kernel live: column block b
// (columns s0[b] .. s0[b] + 63) holds, per group, its row of bw[b] words laid
// out as the kernel stages it ([consumer][column], pairs padded with zero).
struct RingLayout {
  int nb;
  int cg[4], cgp[4], bw[4];
  int64_t off[4];   // word offset of block b (G bw[b'] words per block before it)
};

// finalize, for the G groups counted on the device (G <= Tn, the stride of
// the tables): the merged weights as residues in the ring layout, zero in
// the padding; the squares table UP[a][g] = u_g^(2^a), a < 32, with its
// Shoup quotients UPq; the quotients Uq[g] of u_g.
__global__ void k_eval_finalize(const int64_t* __restrict__ Gdev, int64_t Tn, int S, const int64_t* __restrict__ start,
                                const int32_t* __restrict__ cnt, const int64_t* __restrict__ order,
                                const uint64_t* __restrict__ a, const uint8_t* __restrict__ exps, int nv, int k,
                                const uint64_t* __restrict__ tabC, const uint64_t* __restrict__ U, Mod M, RingLayout L,
                                int rw, uint64_t* __restrict__ Wr, uint64_t* __restrict__ UP,
                                uint64_t* __restrict__ UPq, uint64_t* __restrict__ Uq) {
  const int64_t G = *Gdev;
  // a grid-stride loop: the launch is sized for the SMs, the work for G
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < G * rw; idx += stride) {
    // entry j of group g's rows: block b, consumer q, column c
    const int64_t g = idx / rw;
    int j = (int)(idx - g * rw), b = 0;
    while (j >= L.bw[b]) j -= L.bw[b++];
    const int q = j / L.cgp[b], c = j - q * L.cgp[b], sc = q * L.cg[b] + c, s = 64 * b + sc;
    uint64_t r = 0;
    if (c < L.cg[b] && s < S) {
      // W[g][s] = sum over the group's terms of a_t c_s^{e_{t,k}}
      Acc8 acc{0, 0, 0, 0, 0, 0, 0, 0};
      const uint64_t* cs = tabC + (int64_t)s * kPowTab;
      const int64_t r0 = start[g], n = cnt[g];
      for (int64_t x = 0; x < n; x++) {
        const int64_t t = order[r0 + x];
        const uint64_t at = a[t], w = cs[exps[t * nv + k]];
        mac8(acc, lo32(at), hi32(at), lo32(w), hi32(w));
      }
      r = acc8_value(acc, M);
    }
    Wr[L.off[b] + g * L.bw[b] + j] = r;
  }
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < G; idx += stride) {
    uint64_t x = U[idx];
    Uq[idx] = shoup_pre(x, M);
    for (int e = 0; e < 32; e++) {
      UP[e * Tn + idx] = x;
      UPq[e * Tn + idx] = shoup_pre(x, M);
      x = mul_mod(x, x, M);
    }
  }
}

// The matrix-vector product out[s][i] = sum_g W[g][s] u_g^(i+off),
// warp-specialised like the solve.  A CTA owns a tile of 32 consecutive i and
// a range of groups, walked in chunks of 32 through a ring of shared-memory
// stages:
//   warp 0 (producer)     lane = group: stages the chunk's weights with
//                         cp.async and fills the power table
//                         X[t][g] = u_g^(I0+off+t), t < 32, starting from
//                         u_g^(I0+off) (a product of squares u_g^(2^a) over
//                         the set bits of the exponent) and running a Shoup
//                         multiply by u_g along t (the paper's power table,
//                         Sec. 2.2, one row per group);
//   warps 1.. (consumers) lane = i: CG columns each, acc_s += X[i][g] W[g][s]
//                         in 160-bit accumulators, reduced once.
// Every power is computed once and read by all consumer warps.  Columns
// beyond 64 run as further launches over the next column block.
template <int CG, int G>
struct EvalRingCfg {
  static constexpr int TI = 32;               // i per CTA: one per consumer lane
  static constexpr int GC = 32;               // groups per chunk: one per producer lane
  static constexpr int NST = 4;               // ring stages
  static constexpr int XP = GC + 1;           // padded row of X: the consumers read it across rows
  static constexpr int CGP = (CG + 1) & ~1;   // a consumer's columns, padded to pairs
  static constexpr int BW = G * CGP;          // staged weight row width
  static constexpr int NT = 32 * (1 + G);
  static constexpr int REG = CG <= 2 ? 72 : (CG <= 3 ? 80 : (CG <= 4 ? 104 : (CG <= 6 ? 136 : 168)));
  static constexpr int FIT = 65536 / (NT * REG);
  static constexpr int MINB = FIT < 1 ? 1 : (FIT > 6 ? 6 : FIT);
  static constexpr size_t XB = sizeof(uint64_t) * NST * TI * XP;
  static constexpr size_t WB = sizeof(uint64_t) * NST * GC * BW;
  static constexpr size_t SMEM = XB + WB + sizeof(uint64_t) * 2 * NST;
};

template <int CG, int G>
__global__ void __launch_bounds__(EvalRingCfg<CG, G>::NT, EvalRingCfg<CG, G>::MINB)
    k_eval_ring(int64_t T, int S, int s0, int offset, const int64_t* __restrict__ Gdev, int64_t NG, int gsplit,
                const uint64_t* __restrict__ UP,
                const uint64_t* __restrict__ UPq, const uint64_t* __restrict__ U, const uint64_t* __restrict__ Uq,
                const uint64_t* __restrict__ Wb, Mod M, uint64_t* __restrict__ out, int64_t ldo,
                uint64_t* __restrict__ partial, uint32_t* __restrict__ status) {
  using C = EvalRingCfg<CG, G>;
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t(*xs)[C::TI][C::XP] = reinterpret_cast<uint64_t(*)[C::TI][C::XP]>(smraw);
  uint64_t(*ws)[C::GC][C::BW] = reinterpret_cast<uint64_t(*)[C::GC][C::BW]>(smraw + C::XB);
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + C::XB + C::WB);
  uint64_t* empty = full + C::NST;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int SC = (S - s0) < G * CG ? S - s0 : G * CG;   // columns of this launch
  if (tid == 0)
    for (int st = 0; st < C::NST; st++) {
      mbar_init(&full[st], 32);
      mbar_init(&empty[st], G);
    }
  __syncthreads();
  const int64_t I0 = (int64_t)blockIdx.x * C::TI;
  const int split = blockIdx.y;
  const int64_t G_ = *Gdev;   // groups; NG (>= G_) is the stride of the squares table
  const int64_t glo = G_ * split / gsplit, ghi = G_ * (split + 1) / gsplit;
  const int nch = (int)((ghi - glo + C::GC - 1) / C::GC);

  if (warp == 0) {
    // ---- producer warp
    const uint32_t emask = (uint32_t)(I0 + offset);   // the exponent E < 2^32 of t = 0
    for (int c = 0; c < nch; c++) {
      const int st = c % C::NST;
      const uint32_t ph = (c / C::NST) & 1;
      if (c >= C::NST && !mbar_wait(&empty[st], ph ^ 1)) {
        atomicOr(status, ST_TIMEOUT);
        cp_async_wait<0>();
        return;
      }
      const int64_t gc = glo + (int64_t)c * C::GC;
      const int gn = (ghi - gc) < C::GC ? (int)(ghi - gc) : C::GC;
      // weights of the chunk: gn consecutive rows, already in the staged layout
      {
        const uint64_t* src = Wb + gc * C::BW;
        uint64_t* dst = &ws[st][0][0];
        const int n16 = gn * C::BW / 2;
        for (int q = lane; q < n16; q += 32) cp_async16(dst + 2 * q, src + 2 * q);
      }
      cp_async_commit();
      if (lane < gn) {
        const int64_t gg = gc + lane;
        const uint64_t u = __ldg(U + gg), uq = __ldg(Uq + gg);
        const uint64_t u16 = __ldg(UP + 4 * NG + gg), u16q = __ldg(UPq + 4 * NG + gg);
        // u_g^E: a Shoup product of the squares of E's set bits, their loads
        // issued eight at a time
        uint64_t x = 1;
        for (uint32_t m = emask; m;) {
          uint64_t f[8], fq[8];
          bool have[8];
#pragma unroll
          for (int q = 0; q < 8; q++) {
            have[q] = m != 0;
            const int a = have[q] ? __ffs(m) - 1 : 0;
            m &= m - 1;
            f[q] = have[q] ? __ldg(UP + (int64_t)a * NG + gg) : 0;
            fq[q] = have[q] ? __ldg(UPq + (int64_t)a * NG + gg) : 0;
          }
#pragma unroll
          for (int q = 0; q < 8; q++)
            if (have[q]) x = shoup_lazy(x, f[q], fq[q], M);
        }
        x = canon(x, M);
        // two interleaved chains, t < 16 and t >= 16, one Shoup multiply by u per step
        uint64_t xb = canon(shoup_lazy(x, u16, u16q, M), M);
#pragma unroll 4
        for (int t = 0; t < C::TI / 2; t++) {
          xs[st][t][lane] = x;
          xs[st][t + C::TI / 2][lane] = xb;
          x = canon(shoup_lazy(x, u, uq, M), M);
          xb = canon(shoup_lazy(xb, u, uq, M), M);
        }
      }
      cp_async_wait<0>();
      mbar_arrive(&full[st]);
    }
    return;
  }
  // ---- consumer w: columns s0 + w CG .. s0 + w CG + CG - 1
  const int w = warp - 1;
  Acc8 acc[CG];
#pragma unroll
  for (int q = 0; q < CG; q++) acc[q] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < nch; c++) {
    const int st = c % C::NST;
    const uint32_t ph = (c / C::NST) & 1;
    if (!mbar_wait(&full[st], ph)) {
      atomicOr(status, ST_TIMEOUT);
      return;
    }
    const int64_t gc = glo + (int64_t)c * C::GC;
    const int gn = (ghi - gc) < C::GC ? (int)(ghi - gc) : C::GC;
    const uint64_t* xrow = xs[st][lane];
    if (gn == C::GC) {
#pragma unroll
      for (int g = 0; g < C::GC; g++) {
        const uint64_t x = xrow[g];
        const uint32_t x0 = lo32(x), x1 = hi32(x);
        const uint64_t* row = &ws[st][g][w * C::CGP];
#pragma unroll
        for (int q = 0; q + 1 < CG; q += 2) {
          const uint4 v = *reinterpret_cast<const uint4*>(row + q);
          mac8(acc[q], x0, x1, v.x, v.y);
          mac8(acc[q + 1], x0, x1, v.z, v.w);
        }
        if (CG & 1) {
          const uint2 v = *reinterpret_cast<const uint2*>(row + CG - 1);
          mac8(acc[CG - 1], x0, x1, v.x, v.y);
        }
      }
    } else {
#pragma unroll 1
      for (int g = 0; g < gn; g++) {
        const uint64_t x = xrow[g];
        const uint32_t x0 = lo32(x), x1 = hi32(x);
        const uint64_t* row = &ws[st][g][w * C::CGP];
#pragma unroll
        for (int q = 0; q + 1 < CG; q += 2) {
          const uint4 v = *reinterpret_cast<const uint4*>(row + q);
          mac8(acc[q], x0, x1, v.x, v.y);
          mac8(acc[q + 1], x0, x1, v.z, v.w);
        }
        if (CG & 1) {
          const uint2 v = *reinterpret_cast<const uint2*>(row + CG - 1);
          mac8(acc[CG - 1], x0, x1, v.x, v.y);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  const int64_t i = I0 + lane;
  if (i >= T) return;
#pragma unroll
  for (int q = 0; q < CG; q++) {
    const int sidx = s0 + w * CG + q;
    if (w * CG + q >= SC) continue;
    const uint64_t r = acc8_value(acc[q], M);
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

template <int CG, int G>
static int ring_occupancy_t() {
  using C = EvalRingCfg<CG, G>;
  static DeviceValue occ;
  return occ.get([] {
    cudaFuncSetAttribute(k_eval_ring<CG, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_ring<CG, G>, C::NT, C::SMEM) != cudaSuccess || n < 1)
      n = 1;
    return n;
  });
}

template <int CG, int G>
static void launch_ring_t(int64_t T, int S, int s0, int offset, const int64_t* Gdev, int64_t NG, int gsplit,
                          const uint64_t* UP,
                          const uint64_t* UPq, const uint64_t* U, const uint64_t* Uq, const uint64_t* Wb,
                          const Mod& M, uint64_t* out, int64_t ldo, uint64_t* partial, uint32_t* status,
                          cudaStream_t st) {
  using C = EvalRingCfg<CG, G>;
  ring_occupancy_t<CG, G>();   // also sets the shared-memory attribute
  dim3 grid(cdiv(T, C::TI), gsplit);
  k_eval_ring<CG, G><<<grid, C::NT, C::SMEM, st>>>(T, S, s0, offset, Gdev, NG, gsplit, UP, UPq, U, Uq, Wb, M, out,
                                                   ldo, partial, status);
  note_launch();
}

// The instances: columns per consumer and consumer warps for a block of
// SC <= 64 columns (at most 8 consumers).
using RingLaunch = void (*)(int64_t, int, int, int, const int64_t*, int64_t, int, const uint64_t*, const uint64_t*,
                            const uint64_t*,
                            const uint64_t*, const uint64_t*, const Mod&, uint64_t*, int64_t, uint64_t*, uint32_t*,
                            cudaStream_t);
struct RingInst {
  int cg, g;
  RingLaunch launch;
  int (*occupancy)();
};
#define ZR_RING(CGV, GV) {CGV, GV, launch_ring_t<CGV, GV>, ring_occupancy_t<CGV, GV>}
static const RingInst kRing[] = {ZR_RING(1, 1), ZR_RING(2, 1), ZR_RING(3, 1), ZR_RING(3, 2), ZR_RING(3, 3),
                                 ZR_RING(3, 4), ZR_RING(3, 5), ZR_RING(3, 6), ZR_RING(3, 7), ZR_RING(3, 8),
                                 ZR_RING(4, 7), ZR_RING(4, 8), ZR_RING(6, 6), ZR_RING(6, 7), ZR_RING(6, 8),
                                 ZR_RING(8, 7), ZR_RING(8, 8)};
#undef ZR_RING

static const RingInst* ring_inst(int SC) {
  const int cg = SC <= 2 ? SC : (SC <= 24 ? 3 : (SC <= 32 ? 4 : (SC <= 48 ? 6 : 8)));
  const int g = (SC + cg - 1) / cg;
  for (const RingInst& r : kRing)
    if (r.cg == cg && r.g == g) return &r;
  return nullptr;
}

// The weight layout for S columns over G groups (blocks of 64 columns).
static RingLayout ring_layout(int S, int64_t G) {
  RingLayout L{};
  int64_t off = 0;
  for (int s0 = 0; s0 < S; s0 += 64) {
    const RingInst* r = ring_inst(S - s0 < 64 ? S - s0 : 64);
    const int b = L.nb++;
    L.cg[b] = r->cg;
    L.cgp[b] = (r->cg + 1) & ~1;
    L.bw[b] = r->g * L.cgp[b];
    L.off[b] = off;
    off += G * L.bw[b];
  }
  return L;
}
static int64_t ring_words(int S, int64_t G) {
  const RingLayout L = ring_layout(S, G);
  return L.off[L.nb - 1] + G * L.bw[L.nb - 1];
}

static void launch_ring(int64_t T, int S, int offset, const int64_t* Gdev, int64_t NG, int gsplit, const uint64_t* UP,
                        const uint64_t* UPq, const uint64_t* U, const uint64_t* Uq, const uint64_t* Wr,
                        const RingLayout& L, const Mod& M, uint64_t* out, int64_t ldo, uint64_t* partial,
                        uint32_t* status, cudaStream_t st) {
  for (int b = 0; b < L.nb; b++) {
    const int s0 = 64 * b;
    const RingInst* r = ring_inst(S - s0 < 64 ? S - s0 : 64);
    r->launch(T, S, s0, offset, Gdev, NG, gsplit, UP, UPq, U, Uq, Wr + L.off[b], M, out, ldo, partial, status, st);
  }
}

// Group splits: the smallest count that gives at least two waves of CTAs
// with the last one at least 97% full (else the best fill up to 32 splits),
// keeping 64 or more groups per split.
static int eval_gsplit(const zr_ctx* ctx, int64_t T, int S, int64_t Tf) {
  const int64_t ctas = (int64_t)cdiv(T, 32);
  const int64_t slots = (int64_t)(ctx && ctx->sms ? ctx->sms : 152) * ring_inst(S < 64 ? S : 64)->occupancy();
  if (ctas >= 8 * slots) return 1;
  int best = 1;
  double best_fill = 0;
  for (int gs = 1; gs <= 32; gs++) {
    if (gs > 1 && Tf / gs < 64) break;
    const double waves = (double)(ctas * gs) / (double)slots;
    const double fill = waves / std::ceil(waves);
    if (waves >= 2 && fill >= 0.97) return gs;
    if (fill > best_fill + 1e-9) {
      best = gs;
      best_fill = fill;
    }
  }
  return best;
}

// Workspace bytes the evaluator needs for (f, S, T).
size_t probes_ws_need(const zr_ctx* ctx, const zr_poly* f, int k, int S, int64_t T);

zr_status probes_impl(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                      const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                      cudaStream_t st, int lane) {
  if (lane < 0 || lane >= zr_ctx::kProbeLanes) {
    zr_status r = ensure_ws(ctx, probes_ws_need(ctx, f, k, S, T), st);
    if (r) return r;
    return probes_enqueue(ctx, f, k, y, S, samples, z, T, offset, out, ldo, status, ctx->ws, st);
  }
  // the lane's own scratch, grown (rarely) after its stream's queued work
  const size_t need = probes_ws_need(ctx, f, k, S, T);
  if (ctx->pl_cap[lane] < need) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ctx->pl_ws[lane]) e = cudaFree(ctx->pl_ws[lane]);
    ctx->pl_ws[lane] = nullptr;
    ctx->pl_cap[lane] = 0;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->pl_ws[lane], need + need / 4);
    if (e != cudaSuccess) {
      ctx->pl_ws[lane] = nullptr;
      return cuda_err(ctx, e, "probe lane workspace");
    }
    ctx->pl_cap[lane] = need + need / 4;
  }
  return probes_enqueue(ctx, f, k, y, S, samples, z, T, offset, out, ldo, status, ctx->pl_ws[lane], st,
                        &ctx->pl_fws[lane], &ctx->pl_fcap[lane]);
}

// The evaluator's scratch, carved the same way for sizing and for use.
struct EvalWs {
  uint64_t *tabY, *tabZ, *tabC, *u, *a, *htab, *U, *Wp, *UP, *UPq, *Uq, *partial;
  int64_t *bsum, *cbsum, *start, *order, *Gdev, *total;
  int32_t *gid, *cnt, *tg, *tp;
};
// fast: the probes go through the transposed tree (its own workspace), so
// the matrix-vector kernel's tables are not carved
static EvalWs carve_eval(Carver& cv, int64_t Tf, int nv, int k, int S, int64_t T, int gsplit, bool fast = false) {
  EvalWs w;
  const int64_t Tn = Tf > 0 ? Tf : 1;
  const uint64_t H = hash_slots(Tn);
  const int64_t nbH = (int64_t)((H + kB - 1) / kB), nbT = (Tn + kB - 1) / kB;
  w.tabY = cv.take<uint64_t>((size_t)(k > 0 ? k : 1) * kPowTab);
  w.tabZ = cv.take<uint64_t>((size_t)nv * kPowTab);
  w.tabC = cv.take<uint64_t>((size_t)S * kPowTab);
  w.u = cv.take<uint64_t>(Tn);
  w.a = cv.take<uint64_t>(Tn);
  w.htab = cv.take<uint64_t>(H);
  w.bsum = cv.take<int64_t>(nbH + 1);
  w.gid = cv.take<int32_t>(H);
  w.U = cv.take<uint64_t>(Tn);
  w.cnt = cv.take<int32_t>(Tn);
  w.tg = cv.take<int32_t>(Tn);
  w.tp = cv.take<int32_t>(Tn);
  w.cbsum = cv.take<int64_t>(nbT + 1);
  w.start = cv.take<int64_t>(Tn);
  w.order = cv.take<int64_t>(Tn);
  const int64_t Tr = (fast && Tn <= kFastMaxT) ? 1 : Tn;   // kept when the fast path may fall back
  w.Wp = cv.take<uint64_t>((size_t)ring_words(S, Tr));
  w.UP = cv.take<uint64_t>((size_t)Tr * 32);
  w.UPq = cv.take<uint64_t>((size_t)Tr * 32);
  w.Uq = cv.take<uint64_t>(Tr);
  w.partial = cv.take<uint64_t>(Tr > 1 && gsplit > 1 ? (size_t)gsplit * S * (T > 0 ? T : 1) : 1);
  w.Gdev = cv.take<int64_t>(1);
  w.total = cv.take<int64_t>(1);
  return w;
}

// The merged weights in plain layout for the transposed tree:
// W[s G + g] = sum over group g's terms of a_t c_s^{e_{t,k}}, times u_g when
// the probes start at the first power (offset 1).
__global__ void k_eval_weights(int64_t G, int S, const int64_t* __restrict__ start, const int32_t* __restrict__ cnt,
                               const int64_t* __restrict__ order, const uint64_t* __restrict__ a,
                               const uint8_t* __restrict__ exps, int nv, int k, const uint64_t* __restrict__ tabC,
                               const uint64_t* __restrict__ U, int offset, Mod M, uint64_t* __restrict__ W) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < G * S; idx += stride) {
    const int64_t g = idx / S;
    const int s = (int)(idx - g * S);
    Acc8 acc{0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t* cs = tabC + (int64_t)s * kPowTab;
    const int64_t r0 = start[g], n = cnt[g];
    for (int64_t x = 0; x < n; x++) {
      const int64_t t = order[r0 + x];
      const uint64_t at = a[t], w = cs[exps[t * nv + k]];
      mac8(acc, lo32(at), hi32(at), lo32(w), hi32(w));
    }
    uint64_t r = acc8_value(acc, M);
    if (offset) r = mul_mod(r, U[g], M);
    W[(int64_t)s * G + g] = r;
  }
}

// The evaluation itself, with its scratch at `base` (capacity checked by the caller).
zr_status probes_enqueue(zr_ctx* ctx, const zr_poly* f, int k, const uint64_t* y, int S, const uint64_t* samples,
                         const uint64_t* z, int64_t T, int offset, uint64_t* out, int64_t ldo, uint32_t* status,
                         char* base, cudaStream_t st, char** fws, size_t* fcap) {
  if (!fws || !fcap) {
    fws = &ctx->fprobe_ws;
    fcap = &ctx->fprobe_cap;
  }
  const Mod& M = ctx->M;
  const int64_t Tf = f->T;
  const int nv = f->nv;
  const uint64_t H = hash_slots(Tf > 0 ? Tf : 1);
  const int64_t nbH = (int64_t)((H + kB - 1) / kB);
  const int gsplit = eval_gsplit(ctx, T, S, Tf);
  const bool fast = use_fast_probes(ctx, T, Tf, S);
  Carver cv(base);
  const EvalWs w = carve_eval(cv, Tf, nv, k, S, T, gsplit, fast);

  if (T <= 0) return ZR_OK;
  if (Tf == 0) {
    for (int s = 0; s < S; s++) cudaMemsetAsync(out + (int64_t)s * ldo, 0, sizeof(uint64_t) * T, st);
    return cuda_err(ctx, cudaGetLastError(), "zr_zippel_probes");
  }
  const int64_t Tn = Tf, nbT = (Tn + kB - 1) / kB;
  cudaMemsetAsync(w.htab, 0xFF, H * sizeof(uint64_t), st);
  cudaMemsetAsync(w.cnt, 0, (size_t)Tn * sizeof(int32_t), st);
  if (k > 0) { k_powrows<<<k, kPowTab, 0, st>>>(y, k, M, w.tabY); note_launch(); }
  if (z && nv > k + 1) { k_powrows<<<nv, kPowTab, 0, st>>>(z, nv, M, w.tabZ); note_launch(); }
  else cudaMemsetAsync(w.tabZ, 0, (size_t)nv * kPowTab * sizeof(uint64_t), st);
  { k_powrows<<<S, kPowTab, 0, st>>>(samples, S, M, w.tabC); note_launch(); }
  { k_eval_terms<<<cdiv(Tf, 256), 256, 0, st>>>(Tf, nv, f->exps, f->coef, k, w.tabY, w.tabZ, M, w.u, w.a, w.htab, H - 1); note_launch(); }
  // groups: the distinct u, numbered by a scan over the hash slots
  { k_slot_sums<<<(unsigned)nbH, kB, 0, st>>>((int64_t)H, w.htab, w.bsum); note_launch(); }
  { k_scan_small<<<1, kB, 0, st>>>(nbH, w.bsum, w.Gdev); note_launch(); }
  { k_slot_ids<<<(unsigned)nbH, kB, 0, st>>>((int64_t)H, w.htab, w.bsum, w.gid); note_launch(); }
  // the terms of each group, by a counting sort
  { k_eval_count<<<cdiv(Tf, 256), 256, 0, st>>>(Tf, w.u, w.htab, H - 1, w.gid, w.U, w.cnt, w.tg, w.tp, status); note_launch(); }
  { k_cnt_sums<<<(unsigned)nbT, kB, 0, st>>>(Tn, w.cnt, w.cbsum); note_launch(); }
  { k_scan_small<<<1, kB, 0, st>>>(nbT, w.cbsum, w.total); note_launch(); }
  { k_cnt_start<<<(unsigned)nbT, kB, 0, st>>>(Tn, w.cnt, w.cbsum, w.start); note_launch(); }
  { k_eval_scatter<<<cdiv(Tf, 256), 256, 0, st>>>(Tf, w.tg, w.tp, w.start, w.order); note_launch(); }
  // the transposed tree: its sizes follow the group count, read here (the
  // matrix-vector kernel below when there are more than kFastMaxT groups)
  int64_t G = 0;
  if (fast) {
    cudaError_t e = cudaMemcpyAsync(&G, w.Gdev, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_probes: group count");
    if (G < 1 || G > Tn) return set_err(ctx, ZR_ERR_CUDA, "zr_zippel_probes: group count out of range");
  }
  if (fast && G <= kFastMaxT) {
    cudaError_t e = cudaSuccess;
    const size_t wbytes = (((size_t)S * G * sizeof(uint64_t)) + 255) & ~(size_t)255;
    const size_t need = wbytes + fast_probes_ws_need(G, T, S);
    if (*fcap < need) {
      if (*fws) cudaFree(*fws);
      *fws = nullptr;
      *fcap = 0;
      e = cudaMalloc(fws, need + need / 4);
      if (e != cudaSuccess) {
        *fws = nullptr;
        return cuda_err(ctx, e, "zr_zippel_probes: fast workspace");
      }
      *fcap = need + need / 4;
    }
    uint64_t* W = reinterpret_cast<uint64_t*>(*fws);
    {
      const int64_t want = cdiv(G * S, 256), cap = 8ll * (ctx->sms ? ctx->sms : 152);
      k_eval_weights<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(G, S, w.start, w.cnt, w.order, w.a, f->exps,
                                                                          nv, k, w.tabC, w.U, offset, M, W);
      note_launch();
    }
    return fast_probes_enqueue(ctx, G, w.U, W, G, S, T, out, ldo, *fws + wbytes, st);
  }
  // the group count stays on the device: the kernels read it, sized for Tf groups
  const RingLayout L = ring_layout(S, Tn);
  int rw = 0;
  for (int b = 0; b < L.nb; b++) rw += L.bw[b];
  {
    const int64_t want = cdiv(Tn * rw, 256), cap = 8ll * (ctx->sms ? ctx->sms : 152);
    k_eval_finalize<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(w.Gdev, Tn, S, w.start, w.cnt, w.order, w.a,
                                                                         f->exps, nv, k, w.tabC, w.U, M, L, rw, w.Wp,
                                                                         w.UP, w.UPq, w.Uq);
    note_launch();
  }
  launch_ring(T, S, offset, w.Gdev, Tn, gsplit, w.UP, w.UPq, w.U, w.Uq, w.Wp, L, M, out, ldo, w.partial, status, st);
  if (gsplit > 1) { k_eval_combine<<<cdiv(T * S, 256), 256, 0, st>>>(T, S, gsplit, w.partial, M, out, ldo); note_launch(); }
  return cuda_err(ctx, cudaGetLastError(), "zr_zippel_probes");
}

size_t probes_ws_need(const zr_ctx* ctx, const zr_poly* f, int k, int S, int64_t T) {
  Carver cv(nullptr);
  carve_eval(cv, f->T, f->nv, k, S, T, eval_gsplit(ctx, T, S, f->T), use_fast_probes(ctx, T, f->T, S));
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
