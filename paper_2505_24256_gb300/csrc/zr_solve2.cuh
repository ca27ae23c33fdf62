// zr_solve2.cuh -- the O(T^2) solve's hot loop (a4 + a5) with every warp
// running its own synthetic-division chain.
//
// A work item is one entry, a tile of W x 32 roots, one k-block and one group
// of CG right-hand sides.  Warp w of the CTA owns roots w*32 .. w*32+31 of the
// tile (lane = root) and keeps the group's CG dot products in 160-bit
// accumulators in registers:
//     acc_s += q_{j,k} b[s][k]                          (Sec. 2.2: deferred sum)
//     q_{j,k-1} = m_k + v_j q_{j,k},  u = u v_j + q_{j,k}  (Shoup multiplies)
// u (the block's Horner value toward q_j(v_j)) is run by group 0 only.  The
// right-hand sides and m of a chunk of KC values of k are staged in shared
// memory by cp.async (NST stages, all threads copy), and every lane of every
// warp reads the same staged words (broadcast loads).  Per root and k the
// chain costs two Shoup steps against CG multiply-accumulates, so for the
// usual S (9 to 21) one group holds every right-hand side and the mad.hi
// pipe spends nearly all of its time on the dot products, with no
// producer/consumer hand-off between warps.
#pragma once
#include <cuda_runtime.h>

#include "zr_device.cuh"
#include "zr_kernels.cuh"
#include "zr_ring.cuh"

namespace zr {

template <int CG, int W>
struct Solve2Cfg {
  static constexpr int KC = 32;               // k per chunk
  static constexpr int NST = 3;               // staging buffers
  static constexpr int CGP = (CG + 1) & ~1;   // staged row width (pairs: 16-byte loads)
  static constexpr int NT = 32 * W;
  static constexpr int RT = 32 * W;           // roots per item
  // registers: 8 per accumulator plus the chain and addressing
  static constexpr int REG = 10 * CG + 72;
  static constexpr int FIT = 65536 / (NT * (REG > 255 ? 255 : REG));
  static constexpr int MINB = FIT < 1 ? 1 : (FIT > 8 ? 8 : FIT);
  static constexpr size_t BB = sizeof(uint64_t) * NST * KC * CGP;
  static constexpr size_t MB = sizeof(uint64_t) * NST * KC;
  static constexpr size_t SMEM = BB + MB;
};

template <int CG, int W>
__global__ void __launch_bounds__(Solve2Cfg<CG, W>::NT, Solve2Cfg<CG, W>::MINB)
    k_solve2(const BDesc* __restrict__ Ds, const int4* __restrict__ items, int nitems, Mod M) {
  using C = Solve2Cfg<CG, W>;
  extern __shared__ __align__(16) unsigned char smraw2[];
  uint64_t(*bs)[C::KC][C::CGP] = reinterpret_cast<uint64_t(*)[C::KC][C::CGP]>(smraw2);
  uint64_t(*ms)[C::KC] = reinterpret_cast<uint64_t(*)[C::KC]>(smraw2 + C::BB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int4 wi = items[item];
    const BDesc& D = Ds[wi.x];
    const int64_t T = D.T, BK = D.BK;
    const int S = D.S, kb = wi.z, g = wi.w;
    const int c0 = g * CG;
    const int cols = (S - c0) < CG ? (S - c0) : CG;
    const int64_t j = (int64_t)wi.y * C::RT + warp * 32 + lane;
    const bool live = j < T;
    const int64_t klo = kb * BK, khi = (klo + BK) < T ? (klo + BK) : T;
    const int nch = (int)((khi - klo + C::KC - 1) / C::KC);
    const uint64_t* __restrict__ b = D.b;
    const uint64_t* __restrict__ m = D.m;
    const int64_t ldb = D.ldb;

    uint64_t q = 1, u = 0, v = 0, vp = 0;
    if (live) {
      v = D.v[j];
      vp = D.vp[j];
      // carry-in q_{j, khi-1}: the tail Horner value of the blocks above
      // (the top block's partial includes m_T = 1)
      if (kb < D.NB - 1) {
        const uint64_t vBK = pow_mod(v, (uint64_t)BK, M);
        uint64_t cin = 0;
        for (int kk = D.NB - 1; kk > kb; kk--) cin = add_mod(D.R[(int64_t)(kk - 1) * T + j], mul_mod(vBK, cin, M), M);
        q = cin;
      }
    }
    Acc8 acc[CG];
#pragma unroll
    for (int c = 0; c < CG; c++) acc[c] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};

    // chunk c covers k in [khi - (c+1) KC, khi - c KC) clipped at klo; its
    // right-hand sides are staged with lanes walking k (each row read
    // coalesced), columns of the group beyond S as zeros
    for (int c = 0; c < nch + C::NST - 1; c++) {
      if (c < nch) {
        const int st = c % C::NST;
        const int64_t chi = khi - (int64_t)c * C::KC;
        const int64_t clo = chi - C::KC > klo ? chi - C::KC : klo;
        const int len = (int)(chi - clo);
        for (int e = tid; e < C::KC * C::CGP; e += C::NT) {
          const int col = e / C::KC, kk = e - col * C::KC;
          if (kk < len && col < cols) cp_async8(&bs[st][kk][col], b + (int64_t)(c0 + col) * ldb + clo + kk);
          else bs[st][kk][col] = 0;
        }
        for (int kk = tid; kk < len; kk += C::NT) cp_async8(&ms[st][kk], m + clo + kk);
      }
      cp_async_commit();                          // one group per iteration, empty past the last chunk
      const int cc = c - (C::NST - 1);            // the chunk consumed in this iteration
      if (cc < 0) continue;
      cp_async_wait<C::NST - 1>();
      __syncthreads();
      const int st = cc % C::NST;
      const int64_t chi = khi - (int64_t)cc * C::KC;
      const int len = (int)(chi - (chi - C::KC > klo ? chi - C::KC : klo));
      const uint64_t(*row)[C::CGP] = bs[st];
      const uint64_t* mk = ms[st];
#pragma unroll 1
      for (int kk = len - 1; kk >= 0; kk--) {
        const uint64_t qc = canon(q, M);
        const uint32_t x0 = lo32(qc), x1 = hi32(qc);
#pragma unroll
        for (int t = 0; t + 1 < CG; t += 2) {
          const uint4 w = *reinterpret_cast<const uint4*>(&row[kk][t]);
          mac8(acc[t], x0, x1, w.x, w.y);
          mac8(acc[t + 1], x0, x1, w.z, w.w);
        }
        if (CG & 1) {
          const uint2 w = *reinterpret_cast<const uint2*>(&row[kk][CG - 1]);
          mac8(acc[CG - 1], x0, x1, w.x, w.y);
        }
        if (g == 0) u = canon(shoup_lazy(u, v, vp, M), M) + qc;
        q = canon(shoup_lazy(qc, v, vp, M), M) + mk[kk];
      }
      __syncthreads();                            // the stage is refilled next
    }
    cp_async_wait<0>();
    if (live) {
#pragma unroll
      for (int c = 0; c < CG; c++)
        if (c < cols) D.part[((int64_t)kb * S + c0 + c) * T + j] = acc8_value(acc[c], M);
      if (g == 0) D.denp[(int64_t)kb * T + j] = canon(u, M);
    }
  }
}

template <int CG, int W>
static int solve2_occupancy_t() {
  using C = Solve2Cfg<CG, W>;
  int n = 0;
  cudaFuncSetAttribute(k_solve2<CG, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_solve2<CG, W>, C::NT, C::SMEM) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

template <int CG, int W>
static void launch_solve2_t(const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
  using C = Solve2Cfg<CG, W>;
  static DeviceValue occ;
  const int per_sm = occ.get(solve2_occupancy_t<CG, W>);   // also sets the shared-memory attribute
  const int grid = (sms <= 0 || nitems < sms * per_sm) ? nitems : sms * per_sm;
  if (grid > 0) { k_solve2<CG, W><<<grid, C::NT, C::SMEM, st>>>(Ds, items, nitems, M); note_launch(); }
}

// warps per CTA of each column-group width
constexpr int solve2_warps(int cg) { return cg <= 8 ? 8 : 4; }

}  // namespace zr
