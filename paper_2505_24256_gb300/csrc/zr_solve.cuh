// zr_solve.cuh -- the hot loop of the Zippel step (a4 + a5), included by the
// translation units that instantiate it for their right-hand-side tiles.
#pragma once
#include <cuda_runtime.h>

#include "zr_device.cuh"
#include "zr_kernels.cuh"
#include "zr_ring.cuh"

namespace zr {

// ---------------------------------------------------------------------------
// a4 + a5: the hot loop, warp-specialised.  A work item is one entry, one
// tile of 32 roots j and one k-block; k runs downwards in chunks of KC.
//   warp 0 (producer)     lane = root: stages the right-hand sides of a chunk
//                         with cp.async, runs the synthetic-division chain
//                         q_{j,k-1} = m_k + v_j q_{j,k} and the Horner value
//                         u = u v_j + q_{j,k} of the block (Shoup multiplies),
//                         writes q to shared memory;
//   warps 1.. (consumers) G of them, lane = root: CG right-hand sides each,
//                         acc_s += q_{j,k} b[s][k] in 160-bit accumulators,
//                         reduced once per item.
// Chunks flow through a ring of NST shared-memory stages guarded by
// mbarriers ("full": the producer's 32 lanes arrive; "empty": one arrival
// per consumer warp), across item boundaries, so no warp waits for another
// except the consumers for a filled stage and the producer for the slowest
// consumer NST chunks back.  Every q_{j,k} is computed once and read by all
// G consumer warps, whatever S is.  (A second producer warp for u measured
// slower: the extra warp costs more occupancy than it frees issue slots.)
// ---------------------------------------------------------------------------

template <int CG, int G>
struct SolveCfg {
  static constexpr int RT = 32;               // roots per item: one per lane
  static constexpr int KC = 32;               // k per chunk
  static constexpr int NST = 4;               // ring stages
  static constexpr int CGP = (CG + 1) & ~1;   // a consumer's columns, padded to pairs
  static constexpr int BW = G * CGP;          // staged right-hand-side row width
  static constexpr int NT = 32 * (1 + G);     // threads per CTA: producer warp + G consumer warps
  // resident CTAs the register budget is sized for (measured register needs
  // of the consumer loop: about 8 CG accumulator words plus temporaries)
  static constexpr int REG = CG <= 2 ? 72 : (CG <= 3 ? 80 : (CG <= 4 ? 104 : (CG <= 6 ? 136 : 168)));
  static constexpr int FIT = 65536 / (NT * REG);
  static constexpr int MINB = FIT < 1 ? 1 : (FIT > 6 ? 6 : FIT);
  static constexpr size_t QB = sizeof(uint64_t) * NST * KC * RT;
  static constexpr size_t BB = sizeof(uint64_t) * NST * KC * BW;
  static constexpr size_t SMEM = QB + BB + sizeof(uint64_t) * 2 * NST;
};

template <int CG, int G>
__global__ void __launch_bounds__(SolveCfg<CG, G>::NT, SolveCfg<CG, G>::MINB)
    k_solve(const BDesc* __restrict__ Ds, const int4* __restrict__ items, int nitems, Mod M) {
  using C = SolveCfg<CG, G>;
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t(*qb)[C::KC][C::RT] = reinterpret_cast<uint64_t(*)[C::KC][C::RT]>(smraw);
  uint64_t(*bb)[C::KC][C::BW] = reinterpret_cast<uint64_t(*)[C::KC][C::BW]>(smraw + C::QB);
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + C::QB + C::BB);
  uint64_t* empty = full + C::NST;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0)
    for (int st = 0; st < C::NST; st++) {
      mbar_init(&full[st], 32);
      mbar_init(&empty[st], G);
    }
  __syncthreads();

  uint32_t cc = 0;   // chunks through the ring so far (same count in every warp)
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int4 wi = items[item];
    const BDesc& D = Ds[wi.x];
    const int64_t T = D.T, BK = D.BK;
    const int S = D.S, kb = wi.z;
    const int64_t j = (int64_t)wi.y * C::RT + lane;
    const bool live = j < T;
    const int64_t klo = kb * BK, khi = (klo + BK) < T ? (klo + BK) : T;
    const int nch = (int)((khi - klo + C::KC - 1) / C::KC);

    if (warp == 0) {
      // ---- producer warp
      const int NB = D.NB;
      uint64_t q = 1, u = 0, v = 0, vp = 0;
      if (live) {
        v = D.v[j];
        vp = D.vp[j];
        // carry-in q_{j, khi-1}: the tail Horner value of the blocks above
        // (the top block's partial includes m_T = 1)
        if (kb < NB - 1) {
          const uint64_t vBK = pow_mod(v, (uint64_t)BK, M);
          uint64_t cin = 0;
          for (int kk = NB - 1; kk > kb; kk--) cin = add_mod(D.R[(int64_t)(kk - 1) * T + j], mul_mod(vBK, cin, M), M);
          q = cin;
        }
      }
      const uint64_t* __restrict__ m = D.m;
      const uint64_t* __restrict__ b = D.b;
      const int64_t ldb = D.ldb;
      // m_k of a chunk, one per lane, is loaded a chunk ahead so that the
      // chain never waits for it
      auto m_chunk = [&](int c) -> uint64_t {
        const int64_t chi = khi - (int64_t)c * C::KC;
        const int64_t clo = chi - C::KC > klo ? chi - C::KC : klo;
        return (c < nch && lane < chi - clo) ? __ldg(m + clo + lane) : 0;
      };
      uint64_t mnext = m_chunk(0);
      for (int c = 0; c < nch; c++, cc++) {
        const int st = cc % C::NST;
        const uint32_t ph = (cc / C::NST) & 1;
        if (cc >= (uint32_t)C::NST && !mbar_wait(&empty[st], ph ^ 1)) {
          atomicOr(D.status, ST_TIMEOUT);
          cp_async_wait<0>();
          return;
        }
        const int64_t chi = khi - (int64_t)c * C::KC;
        const int64_t clo = chi - C::KC > klo ? chi - C::KC : klo;
        const int len = (int)(chi - clo);
        // right-hand sides of the chunk, [k][consumer][column]: lane = k, so
        // every row s is read coalesced
        for (int kk = lane; kk < len; kk += 32)
          for (int s = 0; s < S; s++) {
            const int gs = s / CG;
            cp_async8(&bb[st][kk][gs * C::CGP + (s - gs * CG)], b + (int64_t)s * ldb + clo + kk);
          }
        cp_async_commit();
        // m_k of the chunk, one per lane, broadcast by shuffle along the chain
        const uint64_t mreg = mnext;
        mnext = m_chunk(c + 1);
        uint64_t(*qw)[C::RT] = qb[st];
        for (int kk = len - 1; kk >= 0; kk--) {
          const uint64_t mk = __shfl_sync(0xffffffffu, mreg, kk);
          const uint64_t qc = canon(q, M);
          qw[kk][lane] = qc;
          u = canon(shoup_lazy(u, v, vp, M), M) + qc;
          q = canon(shoup_lazy(qc, v, vp, M), M) + mk;
        }
        cp_async_wait<0>();
        mbar_arrive(&full[st]);
      }
      if (live) D.denp[(int64_t)kb * T + j] = canon(u, M);
    } else {
      // ---- consumer g: columns g*CG .. g*CG + CG - 1
      const int g = warp - 1;
      Acc8 acc[CG];
#pragma unroll
      for (int q = 0; q < CG; q++) acc[q] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
      for (int c = 0; c < nch; c++, cc++) {
        const int st = cc % C::NST;
        const uint32_t ph = (cc / C::NST) & 1;
        if (!mbar_wait(&full[st], ph)) {
          atomicOr(D.status, ST_TIMEOUT);
          return;
        }
        const int64_t chi = khi - (int64_t)c * C::KC;
        const int len = (int)(chi - (chi - C::KC > klo ? chi - C::KC : klo));
        if (len == C::KC) {
          // a full chunk: unrolled, so the loads of later k overlap the MACs
#pragma unroll
          for (int kk = 0; kk < C::KC; kk++) {
            const uint64_t x = qb[st][kk][lane];
            const uint32_t x0 = lo32(x), x1 = hi32(x);
            const uint64_t* row = &bb[st][kk][g * C::CGP];
#pragma unroll
            for (int q = 0; q + 1 < CG; q += 2) {
              const uint4 w = *reinterpret_cast<const uint4*>(row + q);
              mac8(acc[q], x0, x1, w.x, w.y);
              mac8(acc[q + 1], x0, x1, w.z, w.w);
            }
            if (CG & 1) {
              const uint2 w = *reinterpret_cast<const uint2*>(row + CG - 1);
              mac8(acc[CG - 1], x0, x1, w.x, w.y);
            }
          }
        } else {
#pragma unroll 1
          for (int kk = 0; kk < len; kk++) {
            const uint64_t x = qb[st][kk][lane];
            const uint32_t x0 = lo32(x), x1 = hi32(x);
            const uint64_t* row = &bb[st][kk][g * C::CGP];
#pragma unroll
            for (int q = 0; q + 1 < CG; q += 2) {
              const uint4 w = *reinterpret_cast<const uint4*>(row + q);
              mac8(acc[q], x0, x1, w.x, w.y);
              mac8(acc[q + 1], x0, x1, w.z, w.w);
            }
            if (CG & 1) {
              const uint2 w = *reinterpret_cast<const uint2*>(row + CG - 1);
              mac8(acc[CG - 1], x0, x1, w.x, w.y);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
      }
      const int s0 = g * CG;
      if (live) {
#pragma unroll
        for (int q = 0; q < CG; q++)
          if (s0 + q < S) D.part[((int64_t)kb * S + s0 + q) * T + j] = acc8_value(acc[q], M);
      }
    }
  }
  if (warp == 0) cp_async_wait<0>();
}

template <int CG, int G>
static int solve_occupancy_t() {
  using C = SolveCfg<CG, G>;
  int n = 0;
  cudaFuncSetAttribute(k_solve<CG, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_solve<CG, G>, C::NT, C::SMEM) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

template <int CG, int G>
static void launch_solve_t(const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
  using C = SolveCfg<CG, G>;
  static DeviceValue occ;
  const int per_sm = occ.get(solve_occupancy_t<CG, G>);   // also sets the shared-memory attribute
  // persistent: one wave walks the work list; sms <= 0: one CTA per item
  const int grid = (sms <= 0 || nitems < sms * per_sm) ? nitems : sms * per_sm;
  if (grid > 0) { k_solve<CG, G><<<grid, C::NT, C::SMEM, st>>>(Ds, items, nitems, M); note_launch(); }
}

// Instances of one tile for every consumer-warp count in [GLO, 8].
template <int CG, int GLO>
struct SolveTile {
  static bool exists(int g) { return g >= GLO && g <= 8; }
  static int occupancy(int g) {
    switch (g) {
      case 1: if constexpr (GLO <= 1) return solve_occupancy_t<CG, 1>(); break;
      case 2: if constexpr (GLO <= 2) return solve_occupancy_t<CG, 2>(); break;
      case 3: if constexpr (GLO <= 3) return solve_occupancy_t<CG, 3>(); break;
      case 4: if constexpr (GLO <= 4) return solve_occupancy_t<CG, 4>(); break;
      case 5: return solve_occupancy_t<CG, 5>();
      case 6: return solve_occupancy_t<CG, 6>();
      case 7: return solve_occupancy_t<CG, 7>();
      case 8: return solve_occupancy_t<CG, 8>();
      default: break;
    }
    return 0;
  }
  static bool launch(int g, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
    switch (g) {
      case 1: if constexpr (GLO <= 1) { launch_solve_t<CG, 1>(Ds, items, nitems, sms, M, st); return true; } break;
      case 2: if constexpr (GLO <= 2) { launch_solve_t<CG, 2>(Ds, items, nitems, sms, M, st); return true; } break;
      case 3: if constexpr (GLO <= 3) { launch_solve_t<CG, 3>(Ds, items, nitems, sms, M, st); return true; } break;
      case 4: if constexpr (GLO <= 4) { launch_solve_t<CG, 4>(Ds, items, nitems, sms, M, st); return true; } break;
      case 5: launch_solve_t<CG, 5>(Ds, items, nitems, sms, M, st); return true;
      case 6: launch_solve_t<CG, 6>(Ds, items, nitems, sms, M, st); return true;
      case 7: launch_solve_t<CG, 7>(Ds, items, nitems, sms, M, st); return true;
      case 8: launch_solve_t<CG, 8>(Ds, items, nitems, sms, M, st); return true;
      default: break;
    }
    return false;
  }
};

// per translation unit: occupancy (0: no instance) and launch for (cg, g)
int solve_occupancy_narrow(int cg, int g);
bool solve_launch_narrow(int cg, int g, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                         cudaStream_t st);
int solve_occupancy_wide(int cg, int g);
bool solve_launch_wide(int cg, int g, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                       cudaStream_t st);

}  // namespace zr
