// zr_solve.cu -- the hot loop of the Zippel step: blocked synthetic division
// with the multi-right-hand-side deferred dot products (Sec. 2.2: a vector of
// powers generated in parallel, multiplied by the vector of values, and the
// modular addition deferred to one reduction per dot product).
#include <cuda_runtime.h>

#include "zr_device.cuh"
#include "zr_kernels.cuh"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// a4: block partials of the tail Horner value for the k-blocked chain:
//   R_kb(v_j) = sum_{l in block kb} m_l v_j^{l - k_lo(kb)},  kb >= 1.
// One CTA = 256 roots of one entry and one k-block (flattened over a batch).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_b_carry(const BDesc* __restrict__ Ds, const int64_t* __restrict__ pre, int n,
                                                 Mod M) {
  const int i = seg_of(pre, n, blockIdx.x);
  const BDesc& D = Ds[i];
  const int64_t local = blockIdx.x - pre[i];
  const int64_t rows = (D.T + 255) / 256;
  const int kb = 1 + (int)(local / rows);
  const int64_t j = (local % rows) * 256 + threadIdx.x;
  if (j >= D.T) return;
  const int64_t klo = kb * D.BK, khi = (klo + D.BK) < D.T ? (klo + D.BK) : D.T;
  const uint64_t vj = D.v[j], vpj = D.vp[j];
  const uint64_t* __restrict__ m = D.m;
  uint64_t r = 0;
  for (int64_t l = khi - 1; l >= klo; l--) r = canon(shoup_lazy(r, vj, vpj, M), M) + __ldg(m + l);
  D.R[(int64_t)(kb - 1) * D.T + j] = canon(r, M);
}

void launch_b_carry(const BDesc* Ds, const int64_t* pre, int n, int64_t nctas, const Mod& M, cudaStream_t st) {
  if (nctas > 0) { k_b_carry<<<(unsigned)nctas, 256, 0, st>>>(Ds, pre, n, M); note_launch(); }
}

// ---------------------------------------------------------------------------
// a4 + a5: the hot loop.  Thread = one root j, one k-block, one tile of ST
// right-hand sides.  Per k (descending):
//     acc_s += q_{j,k} b[s][k]           (even/odd lo/hi carry chains, reduced once)
//     u      = u v_j + q_{j,k}             (Horner value q_j(v_j) of the block)
//     q      = m_k + v_j q_{j,k}           (synthetic division, Shoup multiply)
// The right-hand sides (plain residues, 8 bytes each) and m_k are staged in
// shared memory by cp.async, double buffered; every load is a broadcast and
// two right-hand sides arrive per 16-byte load.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int ST, int KC>
struct SolveSmem {
  static constexpr int STP = (ST + 1) & ~1;   // padded to pairs
  uint64_t b[2][KC][STP];
  uint64_t m[2][KC];
};

template <int ST, int NT, int KC>
__device__ __forceinline__ void solve_stage(SolveSmem<ST, KC>& sm, int buf, const uint64_t* __restrict__ b,
                                            int64_t ldb, const uint64_t* __restrict__ m, int s0, int sn,
                                            int64_t clo, int len) {
  constexpr int STP = SolveSmem<ST, KC>::STP;
  const int pieces = STP * len;
  for (int t = threadIdx.x; t < pieces; t += NT) {
    const int s = t / len, kk = t - s * len;        // consecutive threads walk k: coalesced reads
    uint64_t* dst = &sm.b[buf][kk][s];
    if (s < sn) cp_async8(dst, b + (int64_t)(s0 + s) * ldb + clo + kk);
    else *dst = 0;
  }
  for (int t = threadIdx.x; t < len; t += NT) cp_async8(&sm.m[buf][t], m + clo + t);
}

// resident CTAs per SM the compiler is asked to fit (register budget)
template <int ST>
struct SolveMinBlocks { static constexpr int value = ST <= 6 ? 4 : (ST <= 12 ? 3 : 2); };

template <int ST, int NT, int KC>
__global__ void __launch_bounds__(NT, SolveMinBlocks<ST>::value) k_solve(const BDesc* __restrict__ Ds,
                                                                         const int4* __restrict__ items, int nitems,
                                                                         Mod M) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SolveSmem<ST, KC>& sm = *reinterpret_cast<SolveSmem<ST, KC>*>(smraw);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int4 wi = items[item];
    const BDesc& D = Ds[wi.x];
    const int64_t T = D.T, BK = D.BK, ldb = D.ldb;
    const int S = D.S, NB = D.NB;
    const uint64_t* __restrict__ m = D.m;
    const uint64_t* __restrict__ b = D.b;
    const int64_t j = (int64_t)wi.y * NT + threadIdx.x;
    const int kb = wi.z;
    const int s0 = wi.w * ST;
    const int sn = (S - s0) < ST ? (S - s0) : ST;
    const bool do_den = wi.w == 0;
    const int64_t klo = kb * BK, khi = (klo + BK) < T ? (klo + BK) : T;
    const bool active = j < T;
    const uint64_t vj = active ? D.v[j] : 0, vpj = active ? D.vp[j] : 0;

    // carry-in q_{j, khi-1} = tail Horner value from khi (m_T = 1 at the top)
    uint64_t q = 1;
    if (active && kb < NB - 1) {
      const uint64_t vBK = pow_mod(vj, (uint64_t)BK, M);
      const uint64_t vtop = pow_mod(vj, (uint64_t)(T - (int64_t)(NB - 1) * BK), M);
      uint64_t c = 1;
      for (int kk = NB - 1; kk > kb; kk--)
        c = add_mod(D.R[(int64_t)(kk - 1) * T + j], mul_mod(kk == NB - 1 ? vtop : vBK, c, M), M);
      q = c;
    }
    uint64_t u = 0;
    Acc8 acc[ST];
#pragma unroll
    for (int s = 0; s < ST; s++) acc[s] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};

    const int nchunks = (int)((khi - klo + KC - 1) / KC);
    auto chunk_lo = [&](int c, int& len) -> int64_t {
      int64_t chi = khi - (int64_t)c * KC;
      int64_t clo = chi - KC > klo ? chi - KC : klo;
      len = (int)(chi - clo);
      return clo;
    };
    {
      int len;
      int64_t clo = chunk_lo(0, len);
      solve_stage<ST, NT, KC>(sm, 0, b, ldb, m, s0, sn, clo, len);
      cp_async_commit();
    }
    for (int c = 0; c < nchunks; c++) {
      const int buf = c & 1;
      if (c + 1 < nchunks) {
        int len;
        int64_t clo = chunk_lo(c + 1, len);
        solve_stage<ST, NT, KC>(sm, buf ^ 1, b, ldb, m, s0, sn, clo, len);
      }
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      int len;
      chunk_lo(c, len);
      for (int kk = len - 1; kk >= 0; kk--) {
        const uint64_t qc = canon(q, M);
        const uint32_t x0 = lo32(qc), x1 = hi32(qc);
        const uint4* row = reinterpret_cast<const uint4*>(&sm.b[buf][kk][0]);
#pragma unroll
        for (int s = 0; s + 1 < ST; s += 2) {
          const uint4 w = row[s >> 1];
          mac8(acc[s], x0, x1, w.x, w.y);
          mac8(acc[s + 1], x0, x1, w.z, w.w);
        }
        if (ST & 1) {
          const uint2 w = reinterpret_cast<const uint2*>(row)[ST - 1];
          mac8(acc[ST - 1], x0, x1, w.x, w.y);
        }
        if (do_den) u = canon(shoup_lazy(u, vj, vpj, M), M) + qc;
        q = canon(shoup_lazy(qc, vj, vpj, M), M) + sm.m[buf][kk];
      }
      __syncthreads();
    }
    if (active) {
#pragma unroll
      for (int s = 0; s < ST; s++)
        if (s < sn) D.part[((int64_t)kb * S + s0 + s) * T + j] = acc8_value(acc[s], M);
      if (do_den) D.denp[(int64_t)kb * T + j] = canon(u, M);
    }
    __syncthreads();
  }
}

template <int ST, int NT, int KC>
static void launch_solve_t(const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st);

template <int ST, int NT, int KC>
static int solve_occupancy_t();

template <int ST, int NT, int KC>
static void launch_solve_t(const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M, cudaStream_t st) {
  const size_t smem = sizeof(SolveSmem<ST, KC>);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_solve<ST, NT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int per_sm = solve_occupancy_t<ST, NT, KC>();
  const int grid = nitems < sms * per_sm ? nitems : sms * per_sm;   // persistent: one wave walks the work list
  if (grid > 0) { k_solve<ST, NT, KC><<<grid, NT, smem, st>>>(Ds, items, nitems, M); note_launch(); }
}

template <int ST, int NT, int KC>
static int solve_occupancy_t() {
  int n = 0;
  const size_t smem = sizeof(SolveSmem<ST, KC>);
  cudaFuncSetAttribute(k_solve<ST, NT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_solve<ST, NT, KC>, NT, smem) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

#define ZR_SOLVE_TILES(X) X(4) X(6) X(8) X(9) X(11) X(12) X(16) X(21)

int solve_tiles(int* out, int cap) {
  static const int t[] = {4, 6, 8, 9, 11, 12, 16, 21};
  int n = 0;
  for (int x : t)
    if (n < cap) out[n++] = x;
  return n;
}

int solve_blocks_per_sm(int s_tile) {
  switch (s_tile) {
#define ZR_CASE(ST) \
  case ST: return solve_occupancy_t<ST, 128, 32>();
    ZR_SOLVE_TILES(ZR_CASE)
#undef ZR_CASE
    default: return 1;
  }
}

void launch_b_solve(int s_tile, const BDesc* Ds, const int4* items, int nitems, int sms, const Mod& M,
                    cudaStream_t st) {
  if (nitems <= 0) return;
  switch (s_tile) {
#define ZR_CASE(ST) \
  case ST: launch_solve_t<ST, 128, 32>(Ds, items, nitems, sms, M, st); break;
    ZR_SOLVE_TILES(ZR_CASE)
#undef ZR_CASE
    default: break;
  }
}

}  // namespace zr
