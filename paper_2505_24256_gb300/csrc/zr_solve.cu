// zr_solve.cu -- the hot loop of the Zippel step: blocked synthetic division
// with the multi-right-hand-side deferred dot products (Sec. 2.2: a vector of
// powers generated in parallel, multiplied by the vector of values, and the
// modular addition deferred to one reduction per dot product).
#include <cuda_runtime.h>

#include "zr_kernels.cuh"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// a4: block partials of the tail Horner value for the k-blocked chain:
//   R_kb(v_j) = sum_{l in block kb} m_l v_j^{l - k_lo(kb)},  kb >= 1.
// ---------------------------------------------------------------------------

__global__ void k_carry_partials(int64_t T, int NB, int64_t BK, const uint64_t* __restrict__ m,
                                 const uint64_t* __restrict__ v, const uint64_t* __restrict__ vp, Mod M,
                                 uint64_t* __restrict__ R) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int kb = blockIdx.y + 1;
  if (j >= T || kb >= NB) return;
  const int64_t klo = kb * BK, khi = (klo + BK) < T ? (klo + BK) : T;
  const uint64_t vj = v[j], vpj = vp[j];
  uint64_t r = 0;
  for (int64_t l = khi - 1; l >= klo; l--) r = canon(shoup_lazy(r, vj, vpj, M), M) + __ldg(m + l);
  R[(int64_t)(kb - 1) * T + j] = canon(r, M);
}

void launch_carry_partials(const StepDims& D, const uint64_t* m, const uint64_t* v, const uint64_t* vp,
                           const Mod& M, uint64_t* R, cudaStream_t st) {
  if (D.NB <= 1) return;
  dim3 grid(cdiv(D.T, 256), D.NB - 1);
  { k_carry_partials<<<grid, 256, 0, st>>>(D.T, D.NB, D.BK, m, v, vp, M, R); note_launch(); }
}

// ---------------------------------------------------------------------------
// a4 + a5: the hot loop.  Thread = one root j, one k-block, one tile of ST
// right-hand sides.  Per k (descending):
//     acc_s += q_{j,k} b[s][k]           (deferred, carry-free MAC)
//     u      = u v_j + q_{j,k}             (Horner value q_j(v_j) of the block)
//     q      = m_k + v_j q_{j,k}           (synthetic division, Shoup multiply)
// Right-hand sides (MAC form) and m_k are staged in shared memory by cp.async,
// double buffered; every load is a broadcast.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int ST, int NT, int KC>
struct SolveSmem {
  uint4 bx[2][KC][ST][2];
  uint64_t m[2][KC];
};

template <int ST, int NT, int KC>
__device__ __forceinline__ void solve_stage(SolveSmem<ST, NT, KC>& sm, int buf, const BX* __restrict__ bx,
                                            const uint64_t* __restrict__ m, int S, int s0, int sn, int64_t clo,
                                            int len) {
  // bx rows k in [clo, clo+len), columns s0..s0+sn-1; zero padding for s >= sn.
  const int pieces = len * ST * 2;
  for (int t = threadIdx.x; t < pieces; t += NT) {
    int kk = t / (ST * 2), rem = t - kk * ST * 2, s = rem >> 1, h = rem & 1;
    uint4* dst = &sm.bx[buf][kk][s][h];
    if (s < sn) cp_async16(dst, reinterpret_cast<const uint4*>(bx + (clo + kk) * S + s0 + s) + h);
    else *dst = make_uint4(0, 0, 0, 0);
  }
  for (int t = threadIdx.x; t < len; t += NT) cp_async8(&sm.m[buf][t], m + clo + t);
}

template <int ST, int NT, int KC>
__global__ void __launch_bounds__(NT) k_solve(int64_t T, int S, int NB, int64_t BK, const uint64_t* __restrict__ m,
                                              const uint64_t* __restrict__ v, const uint64_t* __restrict__ vp,
                                              const uint64_t* __restrict__ R, const BX* __restrict__ bx, Mod M,
                                              uint64_t* __restrict__ part, uint64_t* __restrict__ denp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SolveSmem<ST, NT, KC>& sm = *reinterpret_cast<SolveSmem<ST, NT, KC>*>(smraw);
  const int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int kb = blockIdx.y;
  const int s0 = blockIdx.z * ST;
  const int sn = (S - s0) < ST ? (S - s0) : ST;
  const bool do_den = blockIdx.z == 0;
  const int64_t klo = kb * BK, khi = (klo + BK) < T ? (klo + BK) : T;
  const bool active = j < T;
  const uint64_t vj = active ? v[j] : 0, vpj = active ? vp[j] : 0;

  // carry-in q_{j, khi-1} = tail Horner value from khi (m_T = 1 at the top)
  uint64_t q = 1;
  if (active && kb < NB - 1) {
    const uint64_t vBK = pow_mod(vj, (uint64_t)BK, M);
    const uint64_t vtop = pow_mod(vj, (uint64_t)(T - (int64_t)(NB - 1) * BK), M);
    uint64_t c = 1;
    for (int kk = NB - 1; kk > kb; kk--) c = add_mod(R[(int64_t)(kk - 1) * T + j], mul_mod(kk == NB - 1 ? vtop : vBK, c, M), M);
    q = c;
  }
  uint64_t u = 0;
  Acc acc[ST];
#pragma unroll
  for (int s = 0; s < ST; s++) acc[s].L = acc[s].H = 0;
  int fold = 0;

  const int nchunks = (int)((khi - klo + KC - 1) / KC);
  // chunk c covers [chi - len, chi) with chi = khi - c KC (descending)
  auto chunk_lo = [&](int c, int& len) -> int64_t {
    int64_t chi = khi - (int64_t)c * KC;
    int64_t clo = chi - KC > klo ? chi - KC : klo;
    len = (int)(chi - clo);
    return clo;
  };
  {
    int len;
    int64_t clo = chunk_lo(0, len);
    solve_stage<ST, NT, KC>(sm, 0, bx, m, S, s0, sn, clo, len);
    cp_async_commit();
  }
  for (int c = 0; c < nchunks; c++) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      int len;
      int64_t clo = chunk_lo(c + 1, len);
      solve_stage<ST, NT, KC>(sm, buf ^ 1, bx, m, S, s0, sn, clo, len);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    int len;
    chunk_lo(c, len);
    for (int kk = len - 1; kk >= 0; kk--) {
      const uint64_t qc = canon(q, M);
      const XL x = limbs21(qc);
#pragma unroll
      for (int s = 0; s < ST; s++) {
        const uint4 b0 = sm.bx[buf][kk][s][0];
        const uint4 b1 = sm.bx[buf][kk][s][1];
        mac(acc[s], x, b0, make_uint2(b1.x, b1.y));
      }
      if (do_den) u = canon(shoup_lazy(u, vj, vpj, M), M) + qc;
      q = canon(shoup_lazy(qc, vj, vpj, M), M) + sm.m[buf][kk];
      if (++fold == MAC_FOLD) {
#pragma unroll
        for (int s = 0; s < ST; s++) acc_fold(acc[s], M);
        fold = 0;
      }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int s = 0; s < ST; s++)
      if (s < sn) part[((int64_t)kb * S + s0 + s) * T + j] = acc_value(acc[s], M);
    if (do_den) denp[(int64_t)kb * T + j] = canon(u, M);
  }
}

template <int ST, int NT, int KC>
static void launch_solve_t(const StepDims& D, const uint64_t* m, const uint64_t* v, const uint64_t* vp,
                           const uint64_t* R, const BX* bx, const Mod& M, uint64_t* part, uint64_t* denp,
                           cudaStream_t st) {
  const size_t smem = sizeof(SolveSmem<ST, NT, KC>);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_solve<ST, NT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  dim3 grid(cdiv(D.T, NT), D.NB, cdiv(D.S, ST));
  { k_solve<ST, NT, KC><<<grid, NT, smem, st>>>(D.T, D.S, D.NB, D.BK, m, v, vp, R, bx, M, part, denp); note_launch(); }
}

void launch_solve(const StepDims& D, const uint64_t* m, const uint64_t* v, const uint64_t* vp, const uint64_t* R,
                  const BX* bx, const Mod& M, uint64_t* part, uint64_t* denp, cudaStream_t st) {
  if (D.T <= 0 || D.S <= 0) return;
  switch (D.s_tile) {
    case 4: launch_solve_t<4, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 8: launch_solve_t<8, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 9: launch_solve_t<9, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 11: launch_solve_t<11, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 12: launch_solve_t<12, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 16: launch_solve_t<16, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    case 21: launch_solve_t<21, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
    default: launch_solve_t<24, 128, 32>(D, m, v, vp, R, bx, M, part, denp, st); break;
  }
}

}  // namespace zr
