// zr_peak.cu -- measured ceilings of the integer pipes the solve runs on.
//
// The solve's time goes into two instruction sequences: the deferred
// multiply-accumulate of a residue into a 160-bit accumulator (mac8, Sec. 2.2)
// and the Shoup multiply of the synthetic-division chain (Sec. 2.1).  Each
// probe below runs one of them, or a single 32-bit multiply-add form, with
// every operand in registers and enough independent accumulators per thread
// that nothing waits on a dependency; every SM runs as many blocks as fit.
// The rates are what the roofline of the solve is measured against.  A fifth
// probe runs the butterfly of the number-theoretic transforms (Harvey's
// forward butterfly on 32-bit residues with a Shoup twiddle), the ceiling of
// the transform kernels of the O(T log^2 T) solve.
#include <cuda_runtime.h>

#include "zr_internal.h"
#include "zr_ntt.cuh"

namespace zr {

namespace {

constexpr int kPeakThreads = 128;
constexpr int kMacCols = 12;      // independent 160-bit accumulators per thread
constexpr int kChains = 8;        // independent chains per thread
constexpr int kMads = 16;         // independent 32-bit accumulators per thread
constexpr int kBfly = 16;         // residues per thread in the butterfly probe: two radix-8 groups

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// kind 0: mac8, kind 1: chain step, kind 2: mad.lo, kind 3: mad.hi,
// kind 4: forward butterflies, three radix-2 stages over each group of eight
// residues per round (24 butterflies).
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, uint64_t seed, Mod M, uint32_t* __restrict__ sink,
                                                        int write) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t h = (seed + tid) * 0x9E3779B97F4A7C15ull;
  h ^= h >> 29;
  uint32_t out = 0;
  if (KIND == 0) {
    Acc8 a[kMacCols];
    uint32_t b0[kMacCols], b1[kMacCols];
#pragma unroll
    for (int c = 0; c < kMacCols; c++) {
      a[c] = Acc8{0, 0, 0, 0, 0, 0, 0, 0};
      const uint64_t bv = (h * (2 * c + 3)) >> 1;
      b0[c] = lo32(bv);
      b1[c] = hi32(bv) & 0x7fffffffu;
    }
    uint32_t x0 = lo32(h), x1 = hi32(h) & 0x7fffffffu;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int c = 0; c < kMacCols; c++) mac8(a[c], x0, x1, b0[c], b1[c]);
      x0 += 0x9E3779B9u;      // a fresh multiplier each round, as the chain gives the solve
    }
#pragma unroll
    for (int c = 0; c < kMacCols; c++) out ^= a[c].r0 ^ a[c].r4 ^ a[c].t1;
  } else if (KIND == 1) {
    uint64_t q[kChains];
    const uint64_t v = (h >> 2) % M.p, m = (h >> 5) % M.p;
    const uint64_t vp = shoup_pre(v, M);
#pragma unroll
    for (int r = 0; r < kChains; r++) q[r] = (h + r) % M.p;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int r = 0; r < kChains; r++) q[r] = canon(shoup_lazy(canon(q[r], M), v, vp, M), M) + m;
    }
#pragma unroll
    for (int r = 0; r < kChains; r++) out ^= lo32(q[r]);
  } else if (KIND == 4) {
    constexpr uint32_t q = 998244353u;           // the first transform prime
    uint32_t x[kBfly];
    uint2 w[7];
#pragma unroll
    for (int r = 0; r < kBfly; r++) x[r] = (uint32_t)((h >> (r & 31)) % q);
#pragma unroll
    for (int r = 0; r < 7; r++) {
      const uint32_t wv = (uint32_t)(((h >> 3) * (r + 1)) % q);
      w[r] = make_uint2(wv, (uint32_t)(((uint64_t)wv << 32) / q));
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int gbase = 0; gbase < kBfly; gbase += 8) {
#pragma unroll
        for (int i = 0; i < 4; i++) butterfly<false>(x[gbase + i], x[gbase + i + 4], w[0], q);
#pragma unroll
        for (int i = 0; i < 8; i++)
          if (!(i & 2)) butterfly<false>(x[gbase + i], x[gbase + i + 2], w[1 + (i >> 2)], q);
#pragma unroll
        for (int i = 0; i < 8; i += 2) butterfly<false>(x[gbase + i], x[gbase + i + 1], w[3 + (i >> 1)], q);
      }
    }
#pragma unroll
    for (int r = 0; r < kBfly; r++) out ^= x[r];
  } else {
    uint32_t a[kMads];
    const uint32_t x = lo32(h) | 1u, y = hi32(h);
#pragma unroll
    for (int r = 0; r < kMads; r++) a[r] = y + r;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int r = 0; r < kMads; r++) a[r] = KIND == 2 ? mad_lo(a[r], x, a[r]) : mad_hi(a[r], x, a[r]);
    }
#pragma unroll
    for (int r = 0; r < kMads; r++) out ^= a[r];
  }
  if (write) sink[tid] = out;      // never true at run time; keeps the work live
}

template <int KIND>
zr_status time_probe(zr_ctx* ctx, cudaStream_t st, uint32_t* sink, double ops_per_iter, double* rate) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak<KIND>, kPeakThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = ctx->sms * per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // size the timed launch from a short one: about 30 ms of work
  int iters = 256;
  float ms = 0;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
    cudaEventRecord(e0, st);
    k_peak<KIND><<<grid, kPeakThreads, 0, st>>>(iters, 0x5eed + rep, ctx->M, sink, 0);
    note_launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep < 2) {
      const double scale = ms > 0.01 ? 30.0 / ms : 64.0;
      double next = iters * scale;
      if (next > (1 << 24)) next = 1 << 24;
      if (next < 256) next = 256;
      iters = (int)next;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_measure_peaks");
  *rate = (double)grid * kPeakThreads * (double)iters * ops_per_iter / (ms * 1e-3);
  return ZR_OK;
}

}  // namespace
}  // namespace zr

using namespace zr;

extern "C" zr_status zr_measure_peaks(zr_ctx* ctx, zr_peaks* out, void* stream) {
  if (!ctx || !out) return ZR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = (int64_t)ctx->sms * 2048;
  zr_status r = ensure_ws(ctx, 4 * (size_t)n, st);
  if (r) return r;
  uint32_t* sink = reinterpret_cast<uint32_t*>(ctx->ws);
  zr_peaks p{};
  if (!r) r = time_probe<0>(ctx, st, sink, kMacCols, &p.mac_per_s);
  if (!r) r = time_probe<1>(ctx, st, sink, kChains, &p.chain_per_s);
  if (!r) r = time_probe<2>(ctx, st, sink, kMads, &p.imad_lo_per_s);
  if (!r) r = time_probe<3>(ctx, st, sink, kMads, &p.imad_hi_per_s);
  if (!r) r = time_probe<4>(ctx, st, sink, 3 * kBfly / 2, &p.butterfly_per_s);
  if (r) return r;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess) p.sms = prop.multiProcessorCount;
  *out = p;
  return ZR_OK;
}
