// zr_check.cu -- the device modular arithmetic applied to operand arrays, for
// the parity test of the arithmetic core against the oracle (Sec. 2.1: the
// 64-bit modular product with a precomputed reciprocal; Sec. 2.2: long dot
// products accumulated without reduction and reduced once).
//
// Every case calls the same inline functions the step kernels use
// (zr_arith.cuh, warp_batch_inverse in zr_device.cuh), so the test drives the
// production arithmetic on chosen operands: edges, values that reach the
// rare correction steps of the Moller-Granlund division, lazy inputs in
// [p, 2^64), and sums of up to 2^31 full products.
#include <cuda_runtime.h>

#include "zr_device.cuh"
#include "zr_internal.h"

namespace zr {
namespace {

// op codes of zr_check_arith (the header lists them)
enum { OP_MULMOD = 0, OP_REDUCE, OP_SHOUP_PRE, OP_SHOUP_LAZY, OP_POW, OP_INV, OP_DOT, OP_ADD, OP_SUB, OP_BATCH_INV };

__global__ void __launch_bounds__(256) k_check_arith(int op, int64_t n, int64_t len, const uint64_t* __restrict__ a,
                                                     const uint64_t* __restrict__ b, Mod M, uint64_t* __restrict__ out,
                                                     uint32_t* hits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t* hr = hits;                       // corrections of reduce128
  uint32_t* hs = hits ? hits + 2 : nullptr;  // corrections of shoup_pre
  if (op == OP_BATCH_INV) {
    // whole warps take part; lanes past n invert 1 and write nothing
    const uint64_t x = i < n ? a[i] : 1;
    const uint64_t r = warp_batch_inverse(x, M);
    if (i < n) out[i] = r;
    return;
  }
  if (i >= n) return;
  uint64_t r = 0;
  switch (op) {
    case OP_MULMOD: {
      uint64_t hi, lo;
      mul128(a[i], b[i], hi, lo);
      r = hits ? reduce128<true>(hi, lo, M, hr) : reduce128(hi, lo, M);
      break;
    }
    case OP_REDUCE: r = hits ? reduce128<true>(a[i], b[i], M, hr) : reduce128(a[i], b[i], M); break;
    case OP_SHOUP_PRE: r = hits ? shoup_pre<true>(a[i], M, hs) : shoup_pre(a[i], M); break;
    case OP_SHOUP_LAZY: r = shoup_lazy(a[i], b[i], shoup_pre(b[i], M), M); break;
    case OP_POW: r = pow_mod(a[i], b[i], M); break;
    case OP_INV: r = inv_mod(a[i], M); break;
    case OP_DOT: {
      Acc8 acc = {0, 0, 0, 0, 0, 0, 0, 0};
      const uint64_t* x = a + i * len;
      const uint64_t* y = b + i * len;
      for (int64_t t = 0; t < len; t++) mac8(acc, lo32(x[t]), hi32(x[t]), lo32(y[t]), hi32(y[t]));
      r = hits ? acc8_value_counted(acc, M, hr) : acc8_value(acc, M);
      break;
    }
    case OP_ADD: r = add_mod(a[i], b[i], M); break;
    case OP_SUB: r = sub_mod(a[i], b[i], M); break;
    default: break;
  }
  out[i] = r;
}

}  // namespace
}  // namespace zr

using namespace zr;

extern "C" zr_status zr_check_arith(zr_ctx* ctx, int32_t op, int64_t n, int64_t len, const uint64_t* a,
                                    const uint64_t* b, uint64_t* out, uint32_t* hits, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (op < OP_MULMOD || op > OP_BATCH_INV || n < 0 || (op == OP_DOT && (len < 1 || len >= (1ll << 31))))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_check_arith: op or sizes out of range");
  const bool needs_b = op == OP_MULMOD || op == OP_REDUCE || op == OP_SHOUP_LAZY || op == OP_POW || op == OP_DOT ||
                       op == OP_ADD || op == OP_SUB;
  if (n > 0 && (!a || !out || (needs_b && !b))) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_check_arith: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0) {
    const int64_t blocks = (n + 255) / 256;
    k_check_arith<<<(unsigned)blocks, 256, 0, st>>>(op, n, op == OP_DOT ? len : 1, a, b, ctx->M, out, hits);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_err(ctx, e, "zr_check_arith");
}
