// zr_arith.cuh -- device modular arithmetic for 64-bit residues (Sec. 2.1).
//
// The paper ports FLINT's precomputed-inverse reduction to CUDA (Sec. 2.1,
// Table 1: ~17x faster than the next variant) and defers the reduction of long
// dot products with a multi-word accumulator (Sec. 2.2).  This header is
// written from the published methods, for a GPU on which the 32-bit mad.lo
// issues at 64 lanes per SM per clock and mad.hi at 32 (measured), and the
// 32x32->64 mad.wide slower still:
//
//  * products are built from 32-bit mad.lo / mad.hi with carry chains;
//  * reduction of a 128-bit value uses the 2/1 division with a precomputed
//    reciprocal of Moller and Granlund ("Improved division by invariant
//    integers", IEEE TC 60(2), 2011, Algorithm 4) on the normalised modulus;
//  * multiplication by a value w fixed for a whole loop uses Shoup's
//    precomputed quotient w' = floor(w 2^64 / p) (as analysed in D. Harvey,
//    "Faster arithmetic for number-theoretic transforms", JSC 2014), with
//    results kept lazily in [0, 2p);
//  * long dot products add full 128-bit products into a 160-bit accumulator
//    (mac8) and reduce once: the deferred reduction of Sec. 2.2.
//
// The modulus is an odd prime 2^32 < p < 2^63, so 2p < 2^64.
#pragma once
#include <stdint.h>

namespace zr {

// Modulus descriptor, passed by value to kernels.
struct Mod {
  uint64_t p;       // the prime
  uint64_t d;       // p << norm (normalised divisor, top bit set)
  uint64_t v;       // floor((2^128 - 1) / d) - 2^64
  uint32_t norm;    // leading zero count of p, in [1, 31]
  uint32_t pad;
};

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return (uint32_t)x; }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }

// Products are built from 32-bit low/high multiply-adds with carry chains:
// on this GPU mad.lo issues at twice the rate of mad.hi and four times the
// rate of the 32x32->64 mad.wide, so a 32x32->64 product costs least as a
// (lo, hi) pair.

// Full 64x64 -> 128 product.
__device__ __forceinline__ void mul128(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
  const uint32_t a0 = lo32(a), a1 = hi32(a), b0 = lo32(b), b1 = hi32(b);
  uint32_t r0, r1, r2, r3;
  asm("mul.lo.u32 %0, %4, %6;\n\t"
      "mul.hi.u32 %1, %4, %6;\n\t"
      "mul.lo.u32 %2, %5, %7;\n\t"
      "mul.hi.u32 %3, %5, %7;\n\t"
      "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32 %3, %3, 0;"
      : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  lo = ((uint64_t)r1 << 32) | r0;
  hi = ((uint64_t)r3 << 32) | r2;
}

// High 64 bits of a 64x64 product (the low word of a0 b0 cannot carry into them).
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
  const uint32_t a0 = lo32(a), a1 = hi32(a), b0 = lo32(b), b1 = hi32(b);
  uint32_t t0, t1, t2;
  asm("mul.hi.u32 %0, %3, %5;\n\t"
      "mad.lo.cc.u32 %0, %3, %6, %0;\n\t"
      "madc.hi.u32 %1, %3, %6, 0;\n\t"
      "mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %5, %1;\n\t"
      "addc.u32 %2, 0, 0;\n\t"
      "mad.lo.cc.u32 %1, %4, %6, %1;\n\t"
      "madc.hi.u32 %2, %4, %6, %2;"
      : "=&r"(t0), "=&r"(t1), "=&r"(t2)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  (void)t0;   // only its carry reaches the high words
  return ((uint64_t)t2 << 32) | t1;
}

// Low 64 bits of a 64x64 product.
__device__ __forceinline__ uint64_t mullo64(uint64_t a, uint64_t b) {
  const uint32_t a0 = lo32(a), a1 = hi32(a), b0 = lo32(b), b1 = hi32(b);
  uint32_t r0, r1;
  asm("mul.lo.u32 %0, %2, %4;\n\t"
      "mul.hi.u32 %1, %2, %4;\n\t"
      "mad.lo.u32 %1, %2, %5, %1;\n\t"
      "mad.lo.u32 %1, %3, %4, %1;"
      : "=&r"(r0), "=&r"(r1)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  return ((uint64_t)r1 << 32) | r0;
}

// (u1 2^64 + u0) mod p for u1 < p (Moller-Granlund 2/1 division).  With
// COUNT (the arithmetic self-test only) the two correction steps are counted
// in hits[0] and hits[1]; the default form compiles without them.
template <bool COUNT = false>
__device__ __forceinline__ uint64_t reduce128(uint64_t u1, uint64_t u0, const Mod& M, uint32_t* hits = nullptr) {
  uint64_t n1 = (u1 << M.norm) | (u0 >> (64 - M.norm));
  uint64_t n0 = u0 << M.norm;
  uint64_t q1, q0;
  mul128(M.v, n1, q1, q0);
  q0 += n0;
  q1 += n1 + (q0 < n0);
  q1 += 1;
  uint64_t r = n0 - mullo64(q1, M.d);
  if (r > q0) {
    r += M.d;
    if (COUNT) atomicAdd(&hits[0], 1u);
  }
  if (r >= M.d) {
    r -= M.d;
    if (COUNT) atomicAdd(&hits[1], 1u);
  }
  return r >> M.norm;
}

// floor(w 2^64 / p) for w < p: the quotient of the same division (COUNT as
// for reduce128).
template <bool COUNT = false>
__device__ __forceinline__ uint64_t shoup_pre(uint64_t w, const Mod& M, uint32_t* hits = nullptr) {
  uint64_t n1 = w << M.norm, n0 = 0;
  uint64_t q1, q0;
  mul128(M.v, n1, q1, q0);
  q0 += n0;
  q1 += n1 + (q0 < n0);
  q1 += 1;
  uint64_t r = n0 - mullo64(q1, M.d);
  if (r > q0) {
    q1 -= 1;
    r += M.d;
    if (COUNT) atomicAdd(&hits[0], 1u);
  }
  if (r >= M.d) {
    q1 += 1;
    if (COUNT) atomicAdd(&hits[1], 1u);
  }
  return q1;
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, const Mod& M) {
  uint64_t s = a + b;                      // a, b < p < 2^63: no overflow
  return s >= M.p ? s - M.p : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, const Mod& M) {
  return a >= b ? a - b : a + (M.p - b);
}
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const Mod& M) {
  uint64_t hi, lo;
  mul128(a, b, hi, lo);
  return reduce128(hi, lo, M);             // a, b < p => hi < p
}
// x w mod p, lazily in [0, 2p), for any x < 2^64; wp = shoup_pre(w).
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t x, uint64_t w, uint64_t wp, const Mod& M) {
  const uint64_t q = mulhi64(x, wp);
  return mullo64(x, w) - mullo64(q, M.p);
}
__device__ __forceinline__ uint64_t canon(uint64_t x, const Mod& M) {  // [0, 2p) -> [0, p)
  return x >= M.p ? x - M.p : x;
}
__device__ __forceinline__ uint64_t pow_mod(uint64_t a, uint64_t e, const Mod& M) {
  uint64_t r = 1, x = a;
  while (e) {
    if (e & 1) r = mul_mod(r, x, M);
    x = mul_mod(x, x, M);
    e >>= 1;
  }
  return r;
}
// Inverse by Fermat's little theorem (p prime); 0 maps to 0.
__device__ __forceinline__ uint64_t inv_mod(uint64_t a, const Mod& M) { return pow_mod(a, M.p - 2, M); }

// ---------------------------------------------------------------------------
// Deferred multiply-accumulate: acc += x b for 64-bit x, b, reduced once.
// ---------------------------------------------------------------------------

// Even/odd split: x0 b0 and x1 b1 (bit offsets 0 and 64) go into r0..r4, the
// two cross products (bit offset 32) into t0..t2.  Two short independent
// carry chains per product instead of one long one: more instruction-level
// parallelism for the same eight multiplies.  r4 and t2 count carries, so
// fewer than 2^31 products never overflow.
struct Acc8 { uint32_t r0, r1, r2, r3, r4, t0, t1, t2; };
__device__ __forceinline__ void mac8(Acc8& a, uint32_t x0, uint32_t x1, uint32_t b0, uint32_t b1) {
  asm("mad.lo.cc.u32 %0, %8, %10, %0;\n\t"
      "madc.hi.cc.u32 %1, %8, %10, %1;\n\t"
      "madc.lo.cc.u32 %2, %9, %11, %2;\n\t"
      "madc.hi.cc.u32 %3, %9, %11, %3;\n\t"
      "addc.u32 %4, %4, 0;\n\t"
      "mad.lo.cc.u32 %5, %9, %10, %5;\n\t"
      "madc.hi.cc.u32 %6, %9, %10, %6;\n\t"
      "addc.u32 %7, %7, 0;\n\t"
      "mad.lo.cc.u32 %5, %8, %11, %5;\n\t"
      "madc.hi.cc.u32 %6, %8, %11, %6;\n\t"
      "addc.u32 %7, %7, 0;"
      : "+r"(a.r0), "+r"(a.r1), "+r"(a.r2), "+r"(a.r3), "+r"(a.r4), "+r"(a.t0), "+r"(a.t1), "+r"(a.t2)
      : "r"(x0), "r"(x1), "r"(b0), "r"(b1));
}
// residue of r + t 2^32
__device__ __forceinline__ uint64_t acc8_value(const Acc8& a, const Mod& M) {
  const uint64_t L = ((uint64_t)a.r1 << 32) | a.r0;
  const uint64_t Mi = ((uint64_t)a.r3 << 32) | a.r2;
  const uint64_t Tt = ((uint64_t)a.t2 << 32) | a.t1;
  const uint64_t L2 = L + ((uint64_t)a.t0 << 32);
  const uint64_t c1 = L2 < L;
  const uint64_t M1 = Mi + Tt;
  const uint64_t c2 = M1 < Mi;
  const uint64_t M2 = M1 + c1;
  const uint64_t c3 = M2 < M1;
  const uint64_t top = (uint64_t)a.r4 + c2 + c3;       // < 2^33 < p
  return reduce128(reduce128(top, M2, M), L2, M);
}
// The same with the corrections of both reductions counted (self-test only).
__device__ __forceinline__ uint64_t acc8_value_counted(const Acc8& a, const Mod& M, uint32_t* hits) {
  const uint64_t L = ((uint64_t)a.r1 << 32) | a.r0;
  const uint64_t Mi = ((uint64_t)a.r3 << 32) | a.r2;
  const uint64_t Tt = ((uint64_t)a.t2 << 32) | a.t1;
  const uint64_t L2 = L + ((uint64_t)a.t0 << 32);
  const uint64_t c1 = L2 < L;
  const uint64_t M1 = Mi + Tt;
  const uint64_t c2 = M1 < Mi;
  const uint64_t M2 = M1 + c1;
  const uint64_t c3 = M2 < M1;
  const uint64_t top = (uint64_t)a.r4 + c2 + c3;
  return reduce128<true>(reduce128<true>(top, M2, M, hits), L2, M, hits);
}


}  // namespace zr
