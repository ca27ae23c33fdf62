// zr_ntt.cuh -- polynomial products modulo the 63-bit prime through
// number-theoretic transforms over five word-size primes.
//
// p = 2^63 - 25 has 2-adic valuation 1 (p - 1 = 2 * odd), so it has no
// transform of its own.  A product of two polynomials with coefficients below
// p and inner length n <= 2^21 has integer coefficients below n p^2 < 2^147;
// it is computed exactly modulo five primes q_i = c_i 2^23 + 1 < 2^30
// (product about 2^148.1), combined by the Chinese remainder theorem (Garner's
// mixed radix) and reduced modulo p.
//
// Residue arithmetic follows Harvey ("Faster arithmetic for number-theoretic
// transforms", JSC 2014): twiddles are multiplied with Shoup's precomputed
// quotient and values are kept lazily in [0, 2q) or [0, 4q) (q < 2^30, so
// 4q < 2^32); general products use Montgomery's reduction with R = 2^32.
// The forward transform is Cooley-Tukey (natural order in, bit-reversed out),
// the inverse Gentleman-Sande (bit-reversed in, natural out), both driven by
// one table tw[m + i] = w_{2m}^{brev_m(i)} shared by every size: products of
// spectra never need the permutation.
#pragma once
#include <stdint.h>

#include "zr_arith.cuh"

namespace zr {

constexpr int kNP = 5;                 // transform primes
constexpr int kNttMaxLog = 22;         // largest transform: 2^22
constexpr int kNttTile = 8192;         // elements a CTA transforms in shared memory
constexpr int kNttTileLog = 13;
constexpr int kNttThreads = 256;

// Per-context constants of the transform primes and of the Chinese
// remaindering into residues modulo p (host-computed, passed by value).
struct NttConsts {
  uint32_t q[kNP];           // the primes
  uint32_t g[kNP];           // a primitive root of each
  uint32_t qinv[kNP];        // q^-1 mod 2^32
  uint32_t r32[kNP], r32p[kNP];   // 2^32 mod q and its Shoup quotient
  uint32_t onep[kNP];        // floor(2^32 / q): Shoup quotient of 1
  uint32_t gc[kNP][kNP], gcp[kNP][kNP];   // q_j^-1 mod q_i (j < i) and Shoup quotients
  uint64_t pre[kNP];         // prod_{j < i} q_j mod p
};

// Scale applied to every residue before Chinese remaindering: undoes the
// 1/n of an inverse transform of size n and the 2^-32 of one Montgomery
// product (s = 2^32 / n mod q), with Shoup quotients.
struct CrtScale {
  uint32_t s[kNP], sp[kNP];
};

// x w mod q in [0, 2q) for any 32-bit x, w < q, wp = floor(w 2^32 / q).
__device__ __forceinline__ uint32_t shoup32(uint32_t x, uint32_t w, uint32_t wp, uint32_t q) {
  return x * w - __umulhi(x, wp) * q;
}
// a b 2^-32 mod q in [0, q) for a b < q 2^32 (a, b < 2q suffices).
__device__ __forceinline__ uint32_t mont32(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv) {
  const uint32_t lo = a * b, hi = __umulhi(a, b);
  const uint32_t m = lo * qinv;
  const uint32_t u = __umulhi(m, q);
  const uint32_t r = hi - u;
  return (int32_t)r < 0 ? r + q : r;
}
__device__ __forceinline__ uint32_t sub_if(uint32_t x, uint32_t b) { return x >= b ? x - b : x; }

// Harvey's butterflies with a Shoup twiddle: forward (CT) X, Y < 4q -> < 4q;
// inverse (GS) X, Y < 2q -> < 2q.
template <bool INV>
__device__ __forceinline__ void butterfly(uint32_t& X, uint32_t& Y, uint2 w, uint32_t q) {
  if (!INV) {
    const uint32_t x = sub_if(X, 2 * q);
    const uint32_t t = shoup32(Y, w.x, w.y, q);
    X = x + t;
    Y = x - t + 2 * q;
  } else {
    const uint32_t x = X, y = Y;
    X = sub_if(x + y, 2 * q);
    Y = shoup32(x - y + 2 * q, w.x, w.y, q);
  }
}

// A 64-bit value's residue modulo q_i, in [0, 4q): hi 2^32 + lo.
__device__ __forceinline__ uint32_t residue64(uint64_t x, const NttConsts& C, int i) {
  const uint32_t q = C.q[i];
  return shoup32(hi32(x), C.r32[i], C.r32p[i], q) + shoup32(lo32(x), 1u, C.onep[i], q);
}

// Garner: residues r_i in [0, 2q_i) (already scaled) -> the integer's residue mod p.
__device__ __forceinline__ uint64_t crt_to_p(const uint32_t (&r)[kNP], const NttConsts& C, const Mod& M) {
  uint32_t y[kNP];
#pragma unroll
  for (int i = 0; i < kNP; i++) {
    const uint32_t q = C.q[i];
    uint32_t t = sub_if(r[i], q);
#pragma unroll
    for (int j = 0; j < i; j++) {
      const uint32_t yj = sub_if(y[j], q);          // y_j < q_j < 2 q_i
      t = sub_if(shoup32(t + q - yj, C.gc[i][j], C.gcp[i][j], q), q);
    }
    y[i] = t;
  }
  // sum_i y_i prod_{j<i} q_j, taken modulo p: y_i < 2^30, pre_i < 2^63
  uint64_t lo = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < kNP; i++) {
    uint64_t ph, pl;
    mul128(C.pre[i], (uint64_t)y[i], ph, pl);
    lo += pl;
    hi += ph + (lo < pl);
  }
  return reduce128(hi, lo, M);       // hi < 2^33 < p
}

}  // namespace zr
