// zr_lift.cu -- rational numbers from modular images.
//
// The reconstruction runs modulo large primes; the rational numbers are
// recovered as a final step (Sec. 1).  Per value, one thread:
//
//  * Chinese remaindering by Garner's mixed radix: digits
//      v_0 = r_0,  v_i = (r_i - (v_0 + v_1 p_0 + ... + v_{i-1} p_0..p_{i-2})) C_i  (mod p_i),
//      C_i = (p_0 .. p_{i-1})^-1 mod p_i,
//    then x = v_0 + p_0 (v_1 + p_1 (v_2 + ...)) as a W-word integer, x < P;
//  * rational reconstruction (Wang's method): the extended Euclidean
//    algorithm on (P, x), each quotient applied by shift-and-subtract (its
//    bits, high to low, to the remainder and to the cofactor of x), stopped
//    at the first remainder r <= N = floor(sqrt((P - 1) / 2)); with cofactor
//    t the value is sign(t) r / |t|, accepted when 0 < |t| <= N and
//    gcd(r, |t|) = 1 (binary gcd).  2 N^2 < P makes the answer unique.
//
// Words are little-endian uint64; the cofactors are two's complement over W
// words (|t| <= P < 2^(64 W - 2)).
#include <cuda_runtime.h>

#include "zr_internal.h"

namespace zr {

namespace {

constexpr int kMaxPrimes = 8;

struct LiftParams {
  int L;                    // primes
  Mod M[kMaxPrimes];
  uint64_t C[kMaxPrimes];   // Garner constants
  uint64_t P[kMaxPrimes];   // product of the primes, W words
  uint64_t N[kMaxPrimes];   // the bound floor(sqrt((P - 1) / 2)), W words
};

// ---- W-word unsigned / two's complement integers ------------------------------

template <int W>
__host__ __device__ inline int big_bitlen(const uint64_t* a) {
  for (int i = W - 1; i >= 0; i--)
    if (a[i]) {
      int b = 0;
      uint64_t x = a[i];
      while (x) {
        b++;
        x >>= 1;
      }
      return 64 * i + b;
    }
  return 0;
}
template <int W>
__host__ __device__ inline bool big_is_zero(const uint64_t* a) {
  uint64_t o = 0;
  for (int i = 0; i < W; i++) o |= a[i];
  return o == 0;
}
// a <=> b, unsigned
template <int W>
__host__ __device__ inline int big_cmp(const uint64_t* a, const uint64_t* b) {
  for (int i = W - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  return 0;
}
// word i of b << s (s >= 0)
template <int W>
__host__ __device__ inline uint64_t big_shl_word(const uint64_t* b, int s, int i) {
  const int ws = s >> 6, bs = s & 63;
  const int j = i - ws;
  if (j < 0) return 0;
  uint64_t x = b[j] << bs;
  if (bs && j > 0) x |= b[j - 1] >> (64 - bs);
  return x;
}
// a >= (b << s), unsigned, with b << s < 2^(64 W)
template <int W>
__host__ __device__ inline bool big_ge_shl(const uint64_t* a, const uint64_t* b, int s) {
  for (int i = W - 1; i >= 0; i--) {
    const uint64_t x = big_shl_word<W>(b, s, i);
    if (a[i] != x) return a[i] > x;
  }
  return true;
}
// a -= b << s (mod 2^(64 W))
template <int W>
__host__ __device__ inline void big_sub_shl(uint64_t* a, const uint64_t* b, int s) {
  uint64_t borrow = 0;
  for (int i = 0; i < W; i++) {
    const uint64_t x = big_shl_word<W>(b, s, i);
    const uint64_t d = a[i] - x;
    const uint64_t b1 = a[i] < x;
    a[i] = d - borrow;
    borrow = b1 | (d < borrow);
  }
}
template <int W>
__host__ __device__ inline void big_add(uint64_t* a, const uint64_t* b) {
  uint64_t carry = 0;
  for (int i = 0; i < W; i++) {
    const uint64_t s = a[i] + b[i];
    const uint64_t c1 = s < a[i];
    a[i] = s + carry;
    carry = c1 | (a[i] < s);
  }
}
template <int W>
__host__ __device__ inline void big_shr1(uint64_t* a) {
  for (int i = 0; i < W; i++) a[i] = (a[i] >> 1) | (i + 1 < W ? a[i + 1] << 63 : 0);
}
template <int W>
__host__ __device__ inline void big_shr2(uint64_t* a) {
  big_shr1<W>(a);
  big_shr1<W>(a);
}
template <int W>
__host__ __device__ inline void big_neg(uint64_t* a) {
  uint64_t carry = 1;
  for (int i = 0; i < W; i++) {
    const uint64_t x = ~a[i] + carry;
    carry = carry && x == 0;
    a[i] = x;
  }
}
// a = a m + c (m, c < 2^64)
template <int W>
__host__ __device__ inline void big_mul_add(uint64_t* a, uint64_t m, uint64_t c) {
  uint64_t carry = c;
  for (int i = 0; i < W; i++) {
    const unsigned __int128 t = (unsigned __int128)a[i] * m + carry;
    a[i] = (uint64_t)t;
    carry = (uint64_t)(t >> 64);
  }
}
// floor(sqrt(n)) by the digit-by-digit method (shifts, adds, compares)
template <int W>
void big_isqrt(const uint64_t* n, uint64_t* res) {
  uint64_t op[W], one[W], t[W];
  for (int i = 0; i < W; i++) op[i] = n[i], res[i] = 0, one[i] = 0;
  int b = big_bitlen<W>(n);
  if (b == 0) return;
  b = (b - 1) & ~1;   // highest power of four <= n
  one[b >> 6] = 1ull << (b & 63);
  while (!big_is_zero<W>(one)) {
    for (int i = 0; i < W; i++) t[i] = res[i];
    big_add<W>(t, one);
    if (big_cmp<W>(op, t) >= 0) {
      big_sub_shl<W>(op, t, 0);
      big_shr1<W>(res);
      big_add<W>(res, one);
    } else {
      big_shr1<W>(res);
    }
    big_shr2<W>(one);
  }
}

// gcd(a, b) == 1, both nonnegative (binary gcd; a, b are consumed)
template <int W>
__device__ inline bool big_coprime(uint64_t* a, uint64_t* b) {
  if (big_is_zero<W>(a)) return b[0] == 1 && big_bitlen<W>(b) == 1;
  if (big_is_zero<W>(b)) return a[0] == 1 && big_bitlen<W>(a) == 1;
  if (!(a[0] & 1) && !(b[0] & 1)) return false;
  while (!(b[0] & 1)) big_shr1<W>(b);
  while (!big_is_zero<W>(a)) {
    while (!(a[0] & 1)) big_shr1<W>(a);
    if (big_cmp<W>(a, b) >= 0) big_sub_shl<W>(a, b, 0);
    else {
      big_sub_shl<W>(b, a, 0);
      for (int i = 0; i < W; i++) {   // keep b odd and a the difference
        const uint64_t x = a[i];
        a[i] = b[i];
        b[i] = x;
      }
    }
  }
  return b[0] == 1 && big_bitlen<W>(b) == 1;
}

template <int W>
__global__ void __launch_bounds__(128) k_lift(LiftParams prm, int64_t n, const uint64_t* __restrict__ res, int64_t ld,
                                             int words, uint64_t* __restrict__ num, uint64_t* __restrict__ den,
                                             int32_t* __restrict__ ok) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int L = prm.L;
  // Garner's mixed-radix digits
  uint64_t v[kMaxPrimes];
  for (int i = 0; i < L; i++) {
    const Mod& Mi = prm.M[i];
    const uint64_t r = reduce128(0, res[(int64_t)i * ld + j], Mi);
    uint64_t t = 0;
    for (int q = i - 1; q >= 0; q--) t = add_mod(mul_mod(t, reduce128(0, prm.M[q].p, Mi), Mi), reduce128(0, v[q], Mi), Mi);
    v[i] = i == 0 ? r : mul_mod(sub_mod(r, t, Mi), prm.C[i], Mi);
  }
  uint64_t x[W];
  for (int w = 0; w < W; w++) x[w] = 0;
  for (int i = L - 1; i >= 0; i--) big_mul_add<W>(x, i == L - 1 ? 0 : prm.M[i].p, v[i]);
  // extended Euclid on (P, x) down to the first remainder <= N
  uint64_t r0[W], r1[W], t0[W], t1[W];
  for (int w = 0; w < W; w++) r0[w] = prm.P[w], r1[w] = x[w], t0[w] = 0, t1[w] = w == 0;
  while (big_cmp<W>(r1, prm.N) > 0) {
    for (int s = big_bitlen<W>(r0) - big_bitlen<W>(r1); s >= 0; s--)
      if (big_ge_shl<W>(r0, r1, s)) {
        big_sub_shl<W>(r0, r1, s);
        big_sub_shl<W>(t0, t1, s);
      }
    for (int w = 0; w < W; w++) {
      uint64_t a = r0[w];
      r0[w] = r1[w];
      r1[w] = a;
      a = t0[w];
      t0[w] = t1[w];
      t1[w] = a;
    }
  }
  const bool neg = (t1[W - 1] >> 63) != 0;
  if (neg) big_neg<W>(t1);
  bool good = !big_is_zero<W>(t1) && big_cmp<W>(t1, prm.N) <= 0;
  uint64_t a[W], b[W];
  for (int w = 0; w < W; w++) a[w] = r1[w], b[w] = t1[w];
  good = good && big_coprime<W>(a, b);
  if (good && neg) big_neg<W>(r1);
  const uint64_t ext = (good && neg) ? ~0ull : 0;
  for (int w = 0; w < words; w++) {
    num[j * words + w] = good ? (w < W ? r1[w] : ext) : 0;
    den[j * words + w] = good ? (w < W ? t1[w] : 0) : 0;
  }
  ok[j] = good ? 1 : 0;
}

uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }
uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  a %= p;
  while (e) {
    if (e & 1) r = host_mulmod(r, a, p);
    a = host_mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}

template <int W>
void lift_bounds(LiftParams& prm) {
  uint64_t P[W] = {}, h[W], N[W];
  P[0] = 1;
  for (int i = 0; i < prm.L; i++) big_mul_add<W>(P, prm.M[i].p, 0);
  // N = isqrt((P - 1) / 2)
  for (int w = 0; w < W; w++) h[w] = P[w];
  uint64_t one[W] = {};
  one[0] = 1;
  big_sub_shl<W>(h, one, 0);
  big_shr1<W>(h);
  big_isqrt<W>(h, N);
  for (int w = 0; w < kMaxPrimes; w++) {
    prm.P[w] = w < W ? P[w] : 0;
    prm.N[w] = w < W ? N[w] : 0;
  }
}

}  // namespace

}  // namespace zr

using namespace zr;

extern "C" int32_t zr_lift_words(int32_t nprimes) {
  if (nprimes < 1 || nprimes > kMaxPrimes) return 0;
  return nprimes <= 2 ? 2 : (nprimes <= 4 ? 4 : 8);
}

extern "C" zr_status zr_rational_lift(zr_ctx* ctx, int32_t nprimes, const uint64_t* primes, int64_t n,
                                      const uint64_t* res, int64_t ld, int32_t words, uint64_t* num, uint64_t* den,
                                      int32_t* ok, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  const int W = zr_lift_words(nprimes);
  if (!W || !primes || n < 0 || ld < n || words < W || (n > 0 && (!res || !num || !den || !ok)))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_rational_lift: arguments out of range");
  LiftParams prm{};
  prm.L = nprimes;
  for (int i = 0; i < nprimes; i++) {
    if (!mod_for_prime(primes[i], &prm.M[i]))
      return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_rational_lift: each modulus must be a prime in (2^32, 2^63)");
    for (int q = 0; q < i; q++)
      if (primes[q] == primes[i]) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_rational_lift: primes must differ");
  }
  for (int i = 0; i < nprimes; i++) {
    uint64_t m = 1;
    for (int q = 0; q < i; q++) m = host_mulmod(m, primes[q] % primes[i], primes[i]);
    prm.C[i] = host_powmod(m, primes[i] - 2, primes[i]);   // Fermat: p_i is prime
  }
  if (W == 2) lift_bounds<2>(prm);
  else if (W == 4) lift_bounds<4>(prm);
  else lift_bounds<8>(prm);
  if (n == 0) return ZR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((n + 127) / 128);
  if (W == 2) k_lift<2><<<grid, 128, 0, st>>>(prm, n, res, ld, words, num, den, ok);
  else if (W == 4) k_lift<4><<<grid, 128, 0, st>>>(prm, n, res, ld, words, num, den, ok);
  else k_lift<8><<<grid, 128, 0, st>>>(prm, n, res, ld, words, num, den, ok);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_err(ctx, e, "zr_rational_lift");
}
