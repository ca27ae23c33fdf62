// zr_balance.cu -- the balanced Zippel step for rational functions (Sec. 1,
// Sec. 2.2, the balancing identity) and its univariate rational
// reconstruction (Thiele, Eq. thiele).
//
// For probe i the black box gives f(y^(i+off), c_s) for the Sf samples c_s.
// One thread per probe runs Thiele interpolation in the new variable:
//   inverse differences phi_l(x_t) = (x_t - x_{l-1}) / (phi_{l-1}(x_t) - b_{l-1}),
//   b_l = phi_l(x_l), stopped at the first level whose tail is constant on the
//   remaining samples, then the convergent P_L/Q_L of
//   b_0 + (x - x_0)/(b_1 + (x - x_1)/(b_2 + ...)) expanded to coefficients and
//   scaled so that Q(c_0) = 1: n_i = P/Q(c_0), d_i = Q/Q(c_0).
// The inverses of one level are taken together (Montgomery's trick: one
// Fermat inversion per level).  The balancing factor is the previous
// denominator skeleton at the probe, D'(y^(i+off)) = C D(y^i, c_0); with
// d_i(c_0) = 1 it turns the reduced pair into
//   bN[s][i] = D'(y^i) n_i(c_s) = C N(y^i, c_s),   bD[s][i] = D'(y^i) d_i(c_s) = C D(y^i, c_s),
// the probes of one Zippel step for N and one for D with a common scale C.
// (The paper takes the ratio from the numerator skeleton; the denominator
// gives the same factor C/h_i and cannot vanish away from poles.)
#include <cuda_runtime.h>

#include "zr_internal.h"

namespace zr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Per-probe scratch, column i of row-major [row][Tmax] arrays:
//   phi (n rows), bl (n rows), pre (n rows), P and Q (3 x (n+1) rows each)
struct ThieleScratch {
  uint64_t *phi, *bl, *pre, *P, *Q;
};

__global__ void k_thiele_balance(int64_t Tmax, int n, const uint64_t* __restrict__ xs,
                                 const uint64_t* __restrict__ fvals, int64_t ldf,
                                 const uint64_t* __restrict__ dprev, int dN, int dD, int64_t TN, int64_t TD,
                                 ThieleScratch sc, Mod M, uint64_t* __restrict__ bN, int64_t ldN,
                                 uint64_t* __restrict__ bD, int64_t ldD, uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Tmax) return;
  const int64_t ld = Tmax;
  auto PHI = [&](int t) -> uint64_t& { return sc.phi[(int64_t)t * ld + i]; };
  auto BL = [&](int t) -> uint64_t& { return sc.bl[(int64_t)t * ld + i]; };
  auto PRE = [&](int t) -> uint64_t& { return sc.pre[(int64_t)t * ld + i]; };
  const int W = n + 1;
  auto Pr = [&](int row, int e) -> uint64_t& { return sc.P[((int64_t)row * W + e) * ld + i]; };
  auto Qr = [&](int row, int e) -> uint64_t& { return sc.Q[((int64_t)row * W + e) * ld + i]; };

  for (int t = 0; t < n; t++) {
    uint64_t x = fvals[(int64_t)t * ldf + i];
    PHI(t) = x >= M.p ? x - M.p : x;
  }
  BL(0) = PHI(0);
  int L = -1;
  for (int l = 1; l < n; l++) {
    const uint64_t b = BL(l - 1);
    bool all_eq = true, any_eq = false;
    for (int t = l; t < n; t++) {
      if (PHI(t) == b) any_eq = true;
      else all_eq = false;
    }
    if (all_eq) { L = l - 1; break; }
    if (any_eq) { atomicOr(status, ST_THIELE); return; }
    // batch inversion of d_t = phi(t) - b, t = l..n-1
    uint64_t acc = 1;
    for (int t = l; t < n; t++) {
      acc = mul_mod(acc, sub_mod(PHI(t), b, M), M);
      PRE(t) = acc;
    }
    uint64_t inv = inv_mod(acc, M);
    for (int t = n - 1; t >= l; t--) {
      const uint64_t d = sub_mod(PHI(t), b, M);
      const uint64_t it = t > l ? mul_mod(inv, PRE(t - 1), M) : inv;    // 1 / d_t
      inv = mul_mod(inv, d, M);
      PHI(t) = mul_mod(sub_mod(xs[t], xs[l - 1], M), it, M);
    }
    BL(l) = PHI(l);
  }
  if (L < 0) { atomicOr(status, ST_DEGREE); return; }
  // convergents: rows 0 = level l-2, 1 = level l-1, 2 = level l
  for (int e = 0; e < W; e++) {
    Pr(0, e) = e == 0 ? 1 : 0;  Qr(0, e) = 0;
    Pr(1, e) = e == 0 ? BL(0) : 0;  Qr(1, e) = e == 0 ? 1 : 0;
  }
  int r2 = 0, r1 = 1, rc = 2;
  for (int l = 1; l <= L; l++) {
    const uint64_t bl = BL(l), xl = xs[l - 1];
    const int emax = (l + 1) / 2 + 1 < W ? (l + 1) / 2 + 1 : W;     // degrees grow by at most one every level
    for (int e = 0; e < W; e++) {
      if (e > emax) { Pr(rc, e) = 0; Qr(rc, e) = 0; continue; }
      const uint64_t sp = sub_mod(e ? Pr(r2, e - 1) : 0, mul_mod(xl, Pr(r2, e), M), M);
      const uint64_t sq = sub_mod(e ? Qr(r2, e - 1) : 0, mul_mod(xl, Qr(r2, e), M), M);
      Pr(rc, e) = add_mod(mul_mod(bl, Pr(r1, e), M), sp, M);
      Qr(rc, e) = add_mod(mul_mod(bl, Qr(r1, e), M), sq, M);
    }
    const int t = r2;
    r2 = r1;
    r1 = rc;
    rc = t;
  }
  // normalise Q(c_0) = 1
  uint64_t q0 = 0;
  for (int e = W - 1; e >= 0; e--) q0 = add_mod(mul_mod(q0, xs[0], M), Qr(r1, e), M);
  if (q0 == 0) { atomicOr(status, ST_POLE); return; }
  const uint64_t s = inv_mod(q0, M);
  int degp = -1, degq = -1;
  for (int e = 0; e < W; e++) {
    const uint64_t a = mul_mod(Pr(r1, e), s, M), c = mul_mod(Qr(r1, e), s, M);
    Pr(r1, e) = a;
    Qr(r1, e) = c;
    if (a) degp = e;
    if (c) degq = e;
  }
  if (degp >= n || degq >= n || degp > dN || degq > dD) { atomicOr(status, ST_DEGREE); return; }
  const uint64_t fac = dprev[i] >= M.p ? dprev[i] - M.p : dprev[i];
  if (i < TN)
    for (int t = 0; t <= dN; t++) {
      uint64_t v = 0;
      for (int e = degp; e >= 0; e--) v = add_mod(mul_mod(v, xs[t], M), Pr(r1, e), M);
      bN[(int64_t)t * ldN + i] = mul_mod(fac, v, M);
    }
  if (i < TD)
    for (int t = 0; t <= dD; t++) {
      uint64_t v = 0;
      for (int e = degq; e >= 0; e--) v = add_mod(mul_mod(v, xs[t], M), Qr(r1, e), M);
      bD[(int64_t)t * ldD + i] = mul_mod(fac, v, M);
    }
}

// f = N / D elementwise with pole detection: one thread per column i, the
// S divisions of a column share one inversion (Montgomery's trick).
__global__ void k_ratio(int64_t T, int S, const uint64_t* __restrict__ Nv, const uint64_t* __restrict__ Dv, int64_t ld,
                        Mod M, uint64_t* __restrict__ pre, uint64_t* __restrict__ out, int64_t ldo, uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T) return;
  uint64_t acc = 1;
  for (int s = 0; s < S; s++) {
    const uint64_t d = Dv[(int64_t)s * ld + i];
    if (d == 0) { atomicOr(status, ST_POLE); return; }
    acc = mul_mod(acc, d, M);
    pre[(int64_t)s * T + i] = acc;
  }
  uint64_t inv = inv_mod(acc, M);
  for (int s = S - 1; s >= 0; s--) {
    const uint64_t d = Dv[(int64_t)s * ld + i];
    const uint64_t is = s > 0 ? mul_mod(inv, pre[(int64_t)(s - 1) * T + i], M) : inv;
    inv = mul_mod(inv, d, M);
    out[(int64_t)s * ldo + i] = mul_mod(Nv[(int64_t)s * ld + i], is, M);
  }
}

void launch_ratio(int64_t T, int S, const uint64_t* Nv, const uint64_t* Dv, int64_t ld, const Mod& M, uint64_t* pre,
                  uint64_t* out, int64_t ldo, uint32_t* status, cudaStream_t st) {
  if (T > 0) { k_ratio<<<cdiv(T, 128), 128, 0, st>>>(T, S, Nv, Dv, ld, M, pre, out, ldo, status); note_launch(); }
}

// Multiply n coefficients by c (used for the final normalisation).
__global__ void k_scale(int64_t n, uint64_t* __restrict__ a, const uint64_t* __restrict__ c, Mod M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = mul_mod(a[i], *c, M);
}
__global__ void k_inv1(const uint64_t* __restrict__ a, uint64_t* __restrict__ out, Mod M, uint32_t* status) {
  const uint64_t x = *a;
  if (x == 0) atomicOr(status, ST_ZERO_DEN);
  *out = inv_mod(x, M);
}
void launch_normalise(int64_t n1, uint64_t* a1, int64_t n2, uint64_t* a2, const uint64_t* pivot, uint64_t* tmp,
                      const Mod& M, uint32_t* status, cudaStream_t st) {
  { k_inv1<<<1, 1, 0, st>>>(pivot, tmp, M, status); note_launch(); }
  if (n1 > 0) { k_scale<<<cdiv(n1, 256), 256, 0, st>>>(n1, a1, tmp, M); note_launch(); }
  if (n2 > 0) { k_scale<<<cdiv(n2, 256), 256, 0, st>>>(n2, a2, tmp, M); note_launch(); }
}

// Enqueues the per-probe Thiele + balancing.  Scratch is carved from the
// context workspace by the caller.
size_t thiele_scratch_words(int64_t Tmax, int n) { return (size_t)Tmax * (3 * n + 6 * (n + 1)); }

void launch_thiele_balance(int64_t Tmax, int n, const uint64_t* xs, const uint64_t* fvals, int64_t ldf,
                           const uint64_t* dprev, int dN, int dD, int64_t TN, int64_t TD, uint64_t* scratch,
                           const Mod& M, uint64_t* bN, int64_t ldN, uint64_t* bD, int64_t ldD, uint32_t* status,
                           cudaStream_t st) {
  if (Tmax <= 0) return;
  ThieleScratch sc;
  sc.phi = scratch;
  sc.bl = sc.phi + (size_t)n * Tmax;
  sc.pre = sc.bl + (size_t)n * Tmax;
  sc.P = sc.pre + (size_t)n * Tmax;
  sc.Q = sc.P + (size_t)3 * (n + 1) * Tmax;
  { k_thiele_balance<<<cdiv(Tmax, 128), 128, 0, st>>>(Tmax, n, xs, fvals, ldf, dprev, dN, dD, TN, TD, sc, M, bN, ldN, bD, ldD, status); note_launch(); }
}

}  // namespace zr
