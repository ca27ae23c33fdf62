/*
 * zr_oracle.c -- plain, slow CPU oracle for the Zippel reconstruction step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library.  The CUDA
 * library never links, includes or calls anything here, and nothing here
 * includes anything from the CUDA library: the two share no code.
 *
 * Every function is the plain definition of what the paper's method
 * computes, written in the paper's order:
 *   - modular products are (a*b) mod p through a 128-bit product and the C
 *     remainder operator (Sec. 2.1, variant 1), every sum is reduced at every
 *     step, inverses come from the extended Euclidean algorithm;
 *   - the transposed Vandermonde system of the Zippel step (Sec. 1, the
 *     probe family y^1..y^t) is solved through the master polynomial
 *     M(z) = prod_j (z - v_j), expanded factor by factor, the quotient
 *     q_j = M / (z - v_j) by synthetic division, and
 *     c_j = <q_j, b> / q_j(v_j)  (Sec. 2.2, the Lagrange form: powers, dot
 *     with the value vector, scaled by the inverse of a Horner value);
 *   - Newton interpolation is the divided-difference table of Eq. (newton),
 *     then the nested form expanded to monomial coefficients;
 *   - Thiele interpolation is the inverse-difference continued fraction of
 *     Eq. (thiele), turned into a numerator/denominator pair;
 *   - the balanced step scales per-probe univariate reconstructions by the
 *     known denominator skeleton (Sec. 2.2, the balancing identity).
 *
 * Readings of points the paper leaves open (all documented in the design
 * notes): probe exponents start at 0 (offset 0) or 1 (offset 1, the paper's
 * y^1..y^t); the balancing factor is taken from the denominator skeleton;
 * the final normalisation divides by the coefficient of the lexicographically
 * smallest denominator term; zero coefficients are dropped from skeletons.
 *
 * Random draws of the full reconstructions come from splitmix64 (Steele,
 * Lea, Flood 2014) used as a counter-based generator:
 *   key(seed, stream) = mix(seed + (stream + 1) * G)
 *   draw(key, n)      = mix(key + (n + 1) * G),   G = 0x9E3779B97F4A7C15
 * a residue is draw >> 1, rejected when 0 or >= p.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;
typedef __int128 i128;

enum {
  ZRO_OK = 0,
  ZRO_ERR_INVALID_ARG = 1,
  ZRO_ERR_SINGULAR = 2,
  ZRO_ERR_POLE = 3,
  ZRO_ERR_OOM = 4,
  ZRO_ERR_UNLUCKY = 7,
  ZRO_ERR_CAPACITY = 9,
  ZRO_ERR_DEGREE = 10
};

/* ------------------------------------------------------------------------ */
/* Modular arithmetic: the plain definitions (Sec. 2.1, variant 1).          */
/* ------------------------------------------------------------------------ */

static inline u64 mulm(u64 a, u64 b, u64 p) { return (u64)(((u128)a * b) % p); }
static inline u64 addm(u64 a, u64 b, u64 p) { return (u64)(((u128)a + b) % p); }
static inline u64 subm(u64 a, u64 b, u64 p) { return (u64)(((u128)(a % p) + p - (b % p)) % p); }
static inline u64 negm(u64 a, u64 p) { return subm(0, a, p); }

u64 zro_mulmod(u64 a, u64 b, u64 p) { return mulm(a, b, p); }
u64 zro_addmod(u64 a, u64 b, u64 p) { return addm(a, b, p); }
u64 zro_submod(u64 a, u64 b, u64 p) { return subm(a, b, p); }

/* a^e mod p by square-and-multiply. */
u64 zro_powmod(u64 a, u64 e, u64 p) {
  u64 r = 1 % p, x = a % p;
  while (e) {
    if (e & 1) r = mulm(r, x, p);
    x = mulm(x, x, p);
    e >>= 1;
  }
  return r;
}

/* a^-1 mod p by the extended Euclidean algorithm; 0 when gcd(a, p) != 1. */
u64 zro_invmod(u64 a, u64 p) {
  i128 r0 = (i128)p, r1 = (i128)(a % p), s0 = 0, s1 = 1;
  while (r1 != 0) {
    i128 q = r0 / r1, t;
    t = r0 - q * r1; r0 = r1; r1 = t;
    t = s0 - q * s1; s0 = s1; s1 = t;
  }
  if (r0 != 1) return 0;
  s0 %= (i128)p;
  if (s0 < 0) s0 += p;
  return (u64)s0;
}

/* The modular primitives applied elementwise, for the device-arithmetic
 * parity test (Sec. 2.1: modular products of residues below 2^64; Sec. 2.2:
 * a long dot product reduced once).  Each case is the plain definition in
 * 128-bit integers:
 *   0 mulmod      out = a b mod p
 *   1 reduce      out = (a 2^64 + b) mod p                     (a < p)
 *   2 shoup_pre   out = floor(a 2^64 / p)                      (a < p)
 *   3 shoup_lazy  out = a b - floor(a w' / 2^64) p mod 2^64,
 *                 w' = floor(b 2^64 / p): Shoup's product, congruent to
 *                 a b and below 2p                             (b < p)
 *   4 pow         out = a^b mod p
 *   5 inv         out = a^-1 mod p (extended Euclid), 0 for a = 0
 *   6 dot         out[g] = sum_{t < len} a[g len + t] b[g len + t] mod p,
 *                 reduced at every step
 *   7 add, 8 sub  out = a + b, a - b mod p
 *   9 batch inv   out = a^-1 mod p, 0 for a = 0 (as 5)
 * n outputs; returns 1 for an unknown op. */
int zro_arith_batch(int op, i64 n, i64 len, const u64* a, const u64* b, u64 p, u64* out) {
  for (i64 i = 0; i < n; i++) {
    switch (op) {
      case 0: out[i] = mulm(a[i], b[i], p); break;
      case 1: out[i] = (u64)((((u128)a[i]) << 64 | b[i]) % p); break;
      case 2: out[i] = (u64)((((u128)a[i]) << 64) / p); break;
      case 3: {
        const u64 wq = (u64)((((u128)b[i]) << 64) / p);
        const u64 q = (u64)(((u128)a[i] * wq) >> 64);
        out[i] = a[i] * b[i] - q * p;   /* arithmetic mod 2^64 */
        break;
      }
      case 4: out[i] = zro_powmod(a[i], b[i], p); break;
      case 5: case 9: out[i] = a[i] % p ? zro_invmod(a[i], p) : 0; break;
      case 6: {
        u64 acc = 0;
        for (i64 t = 0; t < len; t++) acc = addm(acc, mulm(a[i * len + t], b[i * len + t], p), p);
        out[i] = acc;
        break;
      }
      case 7: out[i] = addm(a[i], b[i], p); break;
      case 8: out[i] = subm(a[i], b[i], p); break;
      default: return 1;
    }
  }
  return 0;
}

/* Deterministic Miller-Rabin for n < 2^64 (bases 2..37). */
int zro_is_prime(u64 n) {
  static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  u64 d = n - 1; int r = 0;
  while ((d & 1) == 0) { d >>= 1; r++; }
  for (int i = 0; i < 12; i++) {
    u64 x = zro_powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int k = 1; k < r; k++) {
      x = mulm(x, x, n);
      if (x == n - 1) { comp = 0; break; }
    }
    if (comp) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* A tiny parallel-for over independent items (roots, probes).              */
/* ------------------------------------------------------------------------ */

typedef void (*range_fn)(void* ctx, i64 lo, i64 hi);
typedef struct { range_fn fn; void* ctx; i64 lo, hi; } pf_arg;
static void* pf_tramp(void* a) { pf_arg* x = (pf_arg*)a; x->fn(x->ctx, x->lo, x->hi); return NULL; }

int zro_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n < 1 ? 1 : (int)n;
}

static void parallel_for(i64 n, int nthreads, range_fn fn, void* ctx) {
  if (nthreads <= 0) nthreads = zro_default_threads();
  if (nthreads > 256) nthreads = 256;
  if (n < nthreads) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads == 1) { fn(ctx, 0, n); return; }
  pthread_t th[256];
  int ok[256];
  pf_arg args[256];
  for (int t = 0; t < nthreads; t++) {
    args[t].fn = fn; args[t].ctx = ctx;
    args[t].lo = n * t / nthreads; args[t].hi = n * (t + 1) / nthreads;
    ok[t] = pthread_create(&th[t], NULL, pf_tramp, &args[t]) == 0;
    if (!ok[t]) fn(ctx, args[t].lo, args[t].hi);   /* run inline when no thread is available */
  }
  for (int t = 0; t < nthreads; t++) if (ok[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* splitmix64 as a counter-based generator (used by the reconstructions).    */
/* ------------------------------------------------------------------------ */

#define SM_GAMMA 0x9E3779B97F4A7C15ull
static u64 sm_mix(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
u64 zro_splitmix_at(u64 key, u64 n) { return sm_mix(key + (n + 1) * SM_GAMMA); }

typedef struct { u64 key, ctr; } rng_t;
static void rng_init(rng_t* r, u64 seed, u64 stream) { r->key = zro_splitmix_at(seed, stream); r->ctr = 0; }
static u64 rng_residue(rng_t* r, u64 p) {
  for (;;) {
    u64 x = zro_splitmix_at(r->key, r->ctr++) >> 1;
    if (x != 0 && x < p) return x;
  }
}

/* ------------------------------------------------------------------------ */
/* Step a2: anchor values v_j = prod_{m<k} y_m^{e_{j,m}}  (Sec. 1).          */
/* ------------------------------------------------------------------------ */

/* exps is T x nv, term-major; only columns 0..k-1 take part. */
void zro_anchor_values(i64 T, int32_t nv, const uint8_t* exps, int32_t k,
                       const u64* y, u64 p, u64* v) {
  for (i64 j = 0; j < T; j++) {
    u64 acc = 1 % p;
    for (int m = 0; m < k; m++) acc = mulm(acc, zro_powmod(y[m], exps[j * nv + m], p), p);
    v[j] = acc;
  }
}

static int cmp_u64(const void* a, const void* b) {
  u64 x = *(const u64*)a, y = *(const u64*)b;
  return x < y ? -1 : (x > y);
}

/* 0: nodes usable; ZRO_ERR_SINGULAR: two equal nodes, or a zero node when
 * offset = 1 (the system with exponents 1..T then has a zero column). */
int zro_check_nodes(i64 T, const u64* v, int32_t offset) {
  if (T <= 0) return ZRO_OK;
  u64* s = (u64*)malloc(sizeof(u64) * T);
  if (!s) return ZRO_ERR_OOM;
  memcpy(s, v, sizeof(u64) * T);
  qsort(s, T, sizeof(u64), cmp_u64);
  int st = ZRO_OK;
  for (i64 j = 1; j < T; j++) if (s[j] == s[j - 1]) { st = ZRO_ERR_SINGULAR; break; }
  if (offset == 1 && s[0] == 0) st = ZRO_ERR_SINGULAR;
  free(s);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Step a3: master polynomial M(z) = prod_j (z - v_j), factor by factor.     */
/* m has T+1 entries, m[l] = coefficient of z^l, m[T] = 1.                   */
/* ------------------------------------------------------------------------ */

void zro_master_poly(i64 T, const u64* v, u64 p, u64* m) {
  m[0] = 1 % p;
  for (i64 l = 1; l <= T; l++) m[l] = 0;
  for (i64 j = 0; j < T; j++) {
    /* multiply the degree-j polynomial m[0..j] by (z - v_j) */
    m[j + 1] = m[j];
    for (i64 l = j; l >= 1; l--) m[l] = subm(m[l - 1], mulm(v[j], m[l], p), p);
    m[0] = negm(mulm(v[j], m[0], p), p);
  }
}

/* ------------------------------------------------------------------------ */
/* Step a4: synthetic division q = M / (z - vj); q has T entries.            */
/* q_{T-1} = m_T, q_{k-1} = m_k + vj * q_k.                                  */
/* ------------------------------------------------------------------------ */

void zro_synthetic_division(i64 T, const u64* m, u64 vj, u64 p, u64* q) {
  if (T <= 0) return;
  q[T - 1] = m[T];
  for (i64 k = T - 1; k >= 1; k--) q[k - 1] = addm(m[k], mulm(vj, q[k], p), p);
}

/* Horner value of a polynomial of degree < n at x. */
static u64 horner(i64 n, const u64* a, u64 x, u64 p) {
  u64 r = 0;
  for (i64 k = n - 1; k >= 0; k--) r = addm(mulm(r, x, p), a[k], p);
  return r;
}

/* ------------------------------------------------------------------------ */
/* Step a5: transposed Vandermonde solve (Sec. 1 and Sec. 2.2).              */
/*   offset 0: sum_j c_j v_j^k     = b_k,  k = 0..T-1                        */
/*   offset 1: sum_j c_j v_j^(k+1) = b_k,  k = 0..T-1  (the paper's y^1..y^t)*/
/* S right-hand sides share the nodes: b is S x ldb, c is S x ldc.           */
/* ------------------------------------------------------------------------ */

typedef struct {
  i64 T; int32_t S, offset; const u64* v; const u64* b; i64 ldb; u64 p;
  u64* c; i64 ldc; const u64* m; const i64* roots; int bad;
} solve_ctx;

static void solve_range(void* vctx, i64 lo, i64 hi) {
  solve_ctx* x = (solve_ctx*)vctx;
  i64 T = x->T; u64 p = x->p;
  u64* q = (u64*)malloc(sizeof(u64) * (T > 0 ? T : 1));
  if (!q) { x->bad = ZRO_ERR_OOM; return; }
  for (i64 r = lo; r < hi; r++) {
    i64 j = x->roots ? x->roots[r] : r;
    zro_synthetic_division(T, x->m, x->v[j], p, q);
    u64 den = horner(T, q, x->v[j], p);          /* q_j(v_j) = prod_{l!=j}(v_j - v_l) */
    if (x->offset == 1) den = mulm(den, x->v[j], p);
    u64 inv = zro_invmod(den, p);
    if (inv == 0) { x->bad = ZRO_ERR_SINGULAR; continue; }
    for (int s = 0; s < x->S; s++) {
      const u64* bs = x->b + (i64)s * x->ldb;
      u64 acc = 0;
      for (i64 k = 0; k < T; k++) acc = addm(acc, mulm(q[k], bs[k], p), p);
      u64 cj = mulm(acc, inv, p);
      if (x->roots) x->c[(i64)s * x->ldc + r] = cj;
      else x->c[(i64)s * x->ldc + j] = cj;
    }
  }
  free(q);
}

int zro_tvandermonde_solve(i64 T, int32_t S, int32_t offset, const u64* v, const u64* b, i64 ldb,
                           u64 p, u64* c, i64 ldc, int32_t nthreads) {
  if (T < 0 || S < 0 || (offset != 0 && offset != 1) || ldb < T || ldc < T) return ZRO_ERR_INVALID_ARG;
  if (T == 0 || S == 0) return ZRO_OK;
  int st = zro_check_nodes(T, v, offset);
  if (st) return st;
  u64* m = (u64*)malloc(sizeof(u64) * (T + 1));
  if (!m) return ZRO_ERR_OOM;
  zro_master_poly(T, v, p, m);
  solve_ctx x = {T, S, offset, v, b, ldb, p, c, ldc, m, NULL, 0};
  parallel_for(T, nthreads, solve_range, &x);
  free(m);
  return x.bad;
}

/* The same solve for a chosen subset of roots (each c_j depends only on M,
 * v_j and b).  Output column r holds root roots[r]; c is S x ldc with
 * ldc >= nroots.  The master polynomial is passed in (T+1 entries). */
int zro_tvandermonde_solve_roots(i64 T, int32_t S, int32_t offset, const u64* v, const u64* m,
                                 const u64* b, i64 ldb, i64 nroots, const i64* roots,
                                 u64 p, u64* c, i64 ldc, int32_t nthreads) {
  if (T <= 0 || S < 0 || (offset != 0 && offset != 1) || ldb < T || ldc < nroots) return ZRO_ERR_INVALID_ARG;
  for (i64 r = 0; r < nroots; r++) if (roots[r] < 0 || roots[r] >= T) return ZRO_ERR_INVALID_ARG;
  solve_ctx x = {T, S, offset, v, b, ldb, p, c, ldc, m, roots, 0};
  parallel_for(nroots, nthreads, solve_range, &x);
  return x.bad;
}

/* ------------------------------------------------------------------------ */
/* Step a6: Newton interpolation, Eq. (newton).                              */
/* ------------------------------------------------------------------------ */

/* Divided differences a_0..a_{n-1} of (x_s, f_s), then the nested form
 * a_0 + (z-x_0)[a_1 + (z-x_1)[...]] expanded to monomial coefficients
 * coef[0..n-1].  Returns ZRO_ERR_SINGULAR when two nodes coincide. */
int zro_newton(int32_t n, const u64* x, const u64* f, u64 p, u64* coef) {
  if (n <= 0) return ZRO_OK;
  u64* a = (u64*)malloc(sizeof(u64) * n);
  if (!a) return ZRO_ERR_OOM;
  for (int s = 0; s < n; s++) a[s] = f[s] % p;
  for (int l = 1; l < n; l++) {
    for (int s = n - 1; s >= l; s--) {
      u64 inv = zro_invmod(subm(x[s], x[s - l], p), p);
      if (inv == 0) { free(a); return ZRO_ERR_SINGULAR; }
      a[s] = mulm(subm(a[s], a[s - 1], p), inv, p);
    }
  }
  /* nested expansion, innermost bracket first */
  for (int e = 0; e < n; e++) coef[e] = 0;
  coef[0] = a[n - 1];
  int deg = 0;
  for (int l = n - 2; l >= 0; l--) {
    /* coef <- coef * (z - x_l) + a_l */
    coef[deg + 1] = coef[deg];
    for (int e = deg; e >= 1; e--) coef[e] = subm(coef[e - 1], mulm(x[l], coef[e], p), p);
    coef[0] = addm(negm(mulm(x[l], coef[0], p), p), a[l], p);
    deg++;
  }
  free(a);
  return ZRO_OK;
}

/* nterms interpolations over the same npts nodes: vals is npts x ld
 * (row s = the values of all terms at x_s), coef is npts x ld (row e =
 * coefficient of z^e). */
int zro_newton_batched(i64 nterms, int32_t npts, const u64* x, const u64* vals, i64 ld, u64 p, u64* coef) {
  if (nterms < 0 || npts < 0 || ld < nterms) return ZRO_ERR_INVALID_ARG;
  u64* f = (u64*)malloc(sizeof(u64) * (npts + 1));
  u64* g = (u64*)malloc(sizeof(u64) * (npts + 1));
  if (!f || !g) { free(f); free(g); return ZRO_ERR_OOM; }
  int st = ZRO_OK;
  for (i64 j = 0; j < nterms && st == ZRO_OK; j++) {
    for (int s = 0; s < npts; s++) f[s] = vals[(i64)s * ld + j];
    st = zro_newton(npts, x, f, p, g);
    for (int e = 0; e < npts; e++) coef[(i64)e * ld + j] = g[e];
  }
  free(f); free(g);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Sparse black box: a polynomial given as terms (exponent rows, coefs).     */
/* ------------------------------------------------------------------------ */

/* f at npts arbitrary points (pts is npts x nv): the plain definition
 * sum_t coef_t prod_m x_m^{e_{t,m}}. */
void zro_eval_points(i64 Tf, int32_t nv, const uint8_t* exps, const u64* coef,
                     i64 npts, const u64* pts, u64 p, u64* out) {
  for (i64 i = 0; i < npts; i++) {
    u64 acc = 0;
    for (i64 t = 0; t < Tf; t++) {
      u64 term = coef[t] % p;
      for (int m = 0; m < nv; m++) term = mulm(term, zro_powmod(pts[i * nv + m], exps[t * nv + m], p), p);
      acc = addm(acc, term, p);
    }
    out[i] = acc;
  }
}

/* Zippel probe family for new variable k: the points
 *   P_{s,i} = (y_0^{i+off}, .., y_{k-1}^{i+off}, c_s, z_{k+1}, .., z_{nv-1})
 * for s < S, i < T; b is S x ldb.  Terms are grouped by their exponents in
 * x_0..x_{k-1}; within a group they share u = prod_{m<k} y_m^{e_m}, so
 *   f(P_{s,i}) = sum_groups W_g(s) * u_g^{i+off},
 *   W_g(s) = sum_{t in g} coef_t c_s^{e_{t,k}} prod_{m>k} z_m^{e_{t,m}}
 * which is the same sum as the plain definition, regrouped. */
typedef struct { const uint8_t* exps; int32_t nv, k; } grp_cmp_ctx;
static grp_cmp_ctx g_gcc; /* qsort has no context argument; guarded by a mutex */
static pthread_mutex_t g_gcc_mu = PTHREAD_MUTEX_INITIALIZER;
static int cmp_prefix(const void* a, const void* b) {
  i64 s = *(const i64*)a, t = *(const i64*)b;
  int c = memcmp(g_gcc.exps + s * g_gcc.nv, g_gcc.exps + t * g_gcc.nv, (size_t)g_gcc.k);
  if (c) return c;
  return s < t ? -1 : (s > t);
}

typedef struct {
  i64 G; const u64* u; const u64* W; int32_t S; i64 T; int32_t offset; u64 p; u64* b; i64 ldb; int bad;
} probe_ctx;

static void probe_range(void* vctx, i64 lo, i64 hi) {
  probe_ctx* x = (probe_ctx*)vctx;
  u64 p = x->p;
  if (lo >= hi) return;
  u64* pw = (u64*)malloc(sizeof(u64) * (x->G > 0 ? x->G : 1));
  if (!pw) { x->bad = ZRO_ERR_OOM; return; }
  for (i64 g = 0; g < x->G; g++) pw[g] = zro_powmod(x->u[g], (u64)(lo + x->offset), p);
  for (i64 i = lo; i < hi; i++) {
    for (int s = 0; s < x->S; s++) {
      u64 acc = 0;
      for (i64 g = 0; g < x->G; g++) acc = addm(acc, mulm(x->W[g * x->S + s], pw[g], p), p);
      x->b[(i64)s * x->ldb + i] = acc;
    }
    for (i64 g = 0; g < x->G; g++) pw[g] = mulm(pw[g], x->u[g], p);
  }
  free(pw);
}

/* Builds the groups (u_g, W_g(s)); returns the group count or -1.
 * Powers come from per-value tables x^e, e <= 255 (exponents are bytes). */
static u64* pow_table(u64 x, u64 p) {
  u64* t = (u64*)malloc(sizeof(u64) * 256);
  if (!t) return NULL;
  t[0] = 1 % p;
  for (int e = 1; e < 256; e++) t[e] = mulm(t[e - 1], x, p);
  return t;
}

static i64 probe_groups(i64 Tf, int32_t nv, const uint8_t* exps, const u64* coef, int32_t k,
                        const u64* y, int32_t S, const u64* cs, const u64* z, u64 p,
                        u64** u_out, u64** W_out) {
  i64* idx = (i64*)malloc(sizeof(i64) * (Tf > 0 ? Tf : 1));
  u64** ty = (u64**)calloc((size_t)nv + (size_t)S, sizeof(u64*));
  if (!idx || !ty) { free(idx); free(ty); return -1; }
  int okt = 1;
  for (int m = 0; m < nv; m++) if (m != k) { ty[m] = pow_table(m < k ? y[m] : z[m], p); okt &= ty[m] != NULL; }
  for (int s = 0; s < S; s++) { ty[nv + s] = pow_table(cs[s], p); okt &= ty[nv + s] != NULL; }
  for (i64 t = 0; t < Tf; t++) idx[t] = t;
  pthread_mutex_lock(&g_gcc_mu);
  g_gcc.exps = exps; g_gcc.nv = nv; g_gcc.k = k;
  qsort(idx, Tf, sizeof(i64), cmp_prefix);
  pthread_mutex_unlock(&g_gcc_mu);
  i64 G = 0;
  for (i64 r = 0; r < Tf; r++)
    if (r == 0 || memcmp(exps + idx[r] * nv, exps + idx[r - 1] * nv, (size_t)k) != 0) G++;
  u64* u = (u64*)malloc(sizeof(u64) * (G > 0 ? G : 1));
  u64* W = (u64*)calloc((size_t)(G > 0 ? G : 1) * (S > 0 ? S : 1), sizeof(u64));
  if (!u || !W || !okt) {
    free(idx); free(u); free(W);
    for (int m = 0; m < nv + S; m++) free(ty[m]);
    free(ty);
    return -1;
  }
  G = 0;
  for (i64 r = 0; r < Tf; r++) {
    i64 t = idx[r];
    const uint8_t* e = exps + t * nv;
    if (r == 0 || memcmp(e, exps + idx[r - 1] * nv, (size_t)k) != 0) {
      u64 uu = 1 % p;
      for (int m = 0; m < k; m++) uu = mulm(uu, ty[m][e[m]], p);
      u[G++] = uu;
    }
    u64 rest = coef[t] % p;
    for (int m = k + 1; m < nv; m++) rest = mulm(rest, ty[m][e[m]], p);
    for (int s = 0; s < S; s++) {
      u64 w = mulm(rest, ty[nv + s][e[k]], p);
      W[(G - 1) * S + s] = addm(W[(G - 1) * S + s], w, p);
    }
  }
  free(idx);
  for (int m = 0; m < nv + S; m++) free(ty[m]);
  free(ty);
  *u_out = u; *W_out = W;
  return G;
}

int zro_zippel_probes(i64 Tf, int32_t nv, const uint8_t* exps, const u64* coef, int32_t k,
                      const u64* y, int32_t S, const u64* cs, const u64* z, i64 T, int32_t offset,
                      u64 p, int32_t nthreads, u64* b, i64 ldb) {
  if (k < 0 || k >= nv || T < 0 || S < 0 || ldb < T) return ZRO_ERR_INVALID_ARG;
  u64 *u, *W;
  i64 G = probe_groups(Tf, nv, exps, coef, k, y, S, cs, z, p, &u, &W);
  if (G < 0) return ZRO_ERR_OOM;
  probe_ctx x = {G, u, W, S, T, offset, p, b, ldb, 0};
  parallel_for(T, nthreads, probe_range, &x);
  free(u); free(W);
  return x.bad;
}

/* Single probe values b[s][i] for listed (s, i) pairs, each computed on its
 * own: sum_g W_g(s) u_g^{i+off}. */
typedef struct { i64 G; const u64* u; const u64* W; int32_t S; const int32_t* sidx; const i64* iidx;
                 int32_t offset; u64 p; u64* out; } probe1_ctx;
static void probe1_range(void* vctx, i64 lo, i64 hi) {
  probe1_ctx* x = (probe1_ctx*)vctx;
  for (i64 r = lo; r < hi; r++) {
    u64 acc = 0;
    for (i64 g = 0; g < x->G; g++)
      acc = addm(acc, mulm(x->W[g * x->S + x->sidx[r]], zro_powmod(x->u[g], (u64)(x->iidx[r] + x->offset), x->p), x->p), x->p);
    x->out[r] = acc;
  }
}
int zro_zippel_probes_sampled(i64 Tf, int32_t nv, const uint8_t* exps, const u64* coef, int32_t k,
                              const u64* y, int32_t S, const u64* cs, const u64* z, int32_t offset,
                              i64 nsamp, const int32_t* sidx, const i64* iidx, u64 p, int32_t nthreads, u64* out) {
  if (k < 0 || k >= nv || S <= 0) return ZRO_ERR_INVALID_ARG;
  for (i64 r = 0; r < nsamp; r++) if (sidx[r] < 0 || sidx[r] >= S || iidx[r] < 0) return ZRO_ERR_INVALID_ARG;
  u64 *u, *W;
  i64 G = probe_groups(Tf, nv, exps, coef, k, y, S, cs, z, p, &u, &W);
  if (G < 0) return ZRO_ERR_OOM;
  probe1_ctx x = {G, u, W, S, sidx, iidx, offset, p, out};
  parallel_for(nsamp, nthreads, probe1_range, &x);
  free(u); free(W);
  return ZRO_OK;
}

/* ------------------------------------------------------------------------ */
/* The Zippel step (Sec. 1): solve the S systems, then Newton per term.      */
/* ------------------------------------------------------------------------ */

/* Input skeleton: T terms, exps T x nv (columns >= k are ignored on input).
 * Output: the terms (exps_j with column k set to e, g_{j,e}) for every
 * nonzero g_{j,e}, ordered by j then e; at most T*S terms.
 * *nout receives the count; ZRO_ERR_CAPACITY when it exceeds cap. */
int zro_zippel_step(i64 T, int32_t nv, const uint8_t* exps, int32_t k, const u64* y,
                    int32_t S, const u64* cs, const u64* b, i64 ldb, int32_t offset, u64 p,
                    int32_t nthreads, i64 cap, i64* nout, uint8_t* out_exps, u64* out_coef,
                    u64* c_out /* optional S x T */) {
  if (T < 0 || S <= 0 || k < 0 || k >= nv || ldb < T || S > 255 + 1) return ZRO_ERR_INVALID_ARG;
  u64* v = (u64*)malloc(sizeof(u64) * (T > 0 ? T : 1));
  u64* c = (u64*)malloc(sizeof(u64) * (T > 0 ? T : 1) * S);
  u64* g = (u64*)malloc(sizeof(u64) * (T > 0 ? T : 1) * S);
  if (!v || !c || !g) { free(v); free(c); free(g); return ZRO_ERR_OOM; }
  zro_anchor_values(T, nv, exps, k, y, p, v);
  int st = zro_tvandermonde_solve(T, S, offset, v, b, ldb, p, c, T, nthreads);
  if (st == ZRO_OK) st = zro_newton_batched(T, S, cs, c, T, p, g);
  if (st == ZRO_OK) {
    i64 n = 0;
    for (i64 j = 0; j < T; j++)
      for (int e = 0; e < S; e++) {
        u64 ge = g[(i64)e * T + j];
        if (ge == 0) continue;
        if (n < cap) {
          for (int m = 0; m < nv; m++) out_exps[n * nv + m] = (m < k) ? exps[j * nv + m] : 0;
          out_exps[n * nv + k] = (uint8_t)e;
          out_coef[n] = ge;
        }
        n++;
      }
    *nout = n;
    if (n > cap) st = ZRO_ERR_CAPACITY;
    if (c_out) memcpy(c_out, c, sizeof(u64) * T * S);
  }
  free(v); free(c); free(g);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Thiele interpolation, Eq. (thiele).                                       */
/* ------------------------------------------------------------------------ */

/* From n points (x_s, f_s): inverse differences
 *   phi_0(x_i) = f_i,  phi_l(x_i) = (x_i - x_{l-1}) / (phi_{l-1}(x_i) - b_{l-1}),
 *   b_l = phi_l(x_l),
 * stopped at the first level L whose tail is constant on all later points
 * (phi_L(x_i) = b_L for every i > L; at least one such point is required).
 * The convergent P_L/Q_L of b_0 + (x-x_0)/(b_1 + (x-x_1)/(b_2 + ...)),
 *   P_l = b_l P_{l-1} + (x - x_{l-1}) P_{l-2},  P_{-1} = 1, P_0 = b_0,
 *   Q_l = b_l Q_{l-1} + (x - x_{l-1}) Q_{l-2},  Q_{-1} = 0, Q_0 = 1,
 * is returned as num/den (n entries each, zero padded) scaled so that
 * den(x_0) = 1.  *dn, *dd receive the degrees.
 * Errors: ZRO_ERR_DEGREE when the fraction does not close within the points
 * or exceeds the bounds; ZRO_ERR_UNLUCKY on a degenerate table; ZRO_ERR_POLE
 * when den(x_0) = 0. */
int zro_thiele(int32_t n, const u64* x, const u64* f, u64 p, int32_t maxdn, int32_t maxdd,
               int32_t* dn, int32_t* dd, u64* num, u64* den) {
  if (n <= 0) return ZRO_ERR_INVALID_ARG;
  u64* phi = (u64*)malloc(sizeof(u64) * n);
  u64* bl = (u64*)malloc(sizeof(u64) * n);
  u64* P = (u64*)calloc((size_t)3 * (n + 1), sizeof(u64));
  u64* Q = (u64*)calloc((size_t)3 * (n + 1), sizeof(u64));
  if (!phi || !bl || !P || !Q) { free(phi); free(bl); free(P); free(Q); return ZRO_ERR_OOM; }
  int st = ZRO_OK, L = -1;
  for (int i = 0; i < n; i++) phi[i] = f[i] % p;
  bl[0] = phi[0];
  for (int l = 1; l < n; l++) {
    int all_eq = 1, any_eq = 0;
    for (int i = l; i < n; i++) { if (phi[i] == bl[l - 1]) any_eq = 1; else all_eq = 0; }
    if (all_eq) { L = l - 1; break; }
    if (any_eq) { st = ZRO_ERR_UNLUCKY; break; }
    for (int i = l; i < n; i++)
      phi[i] = mulm(subm(x[i], x[l - 1], p), zro_invmod(subm(phi[i], bl[l - 1], p), p), p);
    bl[l] = phi[l];
  }
  if (st == ZRO_OK && L < 0) st = ZRO_ERR_DEGREE;
  if (st == ZRO_OK) {
    /* rows: 0 = level l-2, 1 = level l-1, 2 = level l; each n+1 coefficients */
    int W = n + 1;
    u64 *Pm2 = P, *Pm1 = P + W, *Pc = P + 2 * W, *Qm2 = Q, *Qm1 = Q + W, *Qc = Q + 2 * W;
    Pm2[0] = 1; Qm2[0] = 0;            /* level -1 */
    Pm1[0] = bl[0]; Qm1[0] = 1;        /* level 0 */
    for (int l = 1; l <= L; l++) {
      for (int e = 0; e < W; e++) {
        /* (x - x_{l-1}) * R  contributes R[e-1] - x_{l-1} R[e] to degree e */
        u64 sp = subm(e ? Pm2[e - 1] : 0, mulm(x[l - 1], Pm2[e], p), p);
        u64 sq = subm(e ? Qm2[e - 1] : 0, mulm(x[l - 1], Qm2[e], p), p);
        Pc[e] = addm(mulm(bl[l], Pm1[e], p), sp, p);
        Qc[e] = addm(mulm(bl[l], Qm1[e], p), sq, p);
      }
      u64 *t;
      t = Pm2; Pm2 = Pm1; Pm1 = Pc; Pc = t;
      t = Qm2; Qm2 = Qm1; Qm1 = Qc; Qc = t;
    }
    /* level L now sits in Pm1 / Qm1 */
    u64 q0 = horner(W, Qm1, x[0], p);
    u64 s = zro_invmod(q0, p);
    if (s == 0) st = ZRO_ERR_POLE;
    else {
      int degp = -1, degq = -1;
      for (int e = 0; e < W; e++) {
        u64 a = mulm(Pm1[e], s, p), c = mulm(Qm1[e], s, p);
        if (e < n) { num[e] = a; den[e] = c; }
        if (a) degp = e;
        if (c) degq = e;
      }
      *dn = degp; *dd = degq;
      if (degp >= n || degq >= n || degp > maxdn || degq > maxdd) st = ZRO_ERR_DEGREE;
    }
  }
  free(phi); free(bl); free(P); free(Q);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Full reconstructions (Sec. 1): variable by variable.                      */
/* ------------------------------------------------------------------------ */

/* A polynomial in nv variables: T terms, exps T x nv, coef T. */
typedef struct { i64 T; uint8_t* exps; u64* coef; } poly_t;
static void poly_free(poly_t* a) { free(a->exps); free(a->coef); a->exps = NULL; a->coef = NULL; a->T = 0; }

/* Stream numbers of the draws (documented for both implementations). */
#define ZR_STREAM_REST 1ull
#define ZR_STREAM_STEP(k, attempt) (1024ull + 64ull * (u64)(k) + (u64)(attempt))
#define ZR_MAX_ATTEMPTS 64

/* draws the rest values z_0..z_{nv-1} */
static void draw_rest(u64 seed, int nv, u64 p, u64* z) {
  rng_t r; rng_init(&r, seed, ZR_STREAM_REST);
  for (int m = 0; m < nv; m++) z[m] = rng_residue(&r, p);
}

/* Draws, for step k and the given attempt, the anchor y_0..y_{k-1} and the
 * samples: c_0 = c0 when have_c0 (the value x_k held in the previous step),
 * then fresh values distinct from all earlier samples. */
static void draw_step(u64 seed, int k, int attempt, int have_c0, u64 c0, int S, u64 p, u64* y, u64* cs) {
  rng_t r; rng_init(&r, seed, ZR_STREAM_STEP(k, attempt));
  for (int m = 0; m < k; m++) y[m] = rng_residue(&r, p);
  int s0 = 0;
  if (have_c0) { cs[0] = c0; s0 = 1; }
  for (int s = s0; s < S; s++) {
    for (;;) {
      u64 c = rng_residue(&r, p);
      int dup = 0;
      for (int t = 0; t < s; t++) if (cs[t] == c) { dup = 1; break; }
      if (!dup) { cs[s] = c; break; }
    }
  }
}

/* Polynomial reconstruction of a sparse black box with nv variables and
 * per-variable degree bounds deg[m] (S_m = deg[m] + 1 samples).
 * Step 0: dense Newton in x_0 with x_1.. fixed at z.  Steps k >= 1: the
 * Zippel step with the probes f(y^{i+off}, c_s, z_{k+1..}).
 * Output terms in the order the steps emit them. */
int zro_reconstruct_poly(i64 Tf, int32_t nv, const uint8_t* fexps, const u64* fcoef,
                         const int32_t* deg, u64 seed, int32_t offset, u64 p, int32_t nthreads,
                         i64 cap, i64* nout, uint8_t* out_exps, u64* out_coef, i64* work_out) {
  if (nv <= 0 || nv > 64 || (offset != 0 && offset != 1)) return ZRO_ERR_INVALID_ARG;
  for (int m = 0; m < nv; m++) if (deg[m] < 0 || deg[m] > 254) return ZRO_ERR_INVALID_ARG;
  u64 z[64], y[64];
  draw_rest(seed, nv, p, z);
  int st = ZRO_OK;
  poly_t sk = {0, NULL, NULL};
  i64 work = 0;
  /* step 0 */
  {
    int S = deg[0] + 1;
    u64* cs = (u64*)malloc(sizeof(u64) * S);
    u64* pts = (u64*)malloc(sizeof(u64) * S * nv);
    u64* vals = (u64*)malloc(sizeof(u64) * S);
    u64* g = (u64*)malloc(sizeof(u64) * S);
    draw_step(seed, 0, 0, 0, 0, S, p, y, cs);
    for (int s = 0; s < S; s++) for (int m = 0; m < nv; m++) pts[s * nv + m] = (m == 0) ? cs[s] : z[m];
    zro_eval_points(Tf, nv, fexps, fcoef, S, pts, p, vals);
    st = zro_newton(S, cs, vals, p, g);
    i64 n = 0;
    for (int e = 0; e < S; e++) if (g[e]) n++;
    sk.T = n;
    sk.exps = (uint8_t*)calloc((size_t)(n ? n : 1) * nv, 1);
    sk.coef = (u64*)malloc(sizeof(u64) * (n ? n : 1));
    n = 0;
    for (int e = 0; e < S; e++) if (g[e]) { sk.exps[n * nv + 0] = (uint8_t)e; sk.coef[n] = g[e]; n++; }
    free(cs); free(pts); free(vals); free(g);
  }
  for (int k = 1; k < nv && st == ZRO_OK; k++) {
    int S = deg[k] + 1;
    i64 T = sk.T;
    u64* cs = (u64*)malloc(sizeof(u64) * S);
    u64* b = (u64*)malloc(sizeof(u64) * (T ? T : 1) * S);
    i64 cap2 = (T ? T : 1) * S;
    poly_t nk = {0, (uint8_t*)malloc((size_t)cap2 * nv), (u64*)malloc(sizeof(u64) * cap2)};
    int attempt = 0;
    for (;;) {
      draw_step(seed, k, attempt, 1, z[k], S, p, y, cs);
      st = zro_zippel_probes(Tf, nv, fexps, fcoef, k, y, S, cs, z, T, offset, p, nthreads, b, T);
      if (st == ZRO_OK)
        st = zro_zippel_step(T, nv, sk.exps, k, y, S, cs, b, T, offset, p, nthreads, cap2, &nk.T, nk.exps, nk.coef, NULL);
      work += (i64)(S + 2) * T * T;
      if (st == ZRO_ERR_SINGULAR && ++attempt < ZR_MAX_ATTEMPTS) continue;
      break;
    }
    free(cs); free(b);
    poly_free(&sk);
    sk = nk;
  }
  if (st == ZRO_OK) {
    *nout = sk.T;
    if (sk.T > cap) st = ZRO_ERR_CAPACITY;
    else {
      memcpy(out_exps, sk.exps, (size_t)sk.T * nv);
      memcpy(out_coef, sk.coef, sizeof(u64) * sk.T);
    }
  }
  if (work_out) *work_out = work;
  poly_free(&sk);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Balanced Zippel for rational functions (Sec. 1, Sec. 2.2).                */
/* ------------------------------------------------------------------------ */

/* N/D at npts points; ZRO_ERR_POLE when D vanishes at one of them. */
static int eval_ratio(const poly_t* N, const poly_t* D, int nv, i64 npts, const u64* pts, u64 p, u64* out) {
  u64* nvls = (u64*)malloc(sizeof(u64) * (npts ? npts : 1));
  u64* dvls = (u64*)malloc(sizeof(u64) * (npts ? npts : 1));
  zro_eval_points(N->T, nv, N->exps, N->coef, npts, pts, p, nvls);
  zro_eval_points(D->T, nv, D->exps, D->coef, npts, pts, p, dvls);
  int st = ZRO_OK;
  for (i64 i = 0; i < npts; i++) {
    u64 inv = zro_invmod(dvls[i], p);
    if (inv == 0) { st = ZRO_ERR_POLE; break; }
    out[i] = mulm(nvls[i], inv, p);
  }
  free(nvls); free(dvls);
  return st;
}

/* Per-probe univariate reconstruction and balancing for step k.
 * fvals is Sf x ldf: f at (y^{i+off}, c_s, z) for s < Sf, i < Tmax.
 * For each probe i: Thiele over (c_s, fvals[s][i]) -> n_i/d_i with
 * d_i(c_0) = 1; the factor is dprev[i] = D'(y^{i+off}) (the previous
 * denominator skeleton at the probe); then
 *   bN[s][i] = dprev[i] * n_i(c_s)  (s < SN, i < TN)
 *   bD[s][i] = dprev[i] * d_i(c_s)  (s < SD, i < TD).
 * This is the balancing identity of Sec. 2.2 with the ratio taken from the
 * denominator: both equal C * N(y^i, c_s) and C * D(y^i, c_s). */
typedef struct {
  int32_t Sf; const u64* cs; const u64* fvals; i64 ldf; const u64* dprev;
  int32_t SN, SD; i64 TN, TD; int32_t dN, dD; u64 p; u64* bN; i64 ldN; u64* bD; i64 ldD; int bad;
} bal_ctx;
static void bal_range(void* vctx, i64 lo, i64 hi) {
  bal_ctx* x = (bal_ctx*)vctx;
  u64 p = x->p;
  int n = x->Sf;
  u64* f = (u64*)malloc(sizeof(u64) * n);
  u64* num = (u64*)malloc(sizeof(u64) * n);
  u64* den = (u64*)malloc(sizeof(u64) * n);
  for (i64 i = lo; i < hi; i++) {
    for (int s = 0; s < n; s++) f[s] = x->fvals[(i64)s * x->ldf + i];
    int dn, dd;
    int st = zro_thiele(n, x->cs, f, p, x->dN, x->dD, &dn, &dd, num, den);
    if (st) { x->bad = st; continue; }
    u64 fac = x->dprev[i];
    if (i < x->TN)
      for (int s = 0; s < x->SN; s++) x->bN[(i64)s * x->ldN + i] = mulm(fac, horner(n, num, x->cs[s], p), p);
    if (i < x->TD)
      for (int s = 0; s < x->SD; s++) x->bD[(i64)s * x->ldD + i] = mulm(fac, horner(n, den, x->cs[s], p), p);
  }
  free(f); free(num); free(den);
}

int zro_balance_probes(int32_t Sf, const u64* cs, const u64* fvals, i64 ldf, i64 Tmax, const u64* dprev,
                       int32_t dN, int32_t dD, i64 TN, i64 TD, u64 p, int32_t nthreads,
                       u64* bN, i64 ldN, u64* bD, i64 ldD) {
  if (Sf <= 0 || TN > Tmax || TD > Tmax || ldf < Tmax) return ZRO_ERR_INVALID_ARG;
  bal_ctx x = {Sf, cs, fvals, ldf, dprev, dN + 1, dD + 1, TN, TD, dN, dD, p, bN, ldN, bD, ldD, 0};
  parallel_for(Tmax, nthreads, bal_range, &x);
  return x.bad;
}

/* Skeleton polynomial D' evaluated at the probes y^{i+off}: sum_j d_j v_j^{i+off}. */
static void skeleton_at_probes(const poly_t* D, int nv, int k, const u64* y, i64 Tmax, int offset, u64 p, u64* out) {
  u64* v = (u64*)malloc(sizeof(u64) * (D->T ? D->T : 1));
  u64* pw = (u64*)malloc(sizeof(u64) * (D->T ? D->T : 1));
  zro_anchor_values(D->T, nv, D->exps, k, y, p, v);
  for (i64 j = 0; j < D->T; j++) pw[j] = zro_powmod(v[j], (u64)offset, p);
  for (i64 i = 0; i < Tmax; i++) {
    u64 acc = 0;
    for (i64 j = 0; j < D->T; j++) { acc = addm(acc, mulm(D->coef[j], pw[j], p), p); pw[j] = mulm(pw[j], v[j], p); }
    out[i] = acc;
  }
  free(v); free(pw);
}

static int lex_less(const uint8_t* a, const uint8_t* b, int nv) { return memcmp(a, b, (size_t)nv) < 0; }

/* Balanced reconstruction of N/D.  degN[m], degD[m] bound the degrees in
 * x_m; Sf_m = 2 max(degN[m], degD[m]) + 2 Thiele points per probe.  The
 * result is normalised so that the lexicographically smallest exponent
 * vector of D has coefficient 1. */
int zro_reconstruct_rational(i64 TNf, const uint8_t* Nexps, const u64* Ncoef,
                             i64 TDf, const uint8_t* Dexps, const u64* Dcoef, int32_t nv,
                             const int32_t* degN, const int32_t* degD, u64 seed, int32_t offset, u64 p,
                             int32_t nthreads, i64 capN, i64 capD, i64* noutN, uint8_t* outNexps, u64* outNcoef,
                             i64* noutD, uint8_t* outDexps, u64* outDcoef) {
  if (nv <= 0 || nv > 64 || (offset != 0 && offset != 1)) return ZRO_ERR_INVALID_ARG;
  for (int m = 0; m < nv; m++) if (degN[m] < 0 || degD[m] < 0 || degN[m] > 120 || degD[m] > 120) return ZRO_ERR_INVALID_ARG;
  poly_t Nf = {TNf, (uint8_t*)Nexps, (u64*)Ncoef}, Df = {TDf, (uint8_t*)Dexps, (u64*)Dcoef};
  u64 z[64], y[64];
  draw_rest(seed, nv, p, z);
  int st = ZRO_OK;
  poly_t skN = {0, NULL, NULL}, skD = {0, NULL, NULL};
  /* step 0: Thiele in x_0 with x_1.. fixed at z */
  {
    int dmax = degN[0] > degD[0] ? degN[0] : degD[0];
    int Sf = 2 * dmax + 2;
    u64* cs = (u64*)malloc(sizeof(u64) * Sf);
    u64* pts = (u64*)malloc(sizeof(u64) * Sf * nv);
    u64* f = (u64*)malloc(sizeof(u64) * Sf);
    u64* num = (u64*)malloc(sizeof(u64) * Sf);
    u64* den = (u64*)malloc(sizeof(u64) * Sf);
    int attempt = 0, dn = 0, dd = 0;
    for (;;) {
      draw_step(seed, 0, attempt, 0, 0, Sf, p, y, cs);
      for (int s = 0; s < Sf; s++) for (int m = 0; m < nv; m++) pts[s * nv + m] = (m == 0) ? cs[s] : z[m];
      st = eval_ratio(&Nf, &Df, nv, Sf, pts, p, f);
      if (st == ZRO_OK) st = zro_thiele(Sf, cs, f, p, degN[0], degD[0], &dn, &dd, num, den);
      if ((st == ZRO_ERR_POLE || st == ZRO_ERR_UNLUCKY) && ++attempt < ZR_MAX_ATTEMPTS) continue;
      break;
    }
    if (st == ZRO_OK) {
      i64 nn = 0, nd = 0;
      for (int e = 0; e <= dn; e++) if (num[e]) nn++;
      for (int e = 0; e <= dd; e++) if (den[e]) nd++;
      skN.T = nn; skN.exps = (uint8_t*)calloc((size_t)(nn ? nn : 1) * nv, 1); skN.coef = (u64*)malloc(sizeof(u64) * (nn ? nn : 1));
      skD.T = nd; skD.exps = (uint8_t*)calloc((size_t)(nd ? nd : 1) * nv, 1); skD.coef = (u64*)malloc(sizeof(u64) * (nd ? nd : 1));
      nn = nd = 0;
      for (int e = 0; e <= dn; e++) if (num[e]) { skN.exps[nn * nv] = (uint8_t)e; skN.coef[nn++] = num[e]; }
      for (int e = 0; e <= dd; e++) if (den[e]) { skD.exps[nd * nv] = (uint8_t)e; skD.coef[nd++] = den[e]; }
    }
    free(cs); free(pts); free(f); free(num); free(den);
  }
  for (int k = 1; k < nv && st == ZRO_OK; k++) {
    int dmax = degN[k] > degD[k] ? degN[k] : degD[k];
    int Sf = 2 * dmax + 2, SN = degN[k] + 1, SD = degD[k] + 1;
    i64 TN = skN.T, TD = skD.T, Tmax = TN > TD ? TN : TD;
    u64* cs = (u64*)malloc(sizeof(u64) * Sf);
    u64* fv = (u64*)malloc(sizeof(u64) * Sf * (Tmax ? Tmax : 1));
    u64* dvv = (u64*)malloc(sizeof(u64) * Sf * (Tmax ? Tmax : 1));
    u64* dprev = (u64*)malloc(sizeof(u64) * (Tmax ? Tmax : 1));
    u64* bN = (u64*)malloc(sizeof(u64) * SN * (TN ? TN : 1));
    u64* bD = (u64*)malloc(sizeof(u64) * SD * (TD ? TD : 1));
    i64 capn = (TN ? TN : 1) * SN, capd = (TD ? TD : 1) * SD;
    poly_t nN = {0, (uint8_t*)malloc((size_t)capn * nv), (u64*)malloc(sizeof(u64) * capn)};
    poly_t nD = {0, (uint8_t*)malloc((size_t)capd * nv), (u64*)malloc(sizeof(u64) * capd)};
    int attempt = 0;
    for (;;) {
      draw_step(seed, k, attempt, 1, z[k], Sf, p, y, cs);
      /* f = N/D at (y^{i+off}, c_s, z_{k+1..}): N and D through the probe family */
      st = zro_zippel_probes(Nf.T, nv, Nf.exps, Nf.coef, k, y, Sf, cs, z, Tmax, offset, p, nthreads, fv, Tmax);
      if (st == ZRO_OK)
        st = zro_zippel_probes(Df.T, nv, Df.exps, Df.coef, k, y, Sf, cs, z, Tmax, offset, p, nthreads, dvv, Tmax);
      for (i64 r = 0; r < (i64)Sf * Tmax && st == ZRO_OK; r++) {
        u64 inv = zro_invmod(dvv[r], p);
        if (inv == 0) st = ZRO_ERR_POLE;
        else fv[r] = mulm(fv[r], inv, p);
      }
      if (st == ZRO_OK) {
        skeleton_at_probes(&skD, nv, k, y, Tmax, offset, p, dprev);
        st = zro_balance_probes(Sf, cs, fv, Tmax, Tmax, dprev, degN[k], degD[k], TN, TD, p, nthreads, bN, TN, bD, TD);
      }
      if (st == ZRO_OK)
        st = zro_zippel_step(TN, nv, skN.exps, k, y, SN, cs, bN, TN, offset, p, nthreads, capn, &nN.T, nN.exps, nN.coef, NULL);
      if (st == ZRO_OK)
        st = zro_zippel_step(TD, nv, skD.exps, k, y, SD, cs, bD, TD, offset, p, nthreads, capd, &nD.T, nD.exps, nD.coef, NULL);
      if ((st == ZRO_ERR_SINGULAR || st == ZRO_ERR_POLE || st == ZRO_ERR_UNLUCKY) && ++attempt < ZR_MAX_ATTEMPTS) continue;
      break;
    }
    free(cs); free(fv); free(dvv); free(dprev); free(bN); free(bD);
    poly_free(&skN); poly_free(&skD);
    skN = nN; skD = nD;
  }
  if (st == ZRO_OK) {
    /* normalise on the lexicographically smallest denominator term */
    i64 best = -1;
    for (i64 j = 0; j < skD.T; j++) if (best < 0 || lex_less(skD.exps + j * nv, skD.exps + best * nv, nv)) best = j;
    if (best < 0) st = ZRO_ERR_SINGULAR;
    else {
      u64 s = zro_invmod(skD.coef[best], p);
      for (i64 j = 0; j < skN.T; j++) skN.coef[j] = mulm(skN.coef[j], s, p);
      for (i64 j = 0; j < skD.T; j++) skD.coef[j] = mulm(skD.coef[j], s, p);
      *noutN = skN.T; *noutD = skD.T;
      if (skN.T > capN || skD.T > capD) st = ZRO_ERR_CAPACITY;
      else {
        memcpy(outNexps, skN.exps, (size_t)skN.T * nv); memcpy(outNcoef, skN.coef, sizeof(u64) * skN.T);
        memcpy(outDexps, skD.exps, (size_t)skD.T * nv); memcpy(outDcoef, skD.coef, sizeof(u64) * skD.T);
      }
    }
  }
  poly_free(&skN); poly_free(&skD);
  return st;
}
