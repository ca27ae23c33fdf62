/*
 * zr.h -- C ABI of the GB300 Zippel-step library (libzr.so).
 *
 * The library implements the per-variable step of Zippel's sparse
 * reconstruction as described in arXiv 2505.24256 (Smirnov, Rozhnov,
 * Voevodin, "GPU Implementation of Zippel Method for Feynman Integral
 * Reconstruction"):
 *   Sec. 1       the step k-1 -> k: a skeleton of T monomials, probes at the
 *                powers y^i of an anchor (a transposed Vandermonde system per
 *                sample c_s of the new variable), then univariate Newton
 *                interpolation (Eq. newton) per skeleton term;
 *   Sec. 2.1     64-bit modular arithmetic on the GPU;
 *   Sec. 2.2     the solve as Horner values, power vectors dotted with the
 *                probe values and scaled by an inverse, deferred modular
 *                summation, and the balanced variant for rational functions.
 *
 * Conventions shared by every call:
 *   - Every call returns a zr_status; nothing throws or aborts across the ABI.
 *     zr_last_error(ctx) describes the last failure of that context.
 *   - All residues are canonical: 0 <= x < p.
 *   - Pointers documented "device" must be CUDA device pointers of the current
 *     device, owned by the caller and left untouched by the library after the
 *     call's stream work completes.  Library workspace is owned by the context
 *     and reused between calls (it only grows).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls ending in _async only enqueue work; the others wait for their
 *     stream before returning so that device-detected conditions (equal
 *     anchor values, a vanished denominator, a pole) become the return status.
 *   - A context is not thread-safe, except the zr_serve_* submit/poll calls.
 *   - Matrices are row-major with an explicit leading dimension (elements).
 */
#ifndef ZR_H
#define ZR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum zr_status {
  ZR_OK = 0,
  ZR_ERR_INVALID_ARG = 1, /* a size, pointer, modulus or layout is out of range */
  ZR_ERR_SINGULAR = 2,    /* equal anchor values, a zero anchor value with offset 1,
                             or equal samples of the new variable */
  ZR_ERR_POLE = 3,        /* the rational black box has a pole at a probe */
  ZR_ERR_OOM = 4,         /* device or host allocation failed / over budget */
  ZR_ERR_TIMEOUT = 5,     /* a bounded wait gave up */
  ZR_ERR_CUDA = 6,        /* a CUDA runtime call failed (see zr_last_error) */
  ZR_ERR_UNLUCKY = 7,     /* a random choice failed (degenerate table): redraw */
  ZR_ERR_BUSY = 8,        /* the server cannot take the request now */
  ZR_ERR_CAPACITY = 9,    /* an output buffer is too small; the needed size is returned */
  ZR_ERR_DEGREE = 10      /* a reconstruction exceeded its degree bound */
} zr_status;

typedef struct zr_ctx zr_ctx;

/* Creates a context for the prime p, 2^32 < p < 2^63 (checked with a
 * deterministic Miller-Rabin test; Sec. 2.1 works with primes below 2^64, the
 * bound 2^63 keeps sums of two residues below 2^64).  Binds the current CUDA
 * device.  *out receives the context or NULL on error. */
zr_status zr_create(uint64_t prime, zr_ctx** out);
void zr_destroy(zr_ctx* ctx);
const char* zr_last_error(const zr_ctx* ctx);
const char* zr_status_string(zr_status s);
uint64_t zr_prime(const zr_ctx* ctx);
/* Bytes of device workspace the context currently holds. */
size_t zr_workspace_bytes(const zr_ctx* ctx);

/* Diagnostics.  zr_launch_count: kernels launched by the library in this
 * process so far.  The profiler records CUDA events around the phases of
 * every step enqueued by the context (0 anchor values + node check, 1 master
 * polynomial, 2 right-hand sides in MAC form, 3 k-block carries, 4 the
 * synthetic-division/dot kernel, 5 denominators + inverses + Newton,
 * 6 compaction, 7 probe evaluation, 8 the O(T log^2 T) solve of the systems
 * that take it: tree, power sums, descent and leaves; 9 each launch of that
 * solve's transform tile kernel, 10 each launch of its descent's cluster
 * level kernel and 11 each launch of its direct power sums kernel, all inside
 * phase 8); zr_profile_enable resets the totals, zr_profile_query waits for
 * the recorded events and returns the summed milliseconds and the number of
 * timed occurrences of a phase, and zr_profile_work the algorithmic work
 * recorded with them (phases 9 and 10: radix-2 butterflies, n/2 per stage of
 * each transform of n words; 11: the T^2 Shoup steps v_j^k -> v_j^(k+1); 0
 * for the others).  While the profiler is on, the O(T log^2 T) solve runs
 * everything on the call's stream (no auxiliary branch beside it), so that
 * each timed launch has the GPU to itself.  Errors: ZR_ERR_INVALID_ARG for a
 * phase outside 0..11 or a null pointer. */
uint64_t zr_launch_count(void);
zr_status zr_profile_enable(zr_ctx* ctx, int32_t on);
zr_status zr_profile_query(zr_ctx* ctx, int32_t phase, double* total_ms, int64_t* count);
zr_status zr_profile_work(zr_ctx* ctx, int32_t phase, double* units);

/* Self-check of the bounded device waits (the paper has no counterpart):
 * one warp waits on a shared-memory barrier that nothing arrives on, gives
 * up after `tries` tries and reports it, exactly as the solve's pipeline
 * does after its own limit.  Returns ZR_ERR_TIMEOUT when the mechanism works
 * (the context stays usable); synchronous. */
zr_status zr_check_bounded_wait(zr_ctx* ctx, uint32_t tries, void* stream);

/* Self-check of the device modular arithmetic (Sec. 2.1: the 64-bit modular
 * product through a precomputed reciprocal; Sec. 2.2: a long dot product
 * accumulated without reduction and reduced once).  Applies one primitive of
 * the step kernels elementwise, i = 0..n-1, with the context's prime p:
 *   0 mulmod      out = a b mod p                                (a, b < p)
 *   1 reduce      out = (a 2^64 + b) mod p                       (a < p)
 *   2 shoup_pre   out = floor(a 2^64 / p)                        (a < p)
 *   3 shoup_lazy  out = Shoup's product of a (any 64-bit value) and b < p:
 *                 a b - floor(a floor(b 2^64 / p) / 2^64) p mod 2^64, in [0, 2p)
 *   4 pow         out = a^b mod p
 *   5 inv         out = a^(p-2) mod p (0 for a = 0)
 *   6 dot         out[i] = sum_{t < len} a[i len + t] b[i len + t] mod p
 *                 (1 <= len < 2^31; one 160-bit accumulator per i)
 *   7 add, 8 sub  out = a +- b mod p                             (a, b < p)
 *   9 batch_inv   out = a^-1 mod p (0 for a = 0) by Montgomery's batch trick
 *                 over consecutive groups of 32
 * a, b, out: device arrays (b unused by 2, 5, 9); for dot, a and b hold
 * n len values.  hits: NULL, or a device uint32[4] to which the call adds how
 * often the two correction steps of the Moller-Granlund division ran
 * (hits[0], hits[1]: in the reductions of ops 0, 1, 6; hits[2], hits[3]: in
 * op 2).  Synchronous; ZR_ERR_INVALID_ARG for an unknown op or bad sizes.
 * The paper has no counterpart: this is test instrumentation. */
zr_status zr_check_arith(zr_ctx* ctx, int32_t op, int64_t n, int64_t len, const uint64_t* a, const uint64_t* b,
                         uint64_t* out, uint32_t* hits, void* stream);

/* Measured ceilings (the paper has no counterpart: these are the rates the
 * solve's throughput is reported against).  Each probe runs one instruction
 * sequence of the solve with all operands in registers, independent
 * accumulators per thread and every SM filled, times one launch of about
 * 30 ms with CUDA events on `stream`, and returns operations per second:
 *   mac_per_s      64x64-bit products added into a 160-bit accumulator
 *                  (the dot product's multiply-accumulate, Sec. 2.2)
 *   chain_per_s    synthetic-division steps q <- q v + m with Shoup's
 *                  precomputed quotient (Sec. 2.1)
 *   imad_lo_per_s, imad_hi_per_s   32-bit mad.lo / mad.hi
 *   butterfly_per_s   forward transform butterflies on 32-bit residues
 *                  with a Shoup twiddle (the O(T log^2 T) solve's transforms)
 * Synchronous; uses the context workspace. */
typedef struct zr_peaks {
  double mac_per_s, chain_per_s, imad_lo_per_s, imad_hi_per_s, butterfly_per_s;
  int32_t sms, pad;
} zr_peaks;
zr_status zr_measure_peaks(zr_ctx* ctx, zr_peaks* out, void* stream);

/* Autotuner of the O(T^2) solve's launch plan (right-hand-side tile x
 * k-block count): times the `budget` best-ranked candidate plans of that
 * method (whatever zr_solve_method chose) on synthetic data of shape (T, S)
 * and records the fastest in the context; later calls with that shape that
 * take the O(T^2) method use it.  Plans change the schedule only, never the
 * values.
 * zr_step_plan reports the plan a call of shape (T, S) would use. */
zr_status zr_autotune_step(zr_ctx* ctx, int64_t T, int32_t S, int32_t budget, void* stream);
zr_status zr_step_plan(zr_ctx* ctx, int64_t T, int32_t S, int32_t* s_tile, int32_t* nblocks);

/* ---------------------------------------------------------------------------
 * Transposed Vandermonde systems (Sec. 1: the probes y^1..y^t make the system
 * Vandermonde; Sec. 2.2: solved through Horner values and scaled by an
 * inverse).  One zr_vsys holds S right-hand sides that share the nodes v:
 *     offset 0:  sum_j c[s][j] v_j^k     = b[s][k],  k = 0..T-1
 *     offset 1:  sum_j c[s][j] v_j^(k+1) = b[s][k],  k = 0..T-1
 *   T       number of unknowns (>= 0)
 *   S       right-hand sides (1..256)
 *   v       device, T nodes (pairwise distinct; nonzero when offset = 1)
 *   b       device, S x ldb (ldb >= T)
 *   c       device, S x ldc output (ldc >= T); may not alias b
 * Errors: ZR_ERR_SINGULAR when two nodes coincide (or a node is 0 with
 * offset 1); c is then unspecified.
 * ------------------------------------------------------------------------- */
typedef struct zr_vsys {
  int64_t T;
  int32_t S;
  int32_t offset;
  const uint64_t* v;
  const uint64_t* b;
  int64_t ldb;
  uint64_t* c;
  int64_t ldc;
} zr_vsys;

/* Choice of solve method for the systems of every later call on the context
 * (steps, systems, reconstructions, the server):
 *   0  by size: the O(T log^2 T) method for T >= crossover, the O(T^2)
 *      method below it; crossover 0 takes the library's measured rule for a
 *      system of S right-hand sides, T >= 1024 for a system alone in its
 *      call and, in a call of several systems, also T^2 (S + 5) >= 8e7
 *      (about T >= 1750 for S = 21, 3600 for S = 1); for the probes of a
 *      function of Tf terms, the transposed-tree evaluator when T, Tf >=
 *      4096 and T Tf (S + 8) >= 1.8e9;
 *   1  always the O(T^2) method of Sec. 2.2 (Horner quotients, deferred dot
 *      products, one inverse per root);
 *   2  the O(T log^2 T) method for every T it supports.
 * The O(T log^2 T) method evaluates the same solution c_j = N(v_j) / M'(v_j)
 * through a subproduct tree: products of polynomials modulo p by
 * number-theoretic transforms over five 30-bit primes and the Chinese
 * remainder theorem, and a descent of the tree with middle products (a scaled
 * remainder tree), with M'(v_j) from the power sums of the nodes (summed
 * directly, T^2 products on every SM beside the tree, up to T = 12288;
 * above, rev(M') / rev(M) by Newton's iteration).  It handles 1 <= T <= 2^21;
 * larger systems always take the O(T^2) method.  Results are identical.
 * The paper's method is the O(T^2) one; this is a faster route to the same
 * values.  Errors: ZR_ERR_INVALID_ARG for a method outside 0..2 or a negative
 * crossover. */
zr_status zr_solve_method(zr_ctx* ctx, int32_t method, int64_t crossover);

/* Solves nsys independent systems (sys is a host array).  Systems of
 * different T and S share every launch: one set of launches for the whole
 * list, with a persistent solve kernel walking a work list of
 * (system, root tile, k-block, right-hand-side tile) items. */
zr_status zr_vandermonde_solve_batched(zr_ctx* ctx, int32_t nsys, const zr_vsys* sys, void* stream);
/* The plain form: one system after the other, each with its own launches
 * (the comparator the batched form is measured against). */
zr_status zr_vandermonde_solve_plain(zr_ctx* ctx, int32_t nsys, const zr_vsys* sys, void* stream);

/* ---------------------------------------------------------------------------
 * Batched Newton interpolation (Eq. newton): for every column j < nterms,
 * the polynomial of degree < npts through (x[s], vals[s][j]), s < npts,
 * written as monomial coefficients coef[e][j] (coefficient of z^e).
 *   x      device, npts pairwise distinct nodes (1 <= npts <= 64)
 *   vals   device, npts x ld;  coef: device, npts x ld (may alias vals)
 * Errors: ZR_ERR_SINGULAR when two nodes coincide.
 * ------------------------------------------------------------------------- */
zr_status zr_newton_batched(zr_ctx* ctx, int64_t nterms, int32_t npts, const uint64_t* x, const uint64_t* vals,
                            int64_t ld, uint64_t* coef, void* stream);

/* Allocation-free variant of zr_newton_batched, for callers that cannot
 * allocate device memory (a host program whose own pool owns the GPU memory,
 * or a latency-critical path that cannot take cudaMalloc's implicit
 * synchronisation) and therefore cannot create a zr_ctx.  The paper has no
 * counterpart; this is a library convenience.  Same arguments and results as
 * zr_newton_batched, with the prime passed directly (2^32 < p < 2^63) and
 * npts <= 64 (larger npts returns ZR_ERR_INVALID_ARG).  Its only scratch is a
 * fixed device array of 64*64+32 words that every GPU loading the library
 * holds until exit.  The first call on a device looks that array up with the
 * device current.  All calls share the
 * array (the call clears what must start at zero), so calls that overlap on
 * the GPU race: serialise them.  Waits for `stream`; ZR_ERR_SINGULAR when two
 * nodes coincide.  A CUDA error already pending on the calling thread belongs
 * to an earlier call: this call then returns ZR_ERR_CUDA without doing
 * anything and leaves that error pending. */
zr_status zr_newton_batched_noalloc(uint64_t prime, int64_t nterms, int32_t npts, const uint64_t* x,
                                    const uint64_t* vals, int64_t ld, uint64_t* coef, void* stream);

/* ---------------------------------------------------------------------------
 * Anchor values (Sec. 1): v_j = prod_{m < k} y_m^{e_{j,m}} for the T
 * exponent rows of a skeleton, with the distinctness check the solve needs.
 *   exps  device, T x nv bytes (term-major);  y: device, k values
 *   v     device, T outputs
 * Errors: ZR_ERR_SINGULAR as for the solve.
 * ------------------------------------------------------------------------- */
zr_status zr_anchor_values(zr_ctx* ctx, int64_t T, int32_t nv, const uint8_t* exps, int32_t k, const uint64_t* y,
                           int32_t offset, uint64_t* v, void* stream);

/* ---------------------------------------------------------------------------
 * A sparse polynomial: T terms over nv variables (1 <= nv <= 64), exponents
 * as bytes, term-major (row t = exponent vector of term t).
 * ------------------------------------------------------------------------- */
typedef struct zr_poly {
  int32_t nv;
  int64_t T;
  const uint8_t* exps; /* T x nv */
  const uint64_t* coef; /* T (may be NULL where only the support matters) */
} zr_poly;

/* ---------------------------------------------------------------------------
 * The Zippel step (Sec. 1) for the new variable x_k, k = newvar:
 *   skel    the skeleton: T monomials in x_0..x_{k-1} (columns >= k ignored);
 *           device arrays
 *   y       device, k anchor values (the probes are the powers y^(i+offset))
 *   samples device, S distinct values c_s of x_k (1 <= S <= 64)
 *   probes  device, S x ldb:  probes[s][i] = f(y^(i+offset), c_s, rest), i < T
 * Output: the new skeleton in x_0..x_k: for each input term j (in order) and
 * each power e < S (ascending) with nonzero coefficient g_{j,e}, the term
 * (exponents of j with column k = e and columns > k zero, g_{j,e}).
 *   out_exps  device, out_cap x nv;  out_coef: device, out_cap
 *   S*T terms always suffice.
 * zr_zippel_step waits and returns the status; *out_count (host) receives the
 * number of terms (also when it exceeds out_cap: ZR_ERR_CAPACITY).
 * zr_zippel_step_async leaves the count in d_out_count (device int64) and
 * device-detected conditions in the context (zr_stream_status).
 * ------------------------------------------------------------------------- */
zr_status zr_zippel_step(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                         const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                         uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap, int64_t* out_count, void* stream);
zr_status zr_zippel_step_async(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                               const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                               uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap, int64_t* d_out_count,
                               void* stream);
/* Waits for `stream` and returns the status of the device work enqueued by
 * the context's _async calls since the previous zr_stream_status. */
zr_status zr_stream_status(zr_ctx* ctx, void* stream);

/* Several Zippel steps of different T and S in shared launches (one set of
 * kernel launches for the whole list, a persistent solve kernel walking a
 * work list of (step, root tile, k-block, right-hand-side tile) items).
 * Each entry has the meaning of the zr_zippel_step arguments; out_count is a
 * device int64 per entry.  Waits for `stream`; the status covers all entries. */
typedef struct zr_step_desc {
  zr_poly skel;
  int32_t newvar;
  int32_t S;
  int32_t offset;
  int32_t pad;
  const uint64_t* y;
  const uint64_t* samples;
  const uint64_t* probes;
  int64_t ldb;
  uint8_t* out_exps;
  uint64_t* out_coef;
  int64_t out_cap;
  int64_t* out_count;
} zr_step_desc;
zr_status zr_zippel_step_batched(zr_ctx* ctx, int32_t nsteps, const zr_step_desc* steps, void* stream);

/* Steps captured into a CUDA graph (one graph per batch shape).  Create
 * checks the entries like zr_zippel_step_batched (every entry needs T >= 1),
 * stages their tables into workspace the graph owns, runs the steps once on
 * `stream` (waits; returns that run's status) and captures the kernel
 * sequence.  Every pointer of `steps` is baked into the graph: a launch
 * re-runs the same shapes on whatever those buffers hold at that time and
 * overwrites the same outputs, with one graph launch (asynchronous on
 * `stream`).  zr_step_graph_status waits for `stream` and returns the status
 * of the last run (ZR_ERR_SINGULAR etc.); zr_step_graph_kernels is the number
 * of kernels one launch runs.  *out is set whenever the graph was built, also
 * when the first run's status is an error (destroy it either way).  The
 * context must outlive the graph; the graph does not use the context's
 * workspace. */
typedef struct zr_step_graph zr_step_graph;
zr_status zr_step_graph_create(zr_ctx* ctx, int32_t nsteps, const zr_step_desc* steps, void* stream,
                               zr_step_graph** out);
zr_status zr_step_graph_launch(zr_step_graph* graph, void* stream);
zr_status zr_step_graph_status(zr_step_graph* graph, void* stream);
uint64_t zr_step_graph_kernels(const zr_step_graph* graph);
void zr_step_graph_destroy(zr_step_graph* graph);

/* The same step with every array in HOST memory (pinned or pageable): the
 * call copies the inputs in, runs the step on `stream` and copies the new
 * skeleton out.  out_exps / out_coef are host buffers of out_cap terms; the
 * call copies min(T S, out_cap) terms out in one transfer together with the
 * count, so the entries past *out_count are left unspecified (also when the
 * call returns an error). */
zr_status zr_zippel_step_host(zr_ctx* ctx, const zr_poly* skel, int32_t newvar, const uint64_t* y, int32_t S,
                              const uint64_t* samples, const uint64_t* probes, int64_t ldb, int32_t offset,
                              uint8_t* out_exps, uint64_t* out_coef, int64_t out_cap, int64_t* out_count,
                              void* stream);

/* ---------------------------------------------------------------------------
 * Sparse black-box evaluator (Sec. 2.2: powers of the base values substituted
 * into the polynomial, one value per thread group, partial sums reduced).
 * The Zippel probe family for new variable k:
 *     out[s][i] = f(y^(i+offset), c_s, z_{k+1}, .., z_{nv-1}),  s < S, i < T
 *   f        device terms (nv columns), coefficients required
 *   y        device k values; samples: device S values; z: device nv values
 *            (entries > k used; may be NULL when k = nv-1)
 *   out      device, S x ldo
 * ------------------------------------------------------------------------- */
zr_status zr_zippel_probes(zr_ctx* ctx, const zr_poly* f, int32_t k, const uint64_t* y, int32_t S,
                           const uint64_t* samples, const uint64_t* z, int64_t T, int32_t offset, uint64_t* out,
                           int64_t ldo, void* stream);
/* f at npts arbitrary points (device, npts x nv). */
zr_status zr_eval_points(zr_ctx* ctx, const zr_poly* f, int64_t npts, const uint64_t* pts, uint64_t* out,
                         void* stream);

/* The Zippel probe points themselves, for a caller that evaluates its own
 * black box: pts[(s T + i) nv + m] = y_m^(i+offset) (m < k), c_s (m = k),
 * z_m (m > k), for s < S, i < T; device arrays as for zr_zippel_probes, pts
 * a device buffer of S T nv residues.  Asynchronous on `stream`.
 * Errors: ZR_ERR_INVALID_ARG (nv outside 1..64, k outside 0..nv-1, S < 1,
 * T < 0, offset not 0/1, a needed pointer NULL). */
zr_status zr_probe_points(zr_ctx* ctx, int32_t nv, int32_t k, const uint64_t* y, int32_t S, const uint64_t* samples,
                          const uint64_t* z, int64_t T, int32_t offset, uint64_t* pts, void* stream);

/* ---------------------------------------------------------------------------
 * Balanced Zippel step for rational functions (Sec. 2.2, the balancing
 * identity).  For every probe i < max(TN, TD):
 *   fvals[s][i] = f(y^(i+offset), c_s, rest) for s < Sf = 2 max(dN, dD) + 2,
 *   a univariate rational reconstruction (Thiele, Eq. thiele) gives n_i/d_i
 *   with d_i(c_0) = 1; the factor D'(y^(i+offset)) of the previous
 *   denominator skeleton (skelD with coefficients) turns n_i(c_s), d_i(c_s)
 *   into C N(y^i, c_s) and C D(y^i, c_s), which feed one Zippel step for the
 *   numerator (dN+1 samples) and one for the denominator (dD+1 samples),
 *   batched into shared launches.
 * Outputs as for zr_zippel_step, one set per polynomial.
 * Errors: ZR_ERR_UNLUCKY on a degenerate Thiele table, ZR_ERR_DEGREE when a
 * probe needs more than the bounds allow, ZR_ERR_POLE when d_i(c_0) = 0.
 * ------------------------------------------------------------------------- */
zr_status zr_zippel_step_balanced(zr_ctx* ctx, const zr_poly* skelN, const zr_poly* skelD, int32_t newvar,
                                  const uint64_t* y, int32_t dN, int32_t dD, const uint64_t* samples,
                                  const uint64_t* fvals, int64_t ldf, int32_t offset, uint8_t* outN_exps,
                                  uint64_t* outN_coef, int64_t outN_cap, int64_t* outN_count, uint8_t* outD_exps,
                                  uint64_t* outD_coef, int64_t outD_cap, int64_t* outD_count, void* stream);

/* ---------------------------------------------------------------------------
 * Full reconstruction (Sec. 1), variable by variable: step 0 is a dense
 * univariate Newton (polynomial) or Thiele (rational) reconstruction in x_0
 * with x_1.. fixed at seeded rest values z; steps k >= 1 are Zippel steps.
 * Random values come from splitmix64 used as a counter-based generator
 * (key(seed, stream) = mix(seed + (stream+1) G), draw n = mix(key + (n+1) G),
 * G = 0x9E3779B97F4A7C15, residue = draw >> 1 rejected when 0 or >= p):
 *   stream 1:                 z_0 .. z_{nv-1}
 *   stream 1024 + 64 k + a:   attempt a of step k: y_0..y_{k-1}, then the
 *                             samples (c_0 = z_k for k >= 1), each rejected
 *                             when equal to an earlier sample.
 * A step whose anchor gives equal values (or a pole, or a degenerate Thiele
 * table) is redrawn with the next attempt (at most 64).
 * Verification (prm.verify, forced on by an unknown degree): after step k the
 * new skeleton P (N, D for a rational function) is compared with the black
 * box at one point (r_0..r_k, z_{k+1}..), r from stream 2^32 + 64 k + a:
 * P(r) = f(r) (N(r) = f(r) D(r), or N(r) D_f(r) = D(r) N_f(r) for a built-in
 * rational box).  A mismatch (an unlucky anchor, or a degree above the bound)
 * discards the step and redraws it.  A negative degree bound means unknown:
 * the step starts with bound 3 and, after each mismatch (or a Thiele table
 * longer than the bounds allow), doubles it plus one (7, 15, 31, 63; 31 for
 * a rational function), failing with ZR_ERR_DEGREE after three mismatches at
 * the largest bound.  Verification draws no value of the other streams, so
 * a verified run that never mismatches takes the same probes as one without.
 * The rational result is normalised so that the lexicographically smallest
 * exponent vector of the denominator has coefficient 1.
 * ------------------------------------------------------------------------- */
typedef enum zr_bb_kind {
  ZR_BB_POLY = 0,          /* built-in sparse polynomial (term arrays) */
  ZR_BB_RATIONAL = 1,      /* built-in sparse N / D */
  ZR_BB_CALL_POLY = 2,     /* a polynomial evaluated by the caller's function */
  ZR_BB_CALL_RATIONAL = 3  /* a rational function evaluated by the caller's function */
} zr_bb_kind;

/* A black box given as a function.  It evaluates the hidden function at npts
 * points: pts is device memory, npts x nv residues row-major; out is device
 * memory, npts residues (for a rational function the value N/D).  It runs on
 * `stream` (enqueuing work there, or working synchronously) and returns 0, or
 * nonzero when some point cannot be evaluated (for a rational function, a
 * pole): the library then draws new points where the method allows (the
 * rational steps), else the reconstruction fails with ZR_ERR_POLE.  It is
 * called from the thread that runs the reconstruction (the server's lane
 * thread for zr_serve) and must not use the calling context. */
typedef int32_t (*zr_eval_fn)(void* user, int64_t npts, int32_t nv, const uint64_t* pts, uint64_t* out,
                              void* stream);

typedef struct zr_blackbox {
  int32_t kind;  /* zr_bb_kind */
  int32_t nv;
  /* built-in sparse hidden function, HOST arrays (copied by the call):
     N (or the polynomial) and, for ZR_BB_RATIONAL, D.  For the callback
     kinds the arrays are unused and TN + TD is only a size hint (the
     server's lanes and memory estimate). */
  int64_t TN;
  const uint8_t* N_exps;
  const uint64_t* N_coef;
  int64_t TD;
  const uint8_t* D_exps;
  const uint64_t* D_coef;
  zr_eval_fn eval;       /* callback kinds */
  void* user;            /* passed to eval */
} zr_blackbox;

typedef struct zr_recon_params {
  int32_t nv;
  int32_t offset;         /* 0: probes y^0..y^{T-1};  1: y^1..y^T */
  uint64_t seed;
  const int32_t* degN;    /* host, nv degree bounds (the polynomial's for ZR_BB_POLY); < 0: unknown */
  const int32_t* degD;    /* host, nv degree bounds of the denominator (rational only); < 0: unknown */
  int32_t verify;         /* nonzero: check every step at a fresh point (see above) */
  int32_t reserved;       /* 0 */
} zr_recon_params;

/* Library-allocated result (host memory); free with zr_result_free. */
typedef struct zr_result {
  int32_t nv;
  int32_t rational;
  int64_t TN;
  uint8_t* N_exps;
  uint64_t* N_coef;
  int64_t TD;
  uint8_t* D_exps;
  uint64_t* D_coef;
  int32_t steps;          /* Zippel steps run (redraws included) */
  int32_t redraws;
  double device_ms;       /* device time of the steps */
} zr_result;

zr_status zr_reconstruct(zr_ctx* ctx, const zr_blackbox* bb, const zr_recon_params* prm, zr_result** out,
                         void* stream);
void zr_result_free(zr_result* r);

/* ---------------------------------------------------------------------------
 * Rational numbers from modular images (Sec. 1: the reconstruction runs
 * modulo large primes; the rationals are recovered as a final step).
 * For each of n values, res[i ld + j] is value j modulo primes[i] (device,
 * i < nprimes, distinct primes in (2^32, 2^63), host array of nprimes <= 8).
 * The images are combined by the Chinese remainder theorem into x modulo
 * P = prod primes (Garner's mixed radix), then Wang's rational
 * reconstruction finds n / d = x (mod P) with |n|, d <= N =
 * floor(sqrt((P - 1) / 2)): the extended Euclidean algorithm on (P, x) is
 * stopped at the first remainder r <= N; with the cofactor t of x the value
 * is sign(t) r / |t|, accepted when 0 < |t| <= N and gcd(r, |t|) = 1 (the
 * answer is then unique).
 *   num, den  device, n x words uint64 each, little-endian; num in two's
 *             complement, den > 0; words >= zr_lift_words(nprimes) (2, 4 or
 *             8), the high words sign- or zero-extended
 *   ok        device, n int32: 1 accepted, 0 not (num = den = 0): more
 *             primes are needed, or the value is no such fraction
 * Synchronous on `stream`.  Errors: ZR_ERR_INVALID_ARG (sizes, a modulus
 * that is not a prime in range, repeated primes).
 * ------------------------------------------------------------------------- */
int32_t zr_lift_words(int32_t nprimes);   /* 0 when nprimes is not in 1..8 */
zr_status zr_rational_lift(zr_ctx* ctx, int32_t nprimes, const uint64_t* primes, int64_t n, const uint64_t* res,
                           int64_t ld, int32_t words, uint64_t* num, uint64_t* den, int32_t* ok, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of reconstructions.
 *
 * A server owns its context (do not use the context for anything else while
 * the server exists) and runs a scheduler thread.  Requests are admitted
 * while slots (max_slots) are free and the device memory held by the active
 * requests plus the new request's estimate stays within mem_budget bytes (a
 * request too large for the budget runs when nothing else is active).  Each
 * scheduler tick generates the probes of every active request's next step and
 * runs all those steps in one batch of launches; a finished request frees its
 * slot at once and waiting requests join at the next tick.  Skeletons and
 * probes stay on the device.  A request's result depends only on its own
 * black box and seed, never on the other requests in its batches.
 *
 * zr_serve_submit copies the request (thread-safe) and returns a ticket.
 * zr_serve_poll returns ZR_ERR_BUSY until the request is done, then its status
 * and (on success) its result, once; a ticket never issued or already handed
 * out gives ZR_ERR_INVALID_ARG.  zr_serve_wait waits at most timeout_us
 * (ZR_ERR_TIMEOUT).  zr_serve_stats_get reports latencies (completion minus
 * submission, milliseconds) over completed requests and the term throughput
 * between the first submission and the last completion.  zr_serve_destroy
 * completes every submitted request, frees uncollected results and the server.
 * ------------------------------------------------------------------------- */
typedef struct zr_server zr_server;
typedef struct zr_request {
  zr_blackbox bb;        /* host arrays, copied by zr_serve_submit */
  zr_recon_params prm;
} zr_request;
typedef struct zr_serve_stats {
  int64_t submitted, completed, failed, terms, ticks, batch_entries;
  int32_t max_active, pad;
  double p50_ms, p99_ms, mean_ms, wall_s, terms_per_s;
} zr_serve_stats;

zr_status zr_serve_create(zr_ctx* ctx, size_t mem_budget, int32_t max_slots, zr_server** out);
zr_status zr_serve_submit(zr_server* server, const zr_request* req, uint64_t* ticket);
zr_status zr_serve_poll(zr_server* server, uint64_t ticket, zr_result** out);
zr_status zr_serve_wait(zr_server* server, uint64_t ticket, int64_t timeout_us, zr_result** out);
zr_status zr_serve_stats_get(zr_server* server, zr_serve_stats* out);
void zr_serve_destroy(zr_server* server);

#ifdef __cplusplus
}
#endif

#endif /* ZR_H */
