// zr_recon.cu -- full reconstructions (Sec. 1) and the balanced step entry.
//
// zr_reconstruct runs the variable-by-variable loop on the device: step 0 is a
// dense univariate reconstruction in x_0 (Newton for polynomials, Thiele for
// rational functions) with x_1.. fixed at rest values z; every later step k is
// a Zippel step in x_k whose probes come from the sparse evaluator.  The
// skeleton stays on the device between steps; the host reads back only the
// term count of each step (it sizes the next launch) and the final result.
//
// Random values follow the documented splitmix64 schedule (include/zr.h), the
// same one the CPU oracle implements independently, so both pick the same
// anchors and samples.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "zr_internal.h"

using namespace zr;

namespace {

typedef unsigned __int128 u128;

// ---- splitmix64 as a counter-based generator ------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
uint64_t sm_at(uint64_t key, uint64_t n) { return sm_mix(key + (n + 1) * kGamma); }
struct Rng {
  uint64_t key, ctr = 0;
  Rng(uint64_t seed, uint64_t stream) : key(sm_at(seed, stream)) {}
  uint64_t residue(uint64_t p) {
    for (;;) {
      const uint64_t x = sm_at(key, ctr++) >> 1;
      if (x != 0 && x < p) return x;
    }
  }
};
constexpr uint64_t kStreamRest = 1;
uint64_t stream_step(int k, int attempt) { return 1024ull + 64ull * (uint64_t)k + (uint64_t)attempt; }
constexpr int kMaxAttempts = 64;

void draw_rest(uint64_t seed, int nv, uint64_t p, uint64_t* z) {
  Rng r(seed, kStreamRest);
  for (int m = 0; m < nv; m++) z[m] = r.residue(p);
}
void draw_step(uint64_t seed, int k, int attempt, bool have_c0, uint64_t c0, int S, uint64_t p, uint64_t* y,
               uint64_t* cs) {
  Rng r(seed, stream_step(k, attempt));
  for (int m = 0; m < k; m++) y[m] = r.residue(p);
  int s0 = 0;
  if (have_c0) {
    cs[0] = c0;
    s0 = 1;
  }
  for (int s = s0; s < S; s++)
    for (;;) {
      const uint64_t c = r.residue(p);
      bool dup = false;
      for (int t = 0; t < s; t++) dup |= cs[t] == c;
      if (!dup) {
        cs[s] = c;
        break;
      }
    }
}

// ---- owned device memory -----------------------------------------------------
struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { if (p) cudaFree(p); }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 8);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// A device-resident sparse polynomial.
struct DPoly {
  int nv = 0;
  int64_t T = 0;
  DBuf exps, coef;
  zr_poly view() const { return zr_poly{nv, T, exps.as<uint8_t>(), coef.as<uint64_t>()}; }
};

struct Call {
  zr_ctx* ctx;
  cudaStream_t st;
  const Mod& M;
  zr_status fail(zr_status s, const char* what) { return set_err(ctx, s, what); }
  zr_status cuda(cudaError_t e, const char* what) { return cuda_err(ctx, e, what); }
  // waits for the stream and turns the call status word into a zr_status
  zr_status sync_status() {
    cudaError_t e = cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda(e, "reconstruct");
    const uint32_t f = ctx->h_status[1];
    cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
    return status_from_flags(ctx, f);
  }
};

zr_status upload(Call& c, DBuf& b, const void* host, size_t bytes) {
  cudaError_t e = b.ensure(bytes);
  if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, c.st);
  return c.cuda(e, "upload");
}

// Zippel steps on device skeletons, in one batch: entry i turns skel[i] into
// out[i] (capacity T S) with its own samples and probes.  Counts come back
// through the context's count words.
zr_status zippel_steps_dev(Call& c, int n, const DPoly* const* skel, const int* k, const uint64_t* const* d_y,
                           const int* S, const uint64_t* const* d_cs, const uint64_t* const* d_b, const int64_t* ldb,
                           int offset, DPoly* const* out) {
  std::vector<BatchItem> items;
  std::vector<int> which;
  for (int i = 0; i < n; i++) {
    const int64_t T = skel[i]->T;
    const int64_t cap = T * S[i];
    cudaError_t e = out[i]->exps.ensure((size_t)(cap > 0 ? cap : 1) * skel[i]->nv);
    if (e == cudaSuccess) e = out[i]->coef.ensure(sizeof(uint64_t) * (cap > 0 ? cap : 1));
    if (e != cudaSuccess) return c.cuda(e, "step output");
    out[i]->nv = skel[i]->nv;
    out[i]->T = 0;
    if (T == 0) continue;
    BatchItem it;
    it.mode = 0;
    it.T = T;
    it.S = S[i];
    it.k = k[i];
    it.nv = skel[i]->nv;
    it.offset = offset;
    it.exps = skel[i]->exps.as<uint8_t>();
    it.y = d_y[i];
    it.xs = d_cs[i];
    it.b = d_b[i];
    it.ldb = ldb[i];
    it.out_exps = out[i]->exps.as<uint8_t>();
    it.out_coef = out[i]->coef.as<uint64_t>();
    it.out_cap = cap;
    it.out_count = c.ctx->d_count + items.size();
    items.push_back(it);
    which.push_back(i);
  }
  if (items.empty()) return ZR_OK;
  zr_status r = run_batch(c.ctx, items.data(), (int)items.size(), c.ctx->d_status_call, c.st);
  if (r) return r;
  cudaError_t e = cudaMemcpyAsync(c.ctx->h_count, c.ctx->d_count, sizeof(int64_t) * items.size(),
                                  cudaMemcpyDeviceToHost, c.st);
  if (e != cudaSuccess) return c.cuda(e, "step count");
  r = c.sync_status();
  for (size_t t = 0; t < which.size(); t++) out[which[t]]->T = c.ctx->h_count[t];
  return r;
}

zr_status zippel_step_dev(Call& c, const DPoly& skel, int k, const uint64_t* d_y, int S, const uint64_t* d_cs,
                          const uint64_t* d_b, int64_t ldb, int offset, DPoly& out) {
  const DPoly* sk[1] = {&skel};
  DPoly* o[1] = {&out};
  return zippel_steps_dev(c, 1, sk, &k, &d_y, &S, &d_cs, &d_b, &ldb, offset, o);
}

// Univariate dense reconstruction helpers for step 0 --------------------------

// Newton through (cs[s], vals[s]), s < S, on the device; coefficients to host.
zr_status newton_coeffs(Call& c, int S, const uint64_t* d_cs, const uint64_t* d_vals, std::vector<uint64_t>& coef,
                        DBuf& scratch) {
  cudaError_t e = scratch.ensure(sizeof(uint64_t) * ((size_t)S * S + S));
  if (e != cudaSuccess) return c.cuda(e, "newton scratch");
  uint64_t* invd = scratch.as<uint64_t>();
  uint64_t* out = invd + (size_t)S * S;
  launch_newton_table(S, d_cs, c.M, invd, c.ctx->d_status_call, c.st);
  launch_newton(1, S, d_cs, invd, d_vals, 1, c.M, out, c.st);
  coef.assign(S, 0);
  e = cudaMemcpyAsync(coef.data(), out, sizeof(uint64_t) * S, cudaMemcpyDeviceToHost, c.st);
  if (e != cudaSuccess) return c.cuda(e, "newton copy");
  return c.sync_status();
}

// Skeleton in x_0 from coefficients (nonzero powers), uploaded to the device.
zr_status skeleton_from_coeffs(Call& c, int nv, const std::vector<uint64_t>& coef, int deg, DPoly& out) {
  std::vector<uint8_t> ex;
  std::vector<uint64_t> cf;
  for (int e = 0; e <= deg && e < (int)coef.size(); e++)
    if (coef[e]) {
      for (int m = 0; m < nv; m++) ex.push_back(m == 0 ? (uint8_t)e : 0);
      cf.push_back(coef[e]);
    }
  out.nv = nv;
  out.T = (int64_t)cf.size();
  zr_status r = upload(c, out.exps, ex.data(), ex.size());
  if (!r) r = upload(c, out.coef, cf.data(), cf.size() * sizeof(uint64_t));
  return r;
}

// The probe points of step 0: (c_s, z_1, .., z_{nv-1}).
std::vector<uint64_t> step0_points(int nv, int S, const uint64_t* cs, const uint64_t* z) {
  std::vector<uint64_t> pts((size_t)S * nv);
  for (int s = 0; s < S; s++)
    for (int m = 0; m < nv; m++) pts[(size_t)s * nv + m] = m == 0 ? cs[s] : z[m];
  return pts;
}

zr_result* make_result(int nv, bool rational) {
  zr_result* r = (zr_result*)calloc(1, sizeof(zr_result));
  if (r) {
    r->nv = nv;
    r->rational = rational ? 1 : 0;
  }
  return r;
}

zr_status download_poly(Call& c, const DPoly& p, int64_t* T, uint8_t** exps, uint64_t** coef) {
  *T = p.T;
  *exps = (uint8_t*)malloc((size_t)(p.T > 0 ? p.T : 1) * p.nv);
  *coef = (uint64_t*)malloc(sizeof(uint64_t) * (p.T > 0 ? p.T : 1));
  if (!*exps || !*coef) return c.fail(ZR_ERR_OOM, "result allocation");
  cudaError_t e = cudaSuccess;
  if (p.T > 0) {
    e = cudaMemcpyAsync(*exps, p.exps.p, (size_t)p.T * p.nv, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*coef, p.coef.p, sizeof(uint64_t) * p.T, cudaMemcpyDeviceToHost, c.st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  return c.cuda(e, "result copy");
}

bool retryable(zr_status s) { return s == ZR_ERR_SINGULAR || s == ZR_ERR_POLE || s == ZR_ERR_UNLUCKY; }

// ---- polynomial ---------------------------------------------------------------
zr_status reconstruct_poly(Call& c, const zr_blackbox* bb, const zr_recon_params* prm, zr_result* res) {
  const int nv = prm->nv;
  const uint64_t p = c.M.p;
  std::vector<uint64_t> z(nv), y(nv + 1), cs;
  draw_rest(prm->seed, nv, p, z.data());
  DPoly f;
  f.nv = nv;
  f.T = bb->TN;
  zr_status r = upload(c, f.exps, bb->N_exps, (size_t)bb->TN * nv);
  if (!r) r = upload(c, f.coef, bb->N_coef, sizeof(uint64_t) * bb->TN);
  if (r) return r;
  DBuf d_pts, d_vals, d_y, d_cs, d_z, d_b, scratch;
  if ((r = upload(c, d_z, z.data(), sizeof(uint64_t) * nv))) return r;
  DPoly cur, next;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c.st);
  // step 0: dense Newton in x_0
  {
    const int S = prm->degN[0] + 1;
    cs.assign(S, 0);
    draw_step(prm->seed, 0, 0, false, 0, S, p, y.data(), cs.data());
    std::vector<uint64_t> pts = step0_points(nv, S, cs.data(), z.data());
    if ((r = upload(c, d_pts, pts.data(), pts.size() * 8))) return r;
    if ((r = upload(c, d_cs, cs.data(), cs.size() * 8))) return r;
    cudaError_t e = d_vals.ensure(8 * (size_t)S);
    if (e != cudaSuccess) return c.cuda(e, "values");
    zr_poly fv = f.view();
    launch_eval_points(&fv, S, d_pts.as<uint64_t>(), c.M, d_vals.as<uint64_t>(), c.st);
    std::vector<uint64_t> coef;
    if ((r = newton_coeffs(c, S, d_cs.as<uint64_t>(), d_vals.as<uint64_t>(), coef, scratch))) return r;
    if ((r = skeleton_from_coeffs(c, nv, coef, S - 1, cur))) return r;
  }
  int steps = 0, redraws = 0;
  for (int k = 1; k < nv; k++) {
    const int S = prm->degN[k] + 1;
    cs.assign(S, 0);
    for (int attempt = 0;; attempt++) {
      draw_step(prm->seed, k, attempt, true, z[k], S, p, y.data(), cs.data());
      if ((r = upload(c, d_y, y.data(), 8 * (size_t)k))) return r;
      if ((r = upload(c, d_cs, cs.data(), 8 * (size_t)S))) return r;
      const int64_t T = cur.T;
      cudaError_t e = d_b.ensure(8 * (size_t)S * (T > 0 ? T : 1));
      if (e != cudaSuccess) return c.cuda(e, "probes");
      zr_poly fv = f.view();
      if (T > 0) {
        r = probes_impl(c.ctx, &fv, k, d_y.as<uint64_t>(), S, d_cs.as<uint64_t>(), d_z.as<uint64_t>(), T,
                        prm->offset, d_b.as<uint64_t>(), T, c.ctx->d_status_call, c.st);
        if (r) return r;
      }
      r = zippel_step_dev(c, cur, k, d_y.as<uint64_t>(), S, d_cs.as<uint64_t>(), d_b.as<uint64_t>(), T > 0 ? T : 1,
                          prm->offset, next);
      steps++;
      if (r == ZR_ERR_SINGULAR && attempt + 1 < kMaxAttempts) {
        redraws++;
        continue;
      }
      break;
    }
    if (r) return r;
    std::swap(cur.exps.p, next.exps.p);
    std::swap(cur.exps.n, next.exps.n);
    std::swap(cur.coef.p, next.coef.p);
    std::swap(cur.coef.n, next.coef.n);
    cur.T = next.T;
  }
  cudaEventRecord(e1, c.st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  res->steps = steps;
  res->redraws = redraws;
  res->device_ms = ms;
  return download_poly(c, cur, &res->TN, &res->N_exps, &res->N_coef);
}

// ---- rational (balanced) ---------------------------------------------------------

// The balanced step on device skeletons (N without, D with coefficients).
zr_status balanced_step_dev(Call& c, const DPoly& skN, const DPoly& skD, int k, const uint64_t* d_y, int dN, int dD,
                            const uint64_t* d_cs, const uint64_t* d_f, int64_t ldf, int offset, DPoly& outN,
                            DPoly& outD, DBuf& persist) {
  const int64_t TN = skN.T, TD = skD.T, Tmax = std::max(TN, TD);
  const int Sf = 2 * std::max(dN, dD) + 2, SN = dN + 1, SD = dD + 1;
  if (Tmax == 0) {
    outN.T = outD.T = 0;
    outN.nv = skN.nv;
    outD.nv = skD.nv;
    return ZR_OK;
  }
  // persistent per-step buffers: dprev, bN, bD, Thiele scratch
  const size_t w_dprev = (size_t)Tmax, w_bN = (size_t)SN * (TN ? TN : 1), w_bD = (size_t)SD * (TD ? TD : 1);
  const size_t w_th = thiele_scratch_words(Tmax, Sf);
  const size_t w_ones = (size_t)skD.nv;
  cudaError_t e = persist.ensure(8 * (w_dprev + w_bN + w_bD + w_th + w_ones) + 4 * 256);
  if (e != cudaSuccess) return c.cuda(e, "balanced buffers");
  uint64_t* dprev = persist.as<uint64_t>();
  uint64_t* bN = dprev + w_dprev;
  uint64_t* bD = bN + w_bN;
  uint64_t* th = bD + w_bD;
  uint64_t* ones = th + w_th;
  {
    const std::vector<uint64_t> h(w_ones, 1);
    e = cudaMemcpyAsync(ones, h.data(), 8 * w_ones, cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return c.cuda(e, "balanced buffers");
  }
  // D' at the probes: the evaluator on the denominator skeleton, whose
  // exponents of x_k and later variables are zero (their values do not matter)
  zr_poly dv = skD.view();
  if (TD > 0) {
    zr_status r = probes_impl(c.ctx, &dv, k, d_y, 1, ones, ones, Tmax, offset, dprev, Tmax, c.ctx->d_status_call, c.st);
    if (r) return r;
  } else {
    cudaMemsetAsync(dprev, 0, 8 * Tmax, c.st);
  }
  launch_thiele_balance(Tmax, Sf, d_cs, d_f, ldf, dprev, dN, dD, TN, TD, th, c.M, bN, TN ? TN : 1, bD, TD ? TD : 1,
                        c.ctx->d_status_call, c.st);
  zr_status r = c.sync_status();
  if (r) return r;
  // the numerator and denominator steps share one batch of launches
  const DPoly* sk[2] = {&skN, &skD};
  DPoly* o[2] = {&outN, &outD};
  const int ks[2] = {k, k}, Ss[2] = {SN, SD};
  const uint64_t* ys[2] = {d_y, d_y};
  const uint64_t* css[2] = {d_cs, d_cs};
  const uint64_t* bs[2] = {bN, bD};
  const int64_t lds[2] = {TN ? TN : 1, TD ? TD : 1};
  return zippel_steps_dev(c, 2, sk, ks, ys, Ss, css, bs, lds, offset, o);
}

// f = N/D at the step's probe family (Sf samples, Tmax probes).
zr_status rational_probes(Call& c, const DPoly& N, const DPoly& D, int k, const uint64_t* d_y, int Sf,
                          const uint64_t* d_cs, const uint64_t* d_z, int64_t Tmax, int offset, DBuf& vals,
                          uint64_t** fout) {
  cudaError_t e = vals.ensure(8 * (size_t)Sf * Tmax * 4);
  if (e != cudaSuccess) return c.cuda(e, "rational probes");
  uint64_t* nvls = vals.as<uint64_t>();
  uint64_t* dvls = nvls + (size_t)Sf * Tmax;
  uint64_t* pre = dvls + (size_t)Sf * Tmax;
  uint64_t* f = pre + (size_t)Sf * Tmax;
  zr_poly nv_ = N.view(), dv_ = D.view();
  zr_status r = probes_impl(c.ctx, &nv_, k, d_y, Sf, d_cs, d_z, Tmax, offset, nvls, Tmax, c.ctx->d_status_call, c.st);
  if (!r) r = probes_impl(c.ctx, &dv_, k, d_y, Sf, d_cs, d_z, Tmax, offset, dvls, Tmax, c.ctx->d_status_call, c.st);
  if (r) return r;
  launch_ratio(Tmax, Sf, nvls, dvls, Tmax, c.M, pre, f, Tmax, c.ctx->d_status_call, c.st);
  *fout = f;
  return c.sync_status();
}

zr_status reconstruct_rational(Call& c, const zr_blackbox* bb, const zr_recon_params* prm, zr_result* res) {
  const int nv = prm->nv;
  const uint64_t p = c.M.p;
  std::vector<uint64_t> z(nv), y(nv + 1), cs;
  draw_rest(prm->seed, nv, p, z.data());
  DPoly N, D;
  N.nv = D.nv = nv;
  N.T = bb->TN;
  D.T = bb->TD;
  zr_status r = upload(c, N.exps, bb->N_exps, (size_t)bb->TN * nv);
  if (!r) r = upload(c, N.coef, bb->N_coef, 8 * (size_t)bb->TN);
  if (!r) r = upload(c, D.exps, bb->D_exps, (size_t)bb->TD * nv);
  if (!r) r = upload(c, D.coef, bb->D_coef, 8 * (size_t)bb->TD);
  if (r) return r;
  DBuf d_pts, d_vals, d_y, d_cs, d_z, scratch, persist, fv, one;
  if ((r = upload(c, d_z, z.data(), 8 * (size_t)nv))) return r;
  DPoly curN, curD, nextN, nextD;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c.st);
  int steps = 0, redraws = 0;
  // step 0: Thiele in x_0, then Newton through the dN+1 / dD+1 first samples
  {
    const int dN = prm->degN[0], dD = prm->degD[0];
    const int Sf = 2 * std::max(dN, dD) + 2;
    cs.assign(Sf, 0);
    const uint64_t unit = 1;
    if ((r = upload(c, one, &unit, 8))) return r;
    for (int attempt = 0;; attempt++) {
      draw_step(prm->seed, 0, attempt, false, 0, Sf, p, y.data(), cs.data());
      std::vector<uint64_t> pts = step0_points(nv, Sf, cs.data(), z.data());
      if ((r = upload(c, d_pts, pts.data(), pts.size() * 8))) return r;
      if ((r = upload(c, d_cs, cs.data(), cs.size() * 8))) return r;
      cudaError_t e = d_vals.ensure(8 * (size_t)Sf * 4 + 8 * (size_t)(dN + dD + 2));
      if (e != cudaSuccess) return c.cuda(e, "values");
      uint64_t* nvls = d_vals.as<uint64_t>();
      uint64_t* dvls = nvls + Sf;
      uint64_t* pre = dvls + Sf;
      uint64_t* f = pre + Sf;
      uint64_t* nval = f + Sf;
      uint64_t* dval = nval + (dN + 1);
      zr_poly nv_ = N.view(), dv_ = D.view();
      launch_eval_points(&nv_, Sf, d_pts.as<uint64_t>(), c.M, nvls, c.st);
      launch_eval_points(&dv_, Sf, d_pts.as<uint64_t>(), c.M, dvls, c.st);
      launch_ratio(1, Sf, nvls, dvls, 1, c.M, pre, f, 1, c.ctx->d_status_call, c.st);
      r = c.sync_status();
      if (!r) {
        e = persist.ensure(8 * thiele_scratch_words(1, Sf) + 256);
        if (e != cudaSuccess) return c.cuda(e, "thiele scratch");
        launch_thiele_balance(1, Sf, d_cs.as<uint64_t>(), f, 1, one.as<uint64_t>(), dN, dD, 1, 1,
                              persist.as<uint64_t>(), c.M, nval, 1, dval, 1, c.ctx->d_status_call, c.st);
        r = c.sync_status();
      }
      if (retryable(r) && r != ZR_ERR_SINGULAR && attempt + 1 < kMaxAttempts) {
        redraws++;
        continue;
      }
      if (r) return r;
      std::vector<uint64_t> cn, cd;
      if ((r = newton_coeffs(c, dN + 1, d_cs.as<uint64_t>(), nval, cn, scratch))) return r;
      if ((r = newton_coeffs(c, dD + 1, d_cs.as<uint64_t>(), dval, cd, scratch))) return r;
      if ((r = skeleton_from_coeffs(c, nv, cn, dN, curN))) return r;
      if ((r = skeleton_from_coeffs(c, nv, cd, dD, curD))) return r;
      break;
    }
  }
  for (int k = 1; k < nv; k++) {
    const int dN = prm->degN[k], dD = prm->degD[k];
    const int Sf = 2 * std::max(dN, dD) + 2;
    cs.assign(Sf, 0);
    for (int attempt = 0;; attempt++) {
      draw_step(prm->seed, k, attempt, true, z[k], Sf, p, y.data(), cs.data());
      if ((r = upload(c, d_y, y.data(), 8 * (size_t)k))) return r;
      if ((r = upload(c, d_cs, cs.data(), 8 * (size_t)Sf))) return r;
      const int64_t Tmax = std::max(curN.T, curD.T);
      uint64_t* f = nullptr;
      r = Tmax > 0 ? rational_probes(c, N, D, k, d_y.as<uint64_t>(), Sf, d_cs.as<uint64_t>(), d_z.as<uint64_t>(), Tmax,
                                     prm->offset, fv, &f)
                   : ZR_OK;
      if (!r)
        r = balanced_step_dev(c, curN, curD, k, d_y.as<uint64_t>(), dN, dD, d_cs.as<uint64_t>(), f, Tmax, prm->offset,
                              nextN, nextD, persist);
      steps++;
      if (retryable(r) && attempt + 1 < kMaxAttempts) {
        redraws++;
        continue;
      }
      break;
    }
    if (r) return r;
    std::swap(curN.exps.p, nextN.exps.p);
    std::swap(curN.exps.n, nextN.exps.n);
    std::swap(curN.coef.p, nextN.coef.p);
    std::swap(curN.coef.n, nextN.coef.n);
    curN.T = nextN.T;
    std::swap(curD.exps.p, nextD.exps.p);
    std::swap(curD.exps.n, nextD.exps.n);
    std::swap(curD.coef.p, nextD.coef.p);
    std::swap(curD.coef.n, nextD.coef.n);
    curD.T = nextD.T;
  }
  // normalise on the lexicographically smallest denominator term
  if (curD.T == 0) return c.fail(ZR_ERR_SINGULAR, "empty denominator");
  std::vector<uint8_t> dex((size_t)curD.T * nv);
  cudaError_t e = cudaMemcpyAsync(dex.data(), curD.exps.p, dex.size(), cudaMemcpyDeviceToHost, c.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  if (e != cudaSuccess) return c.cuda(e, "denominator exponents");
  int64_t best = 0;
  for (int64_t j = 1; j < curD.T; j++)
    if (memcmp(&dex[(size_t)j * nv], &dex[(size_t)best * nv], nv) < 0) best = j;
  if ((e = scratch.ensure(64)) != cudaSuccess) return c.cuda(e, "normalise");
  launch_normalise(curN.T, curN.coef.as<uint64_t>(), curD.T, curD.coef.as<uint64_t>(), curD.coef.as<uint64_t>() + best,
                   scratch.as<uint64_t>(), c.M, c.ctx->d_status_call, c.st);
  // the pivot itself is scaled last by the second launch only after the
  // inverse was taken, so it becomes 1
  if ((r = c.sync_status())) return r;
  cudaEventRecord(e1, c.st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  res->steps = steps;
  res->redraws = redraws;
  res->device_ms = ms;
  r = download_poly(c, curN, &res->TN, &res->N_exps, &res->N_coef);
  if (!r) r = download_poly(c, curD, &res->TD, &res->D_exps, &res->D_coef);
  return r;
}

}  // namespace

extern "C" void zr_result_free(zr_result* r) {
  if (!r) return;
  free(r->N_exps);
  free(r->N_coef);
  free(r->D_exps);
  free(r->D_coef);
  free(r);
}

extern "C" zr_status zr_reconstruct(zr_ctx* ctx, const zr_blackbox* bb, const zr_recon_params* prm, zr_result** out,
                                    void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (!out) return set_err(ctx, ZR_ERR_INVALID_ARG, "null result pointer");
  *out = nullptr;
  if (!bb || !prm || prm->nv < 1 || prm->nv > kMaxVars || bb->nv != prm->nv || (prm->offset != 0 && prm->offset != 1) ||
      !prm->degN || bb->TN < 0 || (bb->TN > 0 && (!bb->N_exps || !bb->N_coef)))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: bad black box or parameters");
  const bool rational = bb->kind == ZR_BB_RATIONAL;
  if (bb->kind != ZR_BB_POLY && !rational) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: unknown kind");
  if (rational && (!prm->degD || bb->TD <= 0 || !bb->D_exps || !bb->D_coef))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: rational black box needs a denominator");
  for (int m = 0; m < prm->nv; m++) {
    const int dn = prm->degN[m], dd = rational ? prm->degD[m] : 0;
    if (dn < 0 || dd < 0 || dn + 1 > 64 || (rational && 2 * std::max(dn, dd) + 2 > 64))
      return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: degree bounds out of range");
  }
  Call c{ctx, (cudaStream_t)stream, ctx->M};
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), c.st);
  zr_result* res = make_result(prm->nv, rational);
  if (!res) return set_err(ctx, ZR_ERR_OOM, "result allocation");
  zr_status r = rational ? reconstruct_rational(c, bb, prm, res) : reconstruct_poly(c, bb, prm, res);
  if (r) {
    zr_result_free(res);
    return r;
  }
  *out = res;
  return ZR_OK;
}

extern "C" zr_status zr_zippel_step_balanced(zr_ctx* ctx, const zr_poly* skelN, const zr_poly* skelD, int32_t newvar,
                                             const uint64_t* y, int32_t dN, int32_t dD, const uint64_t* samples,
                                             const uint64_t* fvals, int64_t ldf, int32_t offset, uint8_t* outN_exps,
                                             uint64_t* outN_coef, int64_t outN_cap, int64_t* outN_count,
                                             uint8_t* outD_exps, uint64_t* outD_coef, int64_t outD_cap,
                                             int64_t* outD_count, void* stream) {
  if (!ctx) return ZR_ERR_INVALID_ARG;
  if (!skelN || !skelD || skelN->nv != skelD->nv || skelN->nv < 1 || skelN->nv > kMaxVars || newvar < 1 ||
      newvar >= skelN->nv || dN < 0 || dD < 0 || 2 * std::max(dN, dD) + 2 > 64 || (offset != 0 && offset != 1) ||
      skelN->T < 0 || skelD->T < 0 || ldf < std::max(skelN->T, skelD->T) || !samples || !y ||
      (skelD->T > 0 && !skelD->coef))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_zippel_step_balanced: arguments out of range");
  Call c{ctx, (cudaStream_t)stream, ctx->M};
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), c.st);
  // wrap the caller's device arrays (no ownership)
  DPoly sN, sD, oN, oD;
  sN.nv = sD.nv = skelN->nv;
  sN.T = skelN->T;
  sD.T = skelD->T;
  sN.exps.p = (void*)skelN->exps;
  sD.exps.p = (void*)skelD->exps;
  sD.coef.p = (void*)skelD->coef;
  DBuf persist;
  zr_status r = balanced_step_dev(c, sN, sD, newvar, y, dN, dD, samples, fvals, ldf, offset, oN, oD, persist);
  sN.exps.p = sD.exps.p = sD.coef.p = nullptr;   // not owned
  if (outN_count) *outN_count = oN.T;
  if (outD_count) *outD_count = oD.T;
  if (r) return r;
  if (oN.T > outN_cap || oD.T > outD_cap) return set_err(ctx, ZR_ERR_CAPACITY, "output skeleton larger than capacity");
  cudaError_t e = cudaSuccess;
  if (oN.T > 0) {
    e = cudaMemcpyAsync(outN_exps, oN.exps.p, (size_t)oN.T * skelN->nv, cudaMemcpyDeviceToDevice, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(outN_coef, oN.coef.p, 8 * (size_t)oN.T, cudaMemcpyDeviceToDevice, c.st);
  }
  if (e == cudaSuccess && oD.T > 0) {
    e = cudaMemcpyAsync(outD_exps, oD.exps.p, (size_t)oD.T * skelD->nv, cudaMemcpyDeviceToDevice, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(outD_coef, oD.coef.p, 8 * (size_t)oD.T, cudaMemcpyDeviceToDevice, c.st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  return cuda_err(ctx, e, "zr_zippel_step_balanced");
}
