// zr_recon.cu -- full reconstructions (Sec. 1) and the balanced step entry.
//
// A reconstruction runs variable by variable on the device: step 0 is a dense
// univariate reconstruction in x_0 (Newton for polynomials, Thiele for
// rational functions) with x_1.. fixed at rest values z; every later step k
// is a Zippel step in x_k whose probes come from the sparse evaluator.  The
// skeleton stays on the device between steps; the host reads back only the
// term counts (they size the next step) and the final result.
//
// Random values follow the documented splitmix64 schedule (include/zr.h), the
// same one the CPU oracle implements independently, so both pick the same
// anchors and samples.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "zr_recon.h"

namespace zr {

namespace {

// Small uploads (a step's y powers and samples) travel as kernel parameters:
// the launch is asynchronous, where a copy from pageable host memory may wait
// for the stream's queued work.
constexpr int kParamWords = 128;
struct ParamWords {
  uint64_t w[kParamWords];
};
__global__ void k_store_words(uint64_t* __restrict__ dst, int n, ParamWords v) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = v.w[i];
}

// ---- splitmix64 as a counter-based generator --------------------------------
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
uint64_t stream_verify(int k, int attempt) { return (1ull << 32) + 64ull * (uint64_t)k + (uint64_t)attempt; }
constexpr int kMaxAttempts = 64;
constexpr int kAutoDegree = 3;    // first bound of a variable whose degree is unknown

uint64_t hmul(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }

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

bool retryable(zr_status s) { return s == ZR_ERR_SINGULAR || s == ZR_ERR_POLE || s == ZR_ERR_UNLUCKY; }

std::vector<uint64_t> step0_points(int nv, int S, const uint64_t* cs, const uint64_t* z) {
  std::vector<uint64_t> pts((size_t)S * nv);
  for (int s = 0; s < S; s++)
    for (int m = 0; m < nv; m++) pts[(size_t)s * nv + m] = m == 0 ? cs[s] : z[m];
  return pts;
}

}  // namespace

Recon::Recon(zr_ctx* ctx, cudaStream_t st, const zr_blackbox& bb, const zr_recon_params& prm)
    : ctx_(ctx),
      st_(st),
      M_(ctx->M),
      nv_(prm.nv),
      rational_(bb.kind == ZR_BB_RATIONAL || bb.kind == ZR_BB_CALL_RATIONAL),
      callback_(bb.kind == ZR_BB_CALL_POLY || bb.kind == ZR_BB_CALL_RATIONAL),
      eval_(bb.eval),
      user_(bb.user),
      seed_(prm.seed),
      offset_(prm.offset) {
  if (!callback_) {
    Ne_.assign(bb.N_exps, bb.N_exps + (size_t)bb.TN * nv_);
    Nc_.assign(bb.N_coef, bb.N_coef + bb.TN);
    if (rational_) {
      De_.assign(bb.D_exps, bb.D_exps + (size_t)bb.TD * nv_);
      Dc_.assign(bb.D_coef, bb.D_coef + bb.TD);
    }
  }
  for (DBuf* b : {&d_y_, &d_cs_, &d_z_, &d_b_, &d_pts_, &d_vals_, &scratch_, &persist_, &fv_, &one_, &ones_, &d_ppts_,
                  &d_vpt_, &d_vval_, &fN_.exps, &fN_.coef, &fD_.exps, &fD_.coef, &curN_.exps, &curN_.coef,
                  &curD_.exps, &curD_.coef, &nextN_.exps, &nextN_.coef, &nextD_.exps, &nextD_.coef})
    b->s = st_;
  degN_.assign(prm.degN, prm.degN + nv_);
  if (rational_) degD_.assign(prm.degD, prm.degD + nv_);
  else degD_.assign(nv_, 0);
  autoN_.assign(nv_, 0);
  autoD_.assign(nv_, 0);
  verify_ = prm.verify != 0;
  for (int m = 0; m < nv_; m++) {
    if (degN_[m] < 0) autoN_[m] = 1, degN_[m] = kAutoDegree, verify_ = true;
    if (degD_[m] < 0) autoD_[m] = 1, degD_[m] = kAutoDegree, verify_ = true;
  }
}

zr_status Recon::grow_degree(int k) {
  const int maxd = rational_ ? 31 : 63;
  bool any = false, grew = false;
  auto grow = [&](std::vector<int32_t>& d, const std::vector<char>& a) {
    if (!a[k]) return;
    any = true;
    if (d[k] < maxd) {
      d[k] = std::min(2 * d[k] + 1, maxd);
      grew = true;
    }
  };
  grow(degN_, autoN_);
  if (rational_) grow(degD_, autoD_);
  if (any && !grew && ++maxed_fails_ >= 3)
    return set_err(ctx_, ZR_ERR_DEGREE, "zr_reconstruct: degree above the largest detectable bound");
  return ZR_OK;
}

zr_status Recon::verify_step(int k) {
  const uint64_t p = M_.p;
  Rng rng(seed_, stream_verify(k, attempt_));
  std::vector<uint64_t> pt(nv_);
  cudaError_t e = d_vpt_.ensure(8 * (size_t)nv_);
  if (e == cudaSuccess) e = d_vval_.ensure(8 * 4);
  if (e != cudaSuccess) return cuda_err(ctx_, e, "verification");
  uint64_t* vv = d_vval_.as<uint64_t>();
  const uint64_t* dpt = d_vpt_.as<uint64_t>();
  for (int tries = 0; tries < 8; tries++) {
    for (int m = 0; m < nv_; m++) pt[m] = m <= k ? rng.residue(p) : z_[m];
    zr_status r = upload(d_vpt_, pt.data(), 8 * (size_t)nv_);
    if (r) return r;
    // the black box: f (or N_f, D_f for a built-in rational function)
    r = eval_at(fN_, 1, dpt, vv);
    if (!r && rational_ && !callback_) r = eval_at(fD_, 1, dpt, vv + 1);
    if (r == ZR_ERR_POLE) continue;   // the function's pole: another point
    if (r) return r;
    // the skeleton
    zr_poly sN = curN_.view();
    launch_eval_points(&sN, 1, dpt, M_, vv + 2, st_);
    if (rational_) {
      zr_poly sD = curD_.view();
      launch_eval_points(&sD, 1, dpt, M_, vv + 3, st_);
    }
    uint64_t h[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(h, vv, sizeof(h), cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) return cuda_err(ctx_, e, "verification");
    bool ok;
    if (!rational_) ok = h[0] == h[2];
    else if (callback_) ok = h[2] == hmul(h[0], h[3], p);
    else {
      if (h[1] == 0) continue;   // a pole of the built-in function
      ok = hmul(h[2], h[1], p) == hmul(h[3], h[0], p);
    }
    return ok ? ZR_OK : set_err(ctx_, ZR_ERR_UNLUCKY, "verification point mismatch");
  }
  return set_err(ctx_, ZR_ERR_UNLUCKY, "verification: no point off the poles");
}

zr_status Recon::eval_at(const DPoly& f, int64_t npts, const uint64_t* pts, uint64_t* out) {
  if (!callback_) {
    zr_poly fv = f.view();
    launch_eval_points(&fv, npts, pts, M_, out, st_);
    return cuda_err(ctx_, cudaGetLastError(), "black box");
  }
  const int32_t rc = eval_(user_, npts, nv_, pts, out, (void*)st_);
  if (rc) return set_err(ctx_, ZR_ERR_POLE, "the black box could not be evaluated at a probe");
  return cuda_err(ctx_, cudaGetLastError(), "black box");
}

zr_status Recon::fail(zr_status s) {
  phase_ = FAILED;
  err_ = s;
  return s;
}

zr_status Recon::sync_status() {
  cudaError_t e = cudaMemcpyAsync(ctx_->h_status + 1, ctx_->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st_);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx_, e, "reconstruct");
  const uint32_t f = ctx_->h_status[1];
  cudaMemsetAsync(ctx_->d_status_call, 0, sizeof(uint32_t), st_);
  return status_from_flags(ctx_, f);
}

zr_status Recon::upload(DBuf& b, const void* host, size_t bytes) {
  cudaError_t e = b.ensure(bytes);
  if (e == cudaSuccess && bytes && bytes % 8 == 0 && bytes <= 8 * (size_t)kParamWords) {
    ParamWords v;
    memcpy(v.w, host, bytes);
    k_store_words<<<1, kParamWords, 0, st_>>>(b.as<uint64_t>(), (int)(bytes / 8), v);
    note_launch();
    e = cudaGetLastError();
  } else if (e == cudaSuccess && bytes) {
    e = cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, st_);
  }
  return cuda_err(ctx_, e, "upload");
}

size_t Recon::device_bytes() const {
  const DBuf* bufs[] = {&d_y_, &d_cs_, &d_z_, &d_b_, &d_pts_, &d_vals_, &scratch_, &persist_, &fv_, &one_, &ones_};
  size_t s = fN_.bytes() + fD_.bytes() + curN_.bytes() + curD_.bytes() + nextN_.bytes() + nextD_.bytes() + d_ppts_.n;
  for (const DBuf* b : bufs) s += b->n;
  return s;
}

double Recon::next_cost() const {
  if (phase_ != RUN || k_ >= nv_) return 0;
  const int64_t TN = curN_.T, TfN = fN_.T;
  if (!rational_) {
    const int S = degN_[k_] + 1;
    return solve_work(ctx_, TN, S) + probe_work(ctx_, TN, S, TfN);
  }
  const int64_t TD = curD_.T, TfD = fD_.T;
  const int SN = degN_[k_] + 1, SD = degD_[k_] + 1;
  const int Sf = 2 * std::max(degN_[k_], degD_[k_]) + 2;
  const int64_t Tm = std::max(TN, TD);
  return solve_work(ctx_, TN, SN) + solve_work(ctx_, TD, SD) + probe_work(ctx_, Tm, Sf, TfN) +
         probe_work(ctx_, Tm, Sf, TfD);
}

size_t Recon::estimate_bytes(const zr_blackbox& bb, const zr_recon_params& prm) {
  // hidden function(s), the largest step (skeleton <= hidden terms, S <= 64
  // samples or 2 max(deg)+2 Thiele points) with its probes and outputs
  const bool rational = bb.kind == ZR_BB_RATIONAL || bb.kind == ZR_BB_CALL_RATIONAL;
  const bool callback = bb.kind == ZR_BB_CALL_POLY || bb.kind == ZR_BB_CALL_RATIONAL;
  const int64_t Tf = bb.TN + (rational ? bb.TD : 0);
  int smax = 1;
  for (int m = 0; m < prm.nv; m++) {
    // an unknown degree may grow to the largest bound
    const int dn = prm.degN[m] < 0 ? (rational ? 31 : 63) : prm.degN[m];
    const int dd = rational ? (prm.degD[m] < 0 ? 31 : prm.degD[m]) : 0;
    int s = dn + 1;
    if (rational) s = 2 * std::max(dn, dd) + 2;
    smax = std::max(smax, s);
  }
  const size_t row = (size_t)prm.nv + 8;
  return (size_t)Tf * row + 2 * (size_t)Tf * smax * row + (size_t)Tf * smax * 8 * (rational ? 6 : 1) +
         (callback ? (size_t)Tf * smax * 8 * prm.nv : 0) + (1 << 16);
}

zr_status Recon::newton_coeffs(int S, const uint64_t* d_cs, const uint64_t* d_vals, std::vector<uint64_t>& coef) {
  cudaError_t e = scratch_.ensure(sizeof(uint64_t) * ((size_t)S * S + S));
  if (e != cudaSuccess) return cuda_err(ctx_, e, "newton scratch");
  uint64_t* invd = scratch_.as<uint64_t>();
  uint64_t* out = invd + (size_t)S * S;
  launch_newton_table(S, d_cs, M_, invd, ctx_->d_status_call, st_);
  launch_newton(1, S, invd, d_vals, 1, M_, out, st_);
  coef.assign(S, 0);
  e = cudaMemcpyAsync(coef.data(), out, sizeof(uint64_t) * S, cudaMemcpyDeviceToHost, st_);
  if (e != cudaSuccess) return cuda_err(ctx_, e, "newton copy");
  return sync_status();
}

zr_status Recon::skeleton_from_coeffs(const std::vector<uint64_t>& coef, int deg, DPoly& out) {
  std::vector<uint8_t> ex;
  std::vector<uint64_t> cf;
  for (int e = 0; e <= deg && e < (int)coef.size(); e++)
    if (coef[e]) {
      for (int m = 0; m < nv_; m++) ex.push_back(m == 0 ? (uint8_t)e : 0);
      cf.push_back(coef[e]);
    }
  out.nv = nv_;
  out.T = (int64_t)cf.size();
  zr_status r = upload(out.exps, ex.data(), ex.size());
  if (!r) r = upload(out.coef, cf.data(), cf.size() * sizeof(uint64_t));
  return r;
}

zr_status Recon::download(const DPoly& p, int64_t* T, uint8_t** exps, uint64_t** coef) {
  *T = p.T;
  *exps = (uint8_t*)malloc((size_t)(p.T > 0 ? p.T : 1) * nv_);
  *coef = (uint64_t*)malloc(sizeof(uint64_t) * (p.T > 0 ? p.T : 1));
  if (!*exps || !*coef) return set_err(ctx_, ZR_ERR_OOM, "result allocation");
  cudaError_t e = cudaSuccess;
  if (p.T > 0) {
    e = cudaMemcpyAsync(*exps, p.exps.p, (size_t)p.T * nv_, cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*coef, p.coef.p, sizeof(uint64_t) * p.T, cudaMemcpyDeviceToHost, st_);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
  return cuda_err(ctx_, e, "result copy");
}

zr_status Recon::start() {
  const uint64_t p = M_.p;
  z_.assign(nv_, 0);
  y_.assign(nv_ + 1, 0);
  draw_rest(seed_, nv_, p, z_.data());
  cudaMemsetAsync(ctx_->d_status_call, 0, sizeof(uint32_t), st_);
  fN_.nv = fD_.nv = nv_;
  fN_.T = (int64_t)Nc_.size();
  zr_status r = callback_ ? ZR_OK : upload(fN_.exps, Ne_.data(), Ne_.size());
  if (!r && !callback_) r = upload(fN_.coef, Nc_.data(), 8 * Nc_.size());
  if (!r && rational_ && !callback_) {
    fD_.T = (int64_t)Dc_.size();
    r = upload(fD_.exps, De_.data(), De_.size());
    if (!r) r = upload(fD_.coef, Dc_.data(), 8 * Dc_.size());
  }
  if (!r) r = upload(d_z_, z_.data(), 8 * (size_t)nv_);
  if (r) return fail(r);
  attempt_ = 0;
  for (;;) {
    r = rational_ ? step0_rational() : step0_poly();
    if (!r && verify_) r = verify_step(0);
    if (!r) break;
    if (r == ZR_ERR_UNLUCKY || (r == ZR_ERR_DEGREE && (autoN_[0] || autoD_[0]))) {
      const zr_status g = grow_degree(0);
      if (g) return fail(g);
      if (attempt_ + 1 < kMaxAttempts) {
        attempt_++;
        redraws_++;
        continue;
      }
    }
    return fail(r);
  }
  phase_ = RUN;
  k_ = 1;
  attempt_ = 0;
  maxed_fails_ = 0;
  if (k_ >= nv_) return finalize();
  return ZR_OK;
}

zr_status Recon::step0_poly() {
  const int S = degN_[0] + 1;
  cs_.assign(S, 0);
  draw_step(seed_, 0, attempt_, false, 0, S, M_.p, y_.data(), cs_.data());
  std::vector<uint64_t> pts = step0_points(nv_, S, cs_.data(), z_.data());
  zr_status r = upload(d_pts_, pts.data(), pts.size() * 8);
  if (!r) r = upload(d_cs_, cs_.data(), cs_.size() * 8);
  if (r) return r;
  cudaError_t e = d_vals_.ensure(8 * (size_t)S);
  if (e != cudaSuccess) return cuda_err(ctx_, e, "values");
  if ((r = eval_at(fN_, S, d_pts_.as<uint64_t>(), d_vals_.as<uint64_t>()))) return r;
  std::vector<uint64_t> coef;
  if ((r = newton_coeffs(S, d_cs_.as<uint64_t>(), d_vals_.as<uint64_t>(), coef))) return r;
  return skeleton_from_coeffs(coef, S - 1, curN_);
}

zr_status Recon::step0_rational() {
  const int dN = degN_[0], dD = degD_[0];
  const int Sf = 2 * std::max(dN, dD) + 2;
  cs_.assign(Sf, 0);
  const uint64_t unit = 1;
  zr_status r = upload(one_, &unit, 8);
  if (r) return r;
  for (;; attempt_++) {
    draw_step(seed_, 0, attempt_, false, 0, Sf, M_.p, y_.data(), cs_.data());
    std::vector<uint64_t> pts = step0_points(nv_, Sf, cs_.data(), z_.data());
    if ((r = upload(d_pts_, pts.data(), pts.size() * 8))) return r;
    if ((r = upload(d_cs_, cs_.data(), cs_.size() * 8))) return r;
    cudaError_t e = d_vals_.ensure(8 * (size_t)Sf * 4 + 8 * (size_t)(dN + dD + 2));
    if (e != cudaSuccess) return cuda_err(ctx_, e, "values");
    uint64_t* nvls = d_vals_.as<uint64_t>();
    uint64_t* dvls = nvls + Sf;
    uint64_t* pre = dvls + Sf;
    uint64_t* f = pre + Sf;
    uint64_t* nval = f + Sf;
    uint64_t* dval = nval + (dN + 1);
    if (callback_) {
      r = eval_at(fN_, Sf, d_pts_.as<uint64_t>(), f);     // the caller's N / D
    } else {
      if (!(r = eval_at(fN_, Sf, d_pts_.as<uint64_t>(), nvls)) && !(r = eval_at(fD_, Sf, d_pts_.as<uint64_t>(), dvls))) {
        launch_ratio(1, Sf, nvls, dvls, 1, M_, pre, f, 1, ctx_->d_status_call, st_);
        r = sync_status();
      }
    }
    if (!r) {
      e = persist_.ensure(8 * thiele_scratch_words(1, Sf) + 256);
      if (e != cudaSuccess) return cuda_err(ctx_, e, "thiele scratch");
      launch_thiele_balance(1, Sf, d_cs_.as<uint64_t>(), f, 1, one_.as<uint64_t>(), dN, dD, 1, 1,
                            persist_.as<uint64_t>(), M_, nval, 1, dval, 1, ctx_->d_status_call, st_);
      r = sync_status();
    }
    if ((r == ZR_ERR_POLE || r == ZR_ERR_UNLUCKY) && attempt_ + 1 < kMaxAttempts) {
      redraws_++;
      continue;
    }
    if (r) return r;
    std::vector<uint64_t> cn, cd;
    if ((r = newton_coeffs(dN + 1, d_cs_.as<uint64_t>(), nval, cn))) return r;
    if ((r = newton_coeffs(dD + 1, d_cs_.as<uint64_t>(), dval, cd))) return r;
    if ((r = skeleton_from_coeffs(cn, dN, curN_))) return r;
    return skeleton_from_coeffs(cd, dD, curD_);
  }
}

zr_status Recon::step_entry(const DPoly& skel, int S, const uint64_t* b, int64_t ldb, DPoly& out, uint32_t* d_status,
                            int64_t* d_count, std::vector<BatchItem>& items) {
  const int64_t T = skel.T, cap = T * S;
  cudaError_t e = out.exps.ensure((size_t)(cap > 0 ? cap : 1) * nv_);
  if (e == cudaSuccess) e = out.coef.ensure(sizeof(uint64_t) * (cap > 0 ? cap : 1));
  if (e != cudaSuccess) return cuda_err(ctx_, e, "step output");
  out.nv = nv_;
  out.T = 0;
  if (T == 0) {
    cudaMemsetAsync(d_count, 0, 8, st_);
    return ZR_OK;
  }
  BatchItem it;
  it.mode = 0;
  it.T = T;
  it.S = S;
  it.k = k_;
  it.nv = nv_;
  it.offset = offset_;
  it.exps = skel.exps.as<uint8_t>();
  it.y = d_y_.as<uint64_t>();
  it.xs = d_cs_.as<uint64_t>();
  it.b = b;
  it.ldb = ldb;
  it.out_exps = out.exps.as<uint8_t>();
  it.out_coef = out.coef.as<uint64_t>();
  it.out_cap = cap;
  it.out_count = d_count;
  it.status = d_status;
  it.c0 = skel.coef.as<uint64_t>();   // the samples start at c_0 = z_k, where skel was taken
  items.push_back(it);
  return ZR_OK;
}

zr_status Recon::prepare(std::vector<BatchItem>& items, uint32_t* d_status, int64_t* d_counts) {
  if (phase_ != RUN) return err_;
  const uint64_t p = M_.p;
  const int k = k_;
  if (!rational_) {
    const int S = degN_[k] + 1;
    cs_.assign(S, 0);
    draw_step(seed_, k, attempt_, true, z_[k], S, p, y_.data(), cs_.data());
    zr_status r = upload(d_y_, y_.data(), 8 * (size_t)k);
    if (!r) r = upload(d_cs_, cs_.data(), 8 * (size_t)S);
    if (r) return fail(r);
    const int64_t T = curN_.T;
    cudaError_t e = d_b_.ensure(8 * (size_t)S * (T > 0 ? T : 1));
    if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "probes"));
    // the probes of samples 1..S-1 (rows 1.. of b): the step takes the
    // solution at c_0 = z_k from the skeleton's coefficients
    const int S1 = S >= 2 ? 1 : 0;
    uint64_t* b1 = d_b_.as<uint64_t>() + (size_t)S1 * (T > 0 ? T : 1);
    const uint64_t* cs1 = d_cs_.as<uint64_t>() + S1;
    if (T > 0 && callback_) {
      e = d_ppts_.ensure(8 * (size_t)(S - S1) * T * nv_);
      if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "probe points"));
      launch_probe_points(T, S - S1, nv_, k, offset_, d_y_.as<uint64_t>(), cs1, d_z_.as<uint64_t>(), M_,
                          d_ppts_.as<uint64_t>(), st_);
      if ((r = eval_at(fN_, (int64_t)(S - S1) * T, d_ppts_.as<uint64_t>(), b1))) return fail(r);
    } else if (T > 0) {
      zr_poly fv = fN_.view();
      if (pst_ && pev_in_ && pev_out_) {
        cudaEventRecord(pev_in_, st_);
        cudaStreamWaitEvent(pst_, pev_in_, 0);
        r = probes_impl(ctx_, &fv, k, d_y_.as<uint64_t>(), S - S1, cs1, d_z_.as<uint64_t>(), T, offset_, b1, T,
                        d_status, pst_, plane_);
        cudaEventRecord(pev_out_, pst_);
      } else {
        r = probes_impl(ctx_, &fv, k, d_y_.as<uint64_t>(), S - S1, cs1, d_z_.as<uint64_t>(), T, offset_, b1, T,
                        d_status, st_);
      }
      if (r) return fail(r);
    }
    r = step_entry(curN_, S, d_b_.as<uint64_t>(), T > 0 ? T : 1, nextN_, d_status, d_counts, items);
    return r ? fail(r) : ZR_OK;
  }
  // rational: probes of N and D, their ratio, the per-probe Thiele and the
  // balancing, checked before the two steps join the batch
  for (;; attempt_++) {
    // (unknown degrees grow between attempts)
    const int dN = degN_[k], dD = degD_[k];
    const int Sf = 2 * std::max(dN, dD) + 2, SN = dN + 1, SD = dD + 1;
    cs_.assign(Sf, 0);
    draw_step(seed_, k, attempt_, true, z_[k], Sf, p, y_.data(), cs_.data());
    zr_status r = upload(d_y_, y_.data(), 8 * (size_t)k);
    if (!r) r = upload(d_cs_, cs_.data(), 8 * (size_t)Sf);
    if (r) return fail(r);
    const int64_t TN = curN_.T, TD = curD_.T, Tmax = std::max(TN, TD);
    if (Tmax == 0) break;
    // f = N/D at (y^(i+off), c_s, z)
    cudaError_t e = fv_.ensure(8 * (size_t)Sf * Tmax * 4);
    if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "rational probes"));
    uint64_t* nvls = fv_.as<uint64_t>();
    uint64_t* dvls = nvls + (size_t)Sf * Tmax;
    uint64_t* pre = dvls + (size_t)Sf * Tmax;
    uint64_t* f = pre + (size_t)Sf * Tmax;
    if (callback_) {
      // f = N/D from the caller at the probe points
      e = d_ppts_.ensure(8 * (size_t)Sf * Tmax * nv_);
      if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "probe points"));
      launch_probe_points(Tmax, Sf, nv_, k, offset_, d_y_.as<uint64_t>(), d_cs_.as<uint64_t>(), d_z_.as<uint64_t>(),
                          M_, d_ppts_.as<uint64_t>(), st_);
      r = eval_at(fN_, (int64_t)Sf * Tmax, d_ppts_.as<uint64_t>(), f);
      if (r && r != ZR_ERR_POLE) return fail(r);
    } else {
      zr_poly nv_p = fN_.view(), dv_p = fD_.view();
      r = probes_impl(ctx_, &nv_p, k, d_y_.as<uint64_t>(), Sf, d_cs_.as<uint64_t>(), d_z_.as<uint64_t>(), Tmax,
                      offset_, nvls, Tmax, ctx_->d_status_call, st_);
      if (!r)
        r = probes_impl(ctx_, &dv_p, k, d_y_.as<uint64_t>(), Sf, d_cs_.as<uint64_t>(), d_z_.as<uint64_t>(), Tmax,
                        offset_, dvls, Tmax, ctx_->d_status_call, st_);
      if (r) return fail(r);
      launch_ratio(Tmax, Sf, nvls, dvls, Tmax, M_, pre, f, Tmax, ctx_->d_status_call, st_);
      r = sync_status();
    }
    if (!r) {
      // D' at the probes, Thiele per probe, balancing
      const size_t w_dprev = (size_t)Tmax, w_bN = (size_t)SN * (TN ? TN : 1), w_bD = (size_t)SD * (TD ? TD : 1);
      const size_t w_th = thiele_scratch_words(Tmax, Sf);
      e = persist_.ensure(8 * (w_dprev + w_bN + w_bD + w_th) + 256);
      if (e == cudaSuccess) e = ones_.ensure(8 * (size_t)nv_);
      if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "balanced buffers"));
      {
        const std::vector<uint64_t> h(nv_, 1);
        e = cudaMemcpyAsync(ones_.p, h.data(), 8 * (size_t)nv_, cudaMemcpyHostToDevice, st_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
        if (e != cudaSuccess) return fail(cuda_err(ctx_, e, "balanced buffers"));
      }
      uint64_t* dprev = persist_.as<uint64_t>();
      uint64_t* bN = dprev + w_dprev;
      uint64_t* bD = bN + w_bN;
      uint64_t* th = bD + w_bD;
      zr_poly dsk = curD_.view();
      if (TD > 0)
        r = probes_impl(ctx_, &dsk, k, d_y_.as<uint64_t>(), 1, ones_.as<uint64_t>(), ones_.as<uint64_t>(), Tmax,
                        offset_, dprev, Tmax, ctx_->d_status_call, st_);
      else
        cudaMemsetAsync(dprev, 0, 8 * Tmax, st_);
      if (r) return fail(r);
      launch_thiele_balance(Tmax, Sf, d_cs_.as<uint64_t>(), f, Tmax, dprev, dN, dD, TN, TD, th, M_, bN, TN ? TN : 1, bD,
                            TD ? TD : 1, ctx_->d_status_call, st_);
      r = sync_status();
      if (!r) {
        r = step_entry(curN_, SN, bN, TN ? TN : 1, nextN_, d_status, d_counts, items);
        if (!r) r = step_entry(curD_, SD, bD, TD ? TD : 1, nextD_, d_status, d_counts + 1, items);
        return r ? fail(r) : ZR_OK;
      }
    }
    steps_++;
    if (r == ZR_ERR_DEGREE && (autoN_[k] || autoD_[k])) {
      const zr_status g = grow_degree(k);
      if (g) return fail(g);
      r = ZR_ERR_UNLUCKY;
    }
    if (retryable(r) && attempt_ + 1 < kMaxAttempts) {
      redraws_++;
      continue;
    }
    return fail(r);
  }
  // empty skeletons: nothing to run
  cudaMemsetAsync(d_counts, 0, 16, st_);
  return ZR_OK;
}

zr_status Recon::finish(uint32_t flags, const int64_t* counts) {
  if (phase_ != RUN) return err_;
  steps_++;
  const zr_status st = status_from_flags(ctx_, flags);
  if (st) {
    if (retryable(st) && attempt_ + 1 < kMaxAttempts) {
      attempt_++;
      redraws_++;
      return ZR_OK;
    }
    return fail(st);
  }
  nextN_.T = counts[0];
  curN_.swap(nextN_);
  if (rational_) {
    nextD_.T = counts[1];
    curD_.swap(nextD_);
  }
  if (verify_) {
    zr_status v = verify_step(k_);
    if (v == ZR_ERR_UNLUCKY) {
      // back to the previous skeleton; the step runs again
      curN_.swap(nextN_);
      if (rational_) curD_.swap(nextD_);
      v = grow_degree(k_);
      if (!v && attempt_ + 1 < kMaxAttempts) {
        attempt_++;
        redraws_++;
        return ZR_OK;
      }
      return fail(v ? v : ZR_ERR_UNLUCKY);
    }
    if (v) return fail(v);
  }
  k_++;
  attempt_ = 0;
  maxed_fails_ = 0;
  if (k_ >= nv_) return finalize();
  return ZR_OK;
}

zr_status Recon::finalize() {
  zr_result* res = (zr_result*)calloc(1, sizeof(zr_result));
  if (!res) return fail(set_err(ctx_, ZR_ERR_OOM, "result allocation"));
  res->nv = nv_;
  res->rational = rational_ ? 1 : 0;
  res->steps = steps_;
  res->redraws = redraws_;
  zr_status r = ZR_OK;
  if (rational_) {
    // normalise on the lexicographically smallest denominator term
    if (curD_.T == 0) r = set_err(ctx_, ZR_ERR_SINGULAR, "empty denominator");
    std::vector<uint8_t> dex;
    if (!r) {
      dex.resize((size_t)curD_.T * nv_);
      cudaError_t e = cudaMemcpyAsync(dex.data(), curD_.exps.p, dex.size(), cudaMemcpyDeviceToHost, st_);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
      if (e == cudaSuccess) e = scratch_.ensure(64);
      if (e != cudaSuccess) r = cuda_err(ctx_, e, "normalise");
    }
    if (!r) {
      int64_t best = 0;
      for (int64_t j = 1; j < curD_.T; j++)
        if (memcmp(&dex[(size_t)j * nv_], &dex[(size_t)best * nv_], nv_) < 0) best = j;
      launch_normalise(curN_.T, curN_.coef.as<uint64_t>(), curD_.T, curD_.coef.as<uint64_t>(),
                       curD_.coef.as<uint64_t>() + best, scratch_.as<uint64_t>(), M_, ctx_->d_status_call, st_);
      r = sync_status();
    }
    if (!r) r = download(curD_, &res->TD, &res->D_exps, &res->D_coef);
  }
  if (!r) r = download(curN_, &res->TN, &res->N_exps, &res->N_coef);
  if (r) {
    zr_result_free(res);
    return fail(r);
  }
  result_ = res;
  phase_ = DONE;
  return ZR_OK;
}

zr_result* Recon::take_result() {
  zr_result* r = result_;
  result_ = nullptr;
  return r;
}

zr_status check_recon_args(zr_ctx* ctx, const zr_blackbox* bb, const zr_recon_params* prm) {
  if (!bb || !prm || prm->nv < 1 || prm->nv > kMaxVars || bb->nv != prm->nv || (prm->offset != 0 && prm->offset != 1) ||
      !prm->degN || bb->TN < 0 || bb->TD < 0)
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: bad black box or parameters");
  const bool callback = bb->kind == ZR_BB_CALL_POLY || bb->kind == ZR_BB_CALL_RATIONAL;
  const bool rational = bb->kind == ZR_BB_RATIONAL || bb->kind == ZR_BB_CALL_RATIONAL;
  if (bb->kind < ZR_BB_POLY || bb->kind > ZR_BB_CALL_RATIONAL)
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: unknown kind");
  if (callback && !bb->eval) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: callback black box without eval");
  if (!callback && bb->TN > 0 && (!bb->N_exps || !bb->N_coef))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: bad black box or parameters");
  if (rational && !prm->degD) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: rational needs degD");
  if (rational && !callback && (bb->TD <= 0 || !bb->D_exps || !bb->D_coef))
    return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: rational black box needs a denominator");
  if (prm->reserved != 0) return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: reserved must be 0");
  for (int m = 0; m < prm->nv; m++) {
    // negative: unknown (detected); the detection's first bound fits every range
    const int dn = std::max(prm->degN[m], 0), dd = rational ? std::max(prm->degD[m], 0) : 0;
    if (dn + 1 > 64 || (rational && 2 * std::max(dn, dd) + 2 > 64))
      return set_err(ctx, ZR_ERR_INVALID_ARG, "zr_reconstruct: degree bounds out of range");
  }
  return ZR_OK;
}

}  // namespace zr

using namespace zr;

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
  zr_status r = check_recon_args(ctx, bb, prm);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  Recon R(ctx, st, *bb, *prm);
  r = R.start();
  std::vector<BatchItem> items;
  while (!r && !R.done()) {
    items.clear();
    cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
    r = R.prepare(items, ctx->d_status_call, ctx->d_count);
    if (r) break;
    r = run_batch(ctx, items.data(), (int)items.size(), ctx->d_status_call, st);
    if (r) break;
    cudaError_t e = cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_count, ctx->d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      r = cuda_err(ctx, e, "zr_reconstruct");
      break;
    }
    r = R.finish(ctx->h_status[1], ctx->h_count);
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  if (r) return r;
  zr_result* res = R.take_result();
  if (!res) return set_err(ctx, ZR_ERR_CUDA, "reconstruction ended without a result");
  res->device_ms = ms;
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
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = skelN->nv;
  const int64_t TN = skelN->T, TD = skelD->T, Tmax = std::max(TN, TD);
  const int Sf = 2 * std::max(dN, dD) + 2, SN = dN + 1, SD = dD + 1;
  if (outN_count) *outN_count = 0;
  if (outD_count) *outD_count = 0;
  if (Tmax == 0) return ZR_OK;
  cudaMemsetAsync(ctx->d_status_call, 0, sizeof(uint32_t), st);
  DBuf persist, ones;
  persist.s = ones.s = st;   // allocated and freed in the order of the call's stream
  const size_t w_dprev = (size_t)Tmax, w_bN = (size_t)SN * (TN ? TN : 1), w_bD = (size_t)SD * (TD ? TD : 1);
  const size_t w_th = thiele_scratch_words(Tmax, Sf);
  cudaError_t e = persist.ensure(8 * (w_dprev + w_bN + w_bD + w_th) + 256);
  if (e == cudaSuccess) e = ones.ensure(8 * (size_t)nv);
  if (e == cudaSuccess) {
    const std::vector<uint64_t> h(nv, 1);
    e = cudaMemcpyAsync(ones.p, h.data(), 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_step_balanced: buffers");
  uint64_t* dprev = persist.as<uint64_t>();
  uint64_t* bN = dprev + w_dprev;
  uint64_t* bD = bN + w_bN;
  uint64_t* th = bD + w_bD;
  zr_status r = ZR_OK;
  if (TD > 0) {
    zr_poly dsk = *skelD;
    r = probes_impl(ctx, &dsk, newvar, y, 1, ones.as<uint64_t>(), ones.as<uint64_t>(), Tmax, offset, dprev, Tmax,
                    ctx->d_status_call, st);
  } else {
    cudaMemsetAsync(dprev, 0, 8 * Tmax, st);
  }
  if (r) return r;
  launch_thiele_balance(Tmax, Sf, samples, fvals, ldf, dprev, dN, dD, TN, TD, th, ctx->M, bN, TN ? TN : 1, bD,
                        TD ? TD : 1, ctx->d_status_call, st);
  // the numerator and denominator steps share one batch of launches
  BatchItem items[2];
  int n = 0;
  const zr_poly* sk[2] = {skelN, skelD};
  const int Ss[2] = {SN, SD};
  uint64_t* bs[2] = {bN, bD};
  uint8_t* oe[2] = {outN_exps, outD_exps};
  uint64_t* oc[2] = {outN_coef, outD_coef};
  const int64_t caps[2] = {outN_cap, outD_cap};
  cudaMemsetAsync(ctx->d_count, 0, 2 * sizeof(int64_t), st);
  for (int t = 0; t < 2; t++) {
    if (sk[t]->T == 0) continue;
    BatchItem& it = items[n++];
    it.mode = 0;
    it.T = sk[t]->T;
    it.S = Ss[t];
    it.k = newvar;
    it.nv = nv;
    it.offset = offset;
    it.exps = sk[t]->exps;
    it.y = y;
    it.xs = samples;
    it.b = bs[t];
    it.ldb = sk[t]->T;
    it.out_exps = oe[t];
    it.out_coef = oc[t];
    it.out_cap = caps[t];
    it.out_count = ctx->d_count + t;
  }
  if ((r = run_batch(ctx, items, n, ctx->d_status_call, st))) return r;
  e = cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status_call, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_count, ctx->d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "zr_zippel_step_balanced");
  if (outN_count) *outN_count = ctx->h_count[0];
  if (outD_count) *outD_count = ctx->h_count[1];
  r = status_from_flags(ctx, ctx->h_status[1]);
  if (r) return r;
  if (ctx->h_count[0] > outN_cap || ctx->h_count[1] > outD_cap)
    return set_err(ctx, ZR_ERR_CAPACITY, "output skeleton larger than capacity");
  return ZR_OK;
}
