// zr_serve.cu -- the serving loop: continuous batching of reconstructions.
//
// Requests (sparse polynomial or rational black boxes with their parameters)
// are submitted from any thread and routed by size to one of two lanes: small
// requests (at most kSmallTerms hidden terms) to the fast lane, the rest to
// the slow lane.  Each lane has its own context, stream and scheduler thread;
// the fast lane's stream has the highest priority and the slow lane's solve
// runs one CTA per work item, so the small requests' kernels get SMs between
// the items of a large step instead of waiting for the whole step.  Per lane:
//   * admission: a pending request starts when a slot is free and the device
//     memory held by the active requests of both lanes plus its estimate fits
//     the budget (a request that cannot fit even alone runs when nothing else
//     does); starting runs its dense step in x_0;
//   * every tick gathers the next Zippel step of the lane's active requests,
//     oldest first, until the steps add up to kTickWork multiply-accumulate
//     equivalents (each step weighted by the solve and evaluator it takes)
//     -- their probes are generated on the device (polynomial requests' on
//     four probe streams at once, each with its own scratch), then all those
//     steps run in one batch of launches (run_batch) -- reads back each request's own
//     status word and term counts, and advances each request (or redraws its
//     anchor);
//   * finished requests leave their slot at once, so requests that arrive
//     while others are on the GPU join at the next tick.
// A request's result depends only on its own black box and seed, never on
// the lane or the batch it ran in.  Skeletons and probe buffers stay on the
// device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "zr_recon.h"

using namespace zr;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket;
  double t_submit;
  std::vector<uint8_t> Ne, De;
  std::vector<uint64_t> Nc, Dc;
  std::vector<int32_t> degN, degD;
  zr_blackbox bb;
  zr_recon_params prm;
  void bind() {
    bb.N_exps = Ne.data();
    bb.N_coef = Nc.data();
    bb.D_exps = De.empty() ? nullptr : De.data();
    bb.D_coef = Dc.empty() ? nullptr : Dc.data();
    prm.degN = degN.data();
    prm.degD = degD.empty() ? nullptr : degD.data();
  }
};

struct Active {
  uint64_t ticket;
  double t_submit;
  int slot;
  Recon* recon;
};

struct Done {
  zr_status st;
  zr_result* res;
  double t_submit, t_done;
};

}  // namespace

constexpr int64_t kSmallTerms = 2048;   // fast-lane requests: at most this many hidden terms
// A tick takes active requests oldest first until their next steps add up to
// this many multiply-accumulate equivalents (about 50 ms of the GPU), at
// least one: a single large step already fills the GPU, so batching more
// large steps only stretches every one of them, while small steps still
// share a tick.
constexpr double kTickWork = 1e11;

struct Lane {
  zr_ctx* ctx = nullptr;
  bool own_ctx = false;
  cudaStream_t stream = nullptr;
  std::deque<Request> pending;
  std::condition_variable cv_work;
  std::thread th;
  int active = 0;          // under the server mutex
  size_t held = 0;         // device bytes of the lane's active requests (under the mutex)
  uint32_t* d_status = nullptr;
  uint32_t* h_status = nullptr;
  int64_t* d_counts = nullptr;
  int64_t* h_counts = nullptr;
  // probe lanes: a tick's polynomial requests generate their probes on these
  // streams (round-robin, each with its own scratch in the lane's context),
  // and the batch waits for them
  cudaStream_t pst[zr_ctx::kProbeLanes] = {};
  cudaEvent_t pin[zr_ctx::kProbeLanes] = {}, pout[zr_ctx::kProbeLanes] = {};
};

struct zr_server {
  size_t budget = 0;
  int max_slots = 0;
  Lane lanes[2];
  std::mutex mu;
  std::condition_variable cv_done;
  bool stop = false;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_set<uint64_t> live;     // submitted, result not yet handed out
  uint64_t next_ticket = 1;
  // statistics (under mu)
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, terms = 0, ticks = 0, batch_entries = 0;
  int max_active = 0;
  double t_first = -1, t_last = 0;
};

static void finish_request(zr_server* s, int li, Active& a, zr_status st) {
  zr_result* res = st == ZR_OK ? a.recon->take_result() : nullptr;
  const double t = now_ms();
  delete a.recon;
  a.recon = nullptr;
  std::lock_guard<std::mutex> g(s->mu);
  s->lanes[li].active--;
  s->done[a.ticket] = Done{st, res, a.t_submit, t};
  if (st == ZR_OK) {
    s->completed++;
    s->lat_ms.push_back(t - a.t_submit);
    if (res) s->terms += res->TN + res->TD;
  } else {
    s->failed++;
  }
  s->t_last = t;
  s->cv_done.notify_all();
  s->lanes[1 - li].cv_work.notify_one();   // memory and a slot came free
}

static void server_loop(zr_server* s, int li) {
  Lane& L = s->lanes[li];
  cudaSetDevice(L.ctx->device);
  std::vector<Active> active;
  std::vector<int> free_slots;
  for (int i = s->max_slots - 1; i >= 0; i--) free_slots.push_back(i);
  std::vector<BatchItem> items;
  std::vector<char> in_batch;
  for (;;) {
    // admission
    std::vector<Request> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      L.cv_work.wait(lk, [&] { return s->stop || !L.pending.empty() || !active.empty(); });
      if (s->stop && L.pending.empty() && active.empty()) break;
      size_t held = s->lanes[0].held + s->lanes[1].held;
      const int busy = s->lanes[0].active + s->lanes[1].active;
      size_t planned = 0;
      while (!L.pending.empty() && busy + (int)admit.size() < s->max_slots) {
        Request& r = L.pending.front();
        r.bind();
        const size_t need = Recon::estimate_bytes(r.bb, r.prm);
        const bool alone = busy == 0 && admit.empty();
        if (!alone && held + planned + need > s->budget) break;
        planned += need;
        admit.push_back(std::move(r));
        L.pending.pop_front();
      }
      L.active += (int)admit.size();
      L.held += planned;
      s->max_active = std::max(s->max_active, s->lanes[0].active + s->lanes[1].active);
      if (admit.empty() && active.empty()) {
        // waiting for memory or slots the other lane holds: it notifies this
        // lane when a request finishes; the timeout bounds a missed wake-up
        L.cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    for (auto& r : admit) {
      r.bind();
      Active a{r.ticket, r.t_submit, free_slots.back(), new Recon(L.ctx, L.stream, r.bb, r.prm)};
      free_slots.pop_back();
      const zr_status st = a.recon->start();
      if (st || a.recon->done()) {
        free_slots.push_back(a.slot);
        finish_request(s, li, a, st);
      } else {
        active.push_back(a);
      }
    }
    if (active.empty()) {
      std::lock_guard<std::mutex> g(s->mu);
      L.held = 0;
      continue;
    }
    // one tick: the next steps of the oldest active requests, up to kTickWork
    // multiply-accumulates, in one batch
    std::stable_sort(active.begin(), active.end(),
                     [](const Active& x, const Active& y) { return x.t_submit < y.t_submit; });
    items.clear();
    in_batch.assign(active.size(), 0);
    std::vector<char> stepped(active.size(), 0);
    cudaMemsetAsync(L.d_status, 0, sizeof(uint32_t) * s->max_slots, L.stream);
    double work = 0;
    int nprep = 0;
    for (size_t i = 0; i < active.size(); i++) {
      Active& a = active[i];
      const double c = a.recon->next_cost();
      if (i > 0 && work + c > kTickWork) continue;
      work += c;
      stepped[i] = 1;
      const int j = nprep++ % zr_ctx::kProbeLanes;
      if (L.pst[j]) a.recon->set_probe_lane(L.pst[j], j, L.pin[j], L.pout[j]);
      const zr_status st = a.recon->prepare(items, L.d_status + a.slot, L.d_counts + 2 * a.slot);
      a.recon->set_probe_lane(nullptr, -1, nullptr, nullptr);
      in_batch[i] = st == ZR_OK;
    }
    for (int j = 0; j < zr_ctx::kProbeLanes && j < nprep; j++)
      if (L.pst[j]) cudaStreamWaitEvent(L.stream, L.pout[j], 0);
    zr_status bst = run_batch(L.ctx, items.data(), (int)items.size(), L.ctx->d_status_call, L.stream);
    cudaError_t e = cudaMemcpyAsync(L.h_status, L.d_status, sizeof(uint32_t) * s->max_slots, cudaMemcpyDeviceToHost,
                                    L.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.h_counts, L.d_counts, sizeof(int64_t) * 2 * s->max_slots, cudaMemcpyDeviceToHost,
                          L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess && bst == ZR_OK) bst = cuda_err(L.ctx, e, "serve tick");
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->ticks++;
      s->batch_entries += (int64_t)items.size();
    }
    std::vector<Active> still;
    for (size_t i = 0; i < active.size(); i++) {
      Active& a = active[i];
      if (!stepped[i]) {
        still.push_back(a);
        continue;
      }
      zr_status st = in_batch[i] ? (bst ? bst : a.recon->finish(L.h_status[a.slot], L.h_counts + 2 * a.slot))
                                 : a.recon->error();
      if (st || a.recon->done()) {
        free_slots.push_back(a.slot);
        finish_request(s, li, a, st);
      } else {
        still.push_back(a);
      }
    }
    active.swap(still);
    size_t held = 0;
    for (auto& a : active) held += a.recon->device_bytes();
    std::lock_guard<std::mutex> g(s->mu);
    L.held = held;
  }
}

static void lane_free(Lane& L) {
  if (L.d_status) cudaFree(L.d_status);
  if (L.h_status) cudaFreeHost(L.h_status);
  if (L.d_counts) cudaFree(L.d_counts);
  if (L.h_counts) cudaFreeHost(L.h_counts);
  if (L.stream) cudaStreamDestroy(L.stream);
  for (int j = 0; j < zr_ctx::kProbeLanes; j++) {
    if (L.pst[j]) cudaStreamDestroy(L.pst[j]);
    if (L.pin[j]) cudaEventDestroy(L.pin[j]);
    if (L.pout[j]) cudaEventDestroy(L.pout[j]);
    L.pst[j] = nullptr;
    L.pin[j] = L.pout[j] = nullptr;
  }
  if (L.own_ctx && L.ctx) zr_destroy(L.ctx);
  L.d_status = L.h_status = nullptr;
  L.d_counts = L.h_counts = nullptr;
  L.stream = nullptr;
  L.ctx = nullptr;
  L.own_ctx = false;
}

extern "C" zr_status zr_serve_create(zr_ctx* ctx, size_t mem_budget, int32_t max_slots, zr_server** out) {
  if (!ctx || !out || max_slots < 1 || max_slots > 4096 || mem_budget == 0) return ZR_ERR_INVALID_ARG;
  *out = nullptr;
  zr_server* s = new (std::nothrow) zr_server();
  if (!s) return ZR_ERR_OOM;
  s->budget = mem_budget;
  s->max_slots = max_slots;
  int lo = 0, hi = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);   // lo: least, hi: greatest priority
  zr_status r = ZR_OK;
  for (int li = 0; li < 2 && e == cudaSuccess && !r; li++) {
    Lane& L = s->lanes[li];
    if (li == 0) {
      L.ctx = ctx;
    } else {
      r = zr_create(ctx->M.p, &L.ctx);
      if (r) break;
      L.own_ctx = true;
      L.ctx->solve_persistent = false;   // let the fast lane's kernels in between work items
    }
    e = cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, li == 0 ? hi : lo);
    for (int j = 0; j < zr_ctx::kProbeLanes && e == cudaSuccess; j++) {
      e = cudaStreamCreateWithPriority(&L.pst[j], cudaStreamNonBlocking, li == 0 ? hi : lo);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.pin[j], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.pout[j], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&L.d_status, sizeof(uint32_t) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_status, sizeof(uint32_t) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_counts, sizeof(int64_t) * 2 * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_counts, sizeof(int64_t) * 2 * max_slots);
  }
  if (e != cudaSuccess || r) {
    for (auto& L : s->lanes) lane_free(L);
    delete s;
    return r ? r : cuda_err(ctx, e, "zr_serve_create");
  }
  for (int li = 0; li < 2; li++) s->lanes[li].th = std::thread(server_loop, s, li);
  *out = s;
  return ZR_OK;
}

extern "C" zr_status zr_serve_submit(zr_server* s, const zr_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return ZR_ERR_INVALID_ARG;
  zr_status r = check_recon_args(nullptr, &req->bb, &req->prm);
  if (r) return r;
  Request q;
  const int nv = req->prm.nv;
  q.bb = req->bb;
  q.prm = req->prm;
  const bool callback = req->bb.kind == ZR_BB_CALL_POLY || req->bb.kind == ZR_BB_CALL_RATIONAL;
  const bool rational = req->bb.kind == ZR_BB_RATIONAL || req->bb.kind == ZR_BB_CALL_RATIONAL;
  if (!callback) {
    q.Ne.assign(req->bb.N_exps, req->bb.N_exps + (size_t)req->bb.TN * nv);
    q.Nc.assign(req->bb.N_coef, req->bb.N_coef + req->bb.TN);
  }
  q.degN.assign(req->prm.degN, req->prm.degN + nv);
  if (rational) {
    if (!callback) {
      q.De.assign(req->bb.D_exps, req->bb.D_exps + (size_t)req->bb.TD * nv);
      q.Dc.assign(req->bb.D_coef, req->bb.D_coef + req->bb.TD);
    }
    q.degD.assign(req->prm.degD, req->prm.degD + nv);
  }
  q.t_submit = now_ms();
  // a callback's TN + TD is the caller's size hint
  const int li = (int64_t)req->bb.TN + (rational ? req->bb.TD : 0) <= kSmallTerms ? 0 : 1;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return ZR_ERR_BUSY;
    q.ticket = s->next_ticket++;
    *ticket = q.ticket;
    s->live.insert(q.ticket);
    if (s->t_first < 0) s->t_first = q.t_submit;
    s->submitted++;
    s->lanes[li].pending.push_back(std::move(q));
  }
  s->lanes[li].cv_work.notify_one();
  // the other lane may be waiting for memory this request no longer needs
  s->lanes[1 - li].cv_work.notify_one();
  return ZR_OK;
}

static zr_status take_done(zr_server* s, uint64_t ticket, zr_result** out) {
  auto it = s->done.find(ticket);
  const zr_status st = it->second.st;
  if (out) *out = it->second.res;
  else zr_result_free(it->second.res);
  s->done.erase(it);
  s->live.erase(ticket);
  s->cv_done.notify_all();     // other waiters on this ticket see it gone
  return st;
}

extern "C" zr_status zr_serve_poll(zr_server* s, uint64_t ticket, zr_result** out) {
  if (!s) return ZR_ERR_INVALID_ARG;
  if (out) *out = nullptr;
  std::lock_guard<std::mutex> g(s->mu);
  if (!s->live.count(ticket)) return ZR_ERR_INVALID_ARG;     // never issued, or already handed out
  if (!s->done.count(ticket)) return ZR_ERR_BUSY;
  return take_done(s, ticket, out);
}

extern "C" zr_status zr_serve_wait(zr_server* s, uint64_t ticket, int64_t timeout_us, zr_result** out) {
  if (!s) return ZR_ERR_INVALID_ARG;
  if (out) *out = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->live.count(ticket)) return ZR_ERR_INVALID_ARG;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us),
                                      [&] { return s->done.count(ticket) > 0 || !s->live.count(ticket); });
  if (!ok) return ZR_ERR_TIMEOUT;
  if (!s->done.count(ticket)) return ZR_ERR_INVALID_ARG;    // another caller took it meanwhile
  return take_done(s, ticket, out);
}

extern "C" zr_status zr_serve_stats_get(zr_server* s, zr_serve_stats* out) {
  if (!s || !out) return ZR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->terms = s->terms;
  out->ticks = s->ticks;
  out->batch_entries = s->batch_entries;
  out->max_active = s->max_active;
  std::vector<double> l = s->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_ms = sum / l.size();
  }
  if (s->t_first >= 0 && s->t_last > s->t_first) {
    out->wall_s = (s->t_last - s->t_first) / 1e3;
    out->terms_per_s = s->terms / out->wall_s;
  }
  return ZR_OK;
}

extern "C" void zr_serve_destroy(zr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  for (auto& L : s->lanes) L.cv_work.notify_all();
  for (auto& L : s->lanes)
    if (L.th.joinable()) L.th.join();
  for (auto& kv : s->done) zr_result_free(kv.second.res);
  for (auto& L : s->lanes) lane_free(L);
  delete s;
}
