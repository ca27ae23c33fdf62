// zr_serve.cu -- the serving loop: continuous batching of reconstructions.
//
// Requests (sparse polynomial or rational black boxes with their parameters)
// are submitted from any thread.  A scheduler thread owns the context:
//   * admission: a pending request starts when a slot is free and the device
//     memory held by the active requests plus its estimate fits the budget
//     (a request that cannot fit even alone runs when nothing else does);
//     starting runs its dense step in x_0;
//   * every tick gathers the next Zippel step of every active request -- their
//     probes are generated on the device, then all steps run in one batch of
//     launches (run_batch) -- reads back each request's own status word and
//     term counts, and advances each request (or redraws its anchor);
//   * finished requests leave their slot at once, so requests that arrive
//     while others are on the GPU join at the next tick.
// A request's result depends only on its own black box and seed, never on
// the batch it ran in.  Skeletons and probe buffers stay on the device.
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

struct zr_server {
  zr_ctx* ctx = nullptr;
  size_t budget = 0;
  int max_slots = 0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_set<uint64_t> live;     // submitted, result not yet handed out
  uint64_t next_ticket = 1;
  // statistics (under mu)
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, terms = 0, ticks = 0, batch_entries = 0;
  int max_active = 0;
  double t_first = -1, t_last = 0;
  // device per-slot words
  cudaStream_t stream = nullptr;
  uint32_t* d_status = nullptr;
  uint32_t* h_status = nullptr;
  int64_t* d_counts = nullptr;
  int64_t* h_counts = nullptr;
};

static void finish_request(zr_server* s, Active& a, zr_status st) {
  zr_result* res = st == ZR_OK ? a.recon->take_result() : nullptr;
  const double t = now_ms();
  delete a.recon;
  a.recon = nullptr;
  std::lock_guard<std::mutex> g(s->mu);
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
}

static void server_loop(zr_server* s) {
  cudaSetDevice(s->ctx->device);
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
      s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty() || !active.empty(); });
      if (s->stop && s->pending.empty() && active.empty()) break;
      size_t held = 0;
      for (auto& a : active) held += a.recon->device_bytes();
      size_t planned = 0;
      while (!s->pending.empty() && (int)(active.size() + admit.size()) < s->max_slots) {
        Request& r = s->pending.front();
        r.bind();
        const size_t need = Recon::estimate_bytes(r.bb, r.prm);
        const bool alone = active.empty() && admit.empty();
        if (!alone && held + planned + need > s->budget) break;
        planned += need;
        admit.push_back(std::move(r));
        s->pending.pop_front();
      }
    }
    for (auto& r : admit) {
      r.bind();
      Active a{r.ticket, r.t_submit, free_slots.back(), new Recon(s->ctx, s->stream, r.bb, r.prm)};
      free_slots.pop_back();
      const zr_status st = a.recon->start();
      if (st || a.recon->done()) {
        free_slots.push_back(a.slot);
        finish_request(s, a, st);
      } else {
        active.push_back(a);
      }
    }
    if (active.empty()) continue;
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->max_active = std::max(s->max_active, (int)active.size());
    }
    // one tick: the next step of every active request in one batch
    items.clear();
    in_batch.assign(active.size(), 0);
    cudaMemsetAsync(s->d_status, 0, sizeof(uint32_t) * s->max_slots, s->stream);
    for (size_t i = 0; i < active.size(); i++) {
      Active& a = active[i];
      const zr_status st = a.recon->prepare(items, s->d_status + a.slot, s->d_counts + 2 * a.slot);
      in_batch[i] = st == ZR_OK;
    }
    zr_status bst = run_batch(s->ctx, items.data(), (int)items.size(), s->ctx->d_status_call, s->stream);
    cudaError_t e = cudaMemcpyAsync(s->h_status, s->d_status, sizeof(uint32_t) * s->max_slots, cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->h_counts, s->d_counts, sizeof(int64_t) * 2 * s->max_slots, cudaMemcpyDeviceToHost,
                          s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess && bst == ZR_OK) bst = cuda_err(s->ctx, e, "serve tick");
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->ticks++;
      s->batch_entries += (int64_t)items.size();
    }
    std::vector<Active> still;
    for (size_t i = 0; i < active.size(); i++) {
      Active& a = active[i];
      zr_status st = in_batch[i] ? (bst ? bst : a.recon->finish(s->h_status[a.slot], s->h_counts + 2 * a.slot))
                                 : a.recon->error();
      if (st || a.recon->done()) {
        free_slots.push_back(a.slot);
        finish_request(s, a, st);
      } else {
        still.push_back(a);
      }
    }
    active.swap(still);
  }
}

extern "C" zr_status zr_serve_create(zr_ctx* ctx, size_t mem_budget, int32_t max_slots, zr_server** out) {
  if (!ctx || !out || max_slots < 1 || max_slots > 4096 || mem_budget == 0) return ZR_ERR_INVALID_ARG;
  *out = nullptr;
  zr_server* s = new (std::nothrow) zr_server();
  if (!s) return ZR_ERR_OOM;
  s->ctx = ctx;
  s->budget = mem_budget;
  s->max_slots = max_slots;
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_status, sizeof(uint32_t) * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_status, sizeof(uint32_t) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_counts, sizeof(int64_t) * 2 * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_counts, sizeof(int64_t) * 2 * max_slots);
  if (e != cudaSuccess) {
    if (s->d_status) cudaFree(s->d_status);
    if (s->h_status) cudaFreeHost(s->h_status);
    if (s->d_counts) cudaFree(s->d_counts);
    if (s->h_counts) cudaFreeHost(s->h_counts);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return cuda_err(ctx, e, "zr_serve_create");
  }
  s->th = std::thread(server_loop, s);
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
  q.Ne.assign(req->bb.N_exps, req->bb.N_exps + (size_t)req->bb.TN * nv);
  q.Nc.assign(req->bb.N_coef, req->bb.N_coef + req->bb.TN);
  q.degN.assign(req->prm.degN, req->prm.degN + nv);
  if (req->bb.kind == ZR_BB_RATIONAL) {
    q.De.assign(req->bb.D_exps, req->bb.D_exps + (size_t)req->bb.TD * nv);
    q.Dc.assign(req->bb.D_coef, req->bb.D_coef + req->bb.TD);
    q.degD.assign(req->prm.degD, req->prm.degD + nv);
  }
  q.t_submit = now_ms();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return ZR_ERR_BUSY;
    q.ticket = s->next_ticket++;
    *ticket = q.ticket;
    s->live.insert(q.ticket);
    if (s->t_first < 0) s->t_first = q.t_submit;
    s->submitted++;
    s->pending.push_back(std::move(q));
  }
  s->cv_work.notify_one();
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
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& kv : s->done) zr_result_free(kv.second.res);
  cudaFree(s->d_status);
  cudaFreeHost(s->h_status);
  cudaFree(s->d_counts);
  cudaFreeHost(s->h_counts);
  cudaStreamDestroy(s->stream);
  delete s;
}
