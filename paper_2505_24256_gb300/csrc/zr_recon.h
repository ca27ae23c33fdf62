// zr_recon.h -- one reconstruction as a state machine over its steps, so
// that a single request (zr_reconstruct) and many requests at once (the
// serving loop) run the same code: start() does the dense step in x_0,
// prepare() enqueues the probe work of the next Zippel step and contributes
// that step's entries to a shared batch, finish() consumes the batch's
// status and counts for those entries and advances (or redraws).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "zr_internal.h"

namespace zr {

// Device memory owned by one request, allocated and freed in the order of
// the request's stream (the device's memory pool): growing a buffer between
// steps does not synchronise the device, so requests on other streams keep
// running.
struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;   // the owner's stream
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMallocAsync(&p, bytes > 0 ? bytes : 8, s);
    if (e == cudaSuccess) n = bytes > 0 ? bytes : 8;
    else p = nullptr;
    return e;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

struct DPoly {
  int nv = 0;
  int64_t T = 0;
  DBuf exps, coef;
  zr_poly view() const { return zr_poly{nv, T, exps.as<uint8_t>(), coef.as<uint64_t>()}; }
  void swap(DPoly& o) {
    std::swap(T, o.T);
    std::swap(nv, o.nv);
    std::swap(exps.p, o.exps.p);
    std::swap(exps.n, o.exps.n);
    std::swap(coef.p, o.coef.p);
    std::swap(coef.n, o.coef.n);
  }
  size_t bytes() const { return exps.n + coef.n; }
};

class Recon {
 public:
  // The black box arrays are copied.
  Recon(zr_ctx* ctx, cudaStream_t st, const zr_blackbox& bb, const zr_recon_params& prm);
  zr_status start();                  // uploads, dense step in x_0
  bool done() const { return phase_ == DONE; }
  bool failed() const { return phase_ == FAILED; }
  zr_status error() const { return err_; }
  // Enqueues the probes of the next step and appends its batch entries (one
  // for a polynomial, two for N and D) with the given status word and count
  // slots (two int64).  Synchronises when the rational path must check the
  // univariate reconstruction before the step.
  zr_status prepare(std::vector<BatchItem>& items, uint32_t* d_status, int64_t* d_counts);
  // The probe lane the next prepare() uses for a polynomial step's probes:
  // they run on `st` with the context's scratch of `lane`, after ev_in (recorded on
  // the request's stream once its inputs are there), and ev_out is recorded
  // after them; the caller makes its batch wait for ev_out.  st null: the
  // request's own stream, as for every other call.
  void set_probe_lane(cudaStream_t st, int lane, cudaEvent_t ev_in, cudaEvent_t ev_out) {
    pst_ = st;
    plane_ = lane;
    pev_in_ = ev_in;
    pev_out_ = ev_out;
  }
  // After the batch: this request's status flags and its count slots.
  zr_status finish(uint32_t flags, const int64_t* counts);
  zr_result* take_result();           // ownership passes to the caller
  size_t device_bytes() const;
  // multiply-accumulates of the next step (solves and probe evaluation),
  // for scheduling; 0 when the reconstruction is not running
  double next_cost() const;
  static size_t estimate_bytes(const zr_blackbox& bb, const zr_recon_params& prm);
  int steps() const { return steps_; }
  int redraws() const { return redraws_; }

 private:
  enum Phase { NEW, RUN, DONE, FAILED };
  zr_status fail(zr_status s);
  zr_status sync_status();
  zr_status upload(DBuf& b, const void* host, size_t bytes);
  zr_status step0_poly();
  zr_status step0_rational();
  zr_status finalize();
  zr_status newton_coeffs(int S, const uint64_t* d_cs, const uint64_t* d_vals, std::vector<uint64_t>& coef);
  zr_status skeleton_from_coeffs(const std::vector<uint64_t>& coef, int deg, DPoly& out);
  zr_status download(const DPoly& p, int64_t* T, uint8_t** exps, uint64_t** coef);
  // the step of skeleton skel (its coefficients are the solution at the first
  // sample, so only samples 1..S-1 are solved; b's row 0 is not read)
  zr_status step_entry(const DPoly& skel, int S, const uint64_t* b, int64_t ldb, DPoly& out, uint32_t* d_status,
                       int64_t* d_count, std::vector<BatchItem>& items);

  // the skeleton of step k against the black box at one fresh point:
  // ZR_OK, ZR_ERR_UNLUCKY on a mismatch, or an error
  zr_status verify_step(int k);
  // after a mismatch or a Thiele table too long for the bounds of step k:
  // grows the unknown bounds of variable k; ZR_OK to redraw, ZR_ERR_DEGREE
  // after repeated mismatches at the largest bound
  zr_status grow_degree(int k);

  // values of the black box at npts device points (npts x nv_) into out:
  // the built-in evaluator or the caller's function (nonzero: a pole)
  zr_status eval_at(const DPoly& f, int64_t npts, const uint64_t* pts, uint64_t* out);

  zr_ctx* ctx_;
  cudaStream_t st_;
  cudaStream_t pst_ = nullptr;        // probe lane (see set_probe_lane)
  int plane_ = -1;
  cudaEvent_t pev_in_ = nullptr, pev_out_ = nullptr;
  Mod M_;
  // request
  int nv_;
  bool rational_;
  bool callback_ = false;       // the black box is the caller's function
  zr_eval_fn eval_ = nullptr;
  void* user_ = nullptr;
  std::vector<uint8_t> Ne_, De_;
  std::vector<uint64_t> Nc_, Dc_;
  std::vector<int32_t> degN_, degD_;
  std::vector<char> autoN_, autoD_;   // degree of the variable unknown: detected
  bool verify_ = false;
  int maxed_fails_ = 0;
  uint64_t seed_;
  int offset_;
  // state
  Phase phase_ = NEW;
  zr_status err_ = ZR_OK;
  std::vector<uint64_t> z_, y_, cs_;
  int k_ = 1, attempt_ = 0, steps_ = 0, redraws_ = 0;
  DPoly fN_, fD_, curN_, curD_, nextN_, nextD_;
  DBuf d_y_, d_cs_, d_z_, d_b_, d_pts_, d_vals_, scratch_, persist_, fv_, one_, ones_, d_ppts_, d_vpt_, d_vval_;
  zr_result* result_ = nullptr;
};

}  // namespace zr
