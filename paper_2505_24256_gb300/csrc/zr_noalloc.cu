// zr_noalloc.cu -- batched Newton interpolation that allocates nothing.
//
// Some callers cannot allocate device memory.  A host program that hands all
// of the GPU's memory to its own pool before it loads this library leaves
// nothing for cudaMalloc (or must not have a second allocator compete with
// its pool), and code on a latency-critical path cannot accept the implicit
// device-wide synchronisation that cudaMalloc and cudaFree may perform.
// Such callers cannot create a zr_ctx either, because a context allocates its
// status words and workspace.
//
// zr_newton_batched_noalloc serves them: it needs no context, and the one
// piece of scratch the Newton kernels use -- the table of inverse node
// differences 1/(x_s - x_{s-l}) shared by all columns, plus a status word --
// lives in the fixed array below.  The caller still passes the inputs and the
// output.  Limits and rules:
//   * at most kNoAllocMaxPts = 64 nodes per call (larger npts is rejected with
//     ZR_ERR_INVALID_ARG); the array is 64*64 + 32 words (about 33 KB), and
//     every GPU that loads the library holds it until the process exits;
//   * the first call on a device looks the array up with that device current
//     (cudaGetSymbolAddress) and caches the address; make that first call
//     before any stream capture;
//   * every call shares the array and it keeps the previous call's contents:
//     the status word is cleared at the start of each call and the table is
//     rewritten for the entries the call reads.  Calls that overlap on the GPU
//     (other streams, other host threads) race on it: serialise them;
//   * a CUDA error already pending on the calling thread (left by an earlier,
//     unrelated runtime call) is not this call's: the call then returns
//     ZR_ERR_CUDA at once and leaves that error pending for its owner, so that
//     an error reported after the launches is always one of this call's.
#include <cuda_runtime.h>

#include <mutex>

#include "zr_internal.h"

namespace {

constexpr int kNoAllocMaxPts = 64;
constexpr size_t kStatusWord = (size_t)kNoAllocMaxPts * kNoAllocMaxPts;    // index of the status word
constexpr size_t kScratchWords = kStatusWord + 32;

// The scratch array.  In host code its name is only a stand-in: kernels get
// the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) uint64_t g_newton_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device).
zr_status scratch_address(uint64_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return ZR_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return ZR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_newton_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();   // this call's own error: do not leave it pending
      return ZR_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return ZR_OK;
}

}  // namespace

extern "C" zr_status zr_newton_batched_noalloc(uint64_t prime, int64_t nterms, int32_t npts, const uint64_t* x,
                                               const uint64_t* vals, int64_t ld, uint64_t* coef, void* stream) {
  zr::Mod M;
  if (!zr::mod_for_prime(prime, &M)) return ZR_ERR_INVALID_ARG;
  if (npts < 1 || npts > kNoAllocMaxPts || nterms < 0 || ld < nterms || !x || (nterms > 0 && (!vals || !coef)))
    return ZR_ERR_INVALID_ARG;
  // someone else's pending error: report it without taking it
  if (cudaPeekAtLastError() != cudaSuccess) return ZR_ERR_CUDA;
  uint64_t* scratch = nullptr;
  zr_status r = scratch_address(&scratch);
  if (r != ZR_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t* invd = scratch;
  uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kStatusWord);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) {
    zr::launch_newton_table(npts, x, M, invd, status, st);
    e = cudaGetLastError();   // nothing was pending at entry: an error here is this call's
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ZR_ERR_CUDA;
  }
  zr::launch_newton(nterms, npts, invd, vals, ld, M, coef, st);
  uint32_t flags = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ZR_ERR_CUDA;
  }
  if (flags & zr::ST_DUP_SAMPLE) return ZR_ERR_SINGULAR;
  return flags ? ZR_ERR_CUDA : ZR_OK;
}
