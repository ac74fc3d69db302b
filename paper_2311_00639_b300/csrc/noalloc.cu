// syk_krylov_evolve_noalloc: the Krylov propagation of syk_krylov_evolve
// with its workspace taken from a fixed device array that lives in this
// library, so the call itself allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc (or have the library do
// it) while they run, for instance a host program that embeds this library
// under another framework's memory pool which already owns the device memory,
// or a service that must not allocate after start-up so that its memory
// footprint stays fixed.  They still pass x and y; only the Krylov basis,
// the reduction partials and the device scalars come from the array below.
//
// Limits and sharing rules (also stated in include/syk.h):
//   * the array holds kScratchBytes (16 MiB) on every GPU where the entry
//     point has been called, until the process exits;
//   * a call whose workspace (syk_krylov_workspace_bytes) is larger is
//     rejected with SYK_EINVAL before any work is queued;
//   * every call on a device uses the same array and leaves its contents
//     behind; calls that overlap on the GPU (different streams, or host
//     threads racing) corrupt each other, so serialise them;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current).  CUDA
//     loads this library's device code lazily, so that lookup is also when the
//     16 MiB are reserved on the device: the first call does take device
//     memory.  Callers that must not allocate later make one warm-up call at
//     start-up, before any stream capture: a call with tau = t = 0 reserves
//     the array (it only copies x to y); a real evolve also loads the kernels
//     the later calls run.  Later calls allocate nothing;
//   * the cached address belongs to the device context that was current at the
//     first call; after cudaDeviceReset (or the primary context being released
//     and created again) it is stale, like every handle of this library, so
//     the library must not be used across a context reset.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "entry.h"
#include "kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 128;

// Device-side workspace shared by all calls on a device.  In host code this
// name is only a handle for cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

void* scratch_address(int dev) {
  SYK_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw syk::Error(SYK_ECUDA, std::string("cudaGetSymbolAddress of the static workspace failed: ") +
                                      cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int syk_krylov_evolve_noalloc(const syk_terms_t* h, int block, double tau, double t, const void* x,
                                         void* y, int64_t nstates, const syk_krylov_params* p,
                                         syk_krylov_stats* stats, syk_stream_t stream) {
  try {
    SYK_REQUIRE(h != nullptr, "null terms handle");
    int dev = -1;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_REQUIRE(dev == h->device, "the current CUDA device is not the one the terms were built on");
    SYK_REQUIRE(block == 0 || block == 1, "block must be SYK_BLOCK_U or SYK_BLOCK_D");
    SYK_REQUIRE(std::isfinite(tau) && std::isfinite(t), "tau and t must be finite");
    SYK_REQUIRE(nstates >= 1, "nstates must be >= 1");
    SYK_REQUIRE(x && y, "null x or y");
    SYK_REQUIRE(((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0,
                "x and y must be 16-byte aligned");
    // the same defaults and checks as syk_krylov_evolve
    const syk::KrylovSettings ks = syk::krylov_settings(h->dtype, p);
    const int m = ks.m;
    const double tol = ks.tol;
    const int max_sub = ks.max_sub;
    const bool reorth = ks.reorth, two_pass = ks.two_pass;
    const size_t need = syk::krylov_ws_bytes(h, m, two_pass);
    if (need > kScratchBytes)
      throw syk::Error(SYK_EINVAL, "needs " + std::to_string(need) + " bytes of workspace; the static workspace of "
                                       "syk_krylov_evolve_noalloc holds " + std::to_string(kScratchBytes) +
                                       " bytes (use syk_krylov_evolve with your own workspace)");
    const size_t vb = static_cast<size_t>(h->D) * syk::elem_bytes(h->dtype);
    const char* xs = static_cast<const char*>(x);
    const char* ys = static_cast<const char*>(y);
    SYK_REQUIRE(x == y || xs + nstates * vb <= ys || ys + nstates * vb <= xs,
                "y must either equal x or not overlap it");
    void* ws = scratch_address(dev);
    auto st = reinterpret_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents; start the device scalars
    // from zero (everything else is written before it is read).
    SYK_CUDA(cudaMemsetAsync(ws, 0, sizeof(syk::KScalars), st));
    syk::KrylovResult tot;
    for (int64_t s = 0; s < nstates; ++s) {
      auto r = syk::krylov_evolve_one(h, block, tau, t, xs + s * vb, static_cast<char*>(y) + s * vb, m, tol, max_sub,
                                      reorth, two_pass, ws, st);
      tot.matvecs += r.matvecs;
      tot.substeps += r.substeps;
      tot.err += r.err;
    }
    syk::krylov_totals_collect(ws, st, tot);  // one synchronisation for the whole call
    if (stats) {
      stats->matvecs = tot.matvecs;
      stats->substeps = tot.substeps;
      stats->err_est = tot.err;
    }
    return SYK_OK;
  } catch (const syk::Error& e) {
    syk::set_last_error(std::string("syk_krylov_evolve_noalloc: ") + e.what());
    return e.code;
  } catch (const std::exception& e) {
    syk::set_last_error(std::string("syk_krylov_evolve_noalloc: ") + e.what());
    return SYK_EINVAL;
  }
}
