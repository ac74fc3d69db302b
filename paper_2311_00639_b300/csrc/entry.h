// Shared by the extern "C" entry points that live outside capi.cu (spin
// chains, non-Hermitian SYK, host plan views): status mapping and handle
// construction from an already compiled list of block strings.
#pragma once

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace syk {

// Runs f; maps a thrown syk::Error to its status and records "fn: message"
// for syk_last_error (no exception leaves an entry point).
template <typename F>
int guard_call(const char* fn, F&& f) {
  try {
    f();
    return SYK_OK;
  } catch (const Error& e) {
    set_last_error(std::string(fn) + ": " + e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error(std::string(fn) + ": host allocation failed");
    return SYK_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(std::string(fn) + ": " + e.what());
    return SYK_EINVAL;
  } catch (...) {
    set_last_error(std::string(fn) + ": unknown failure");
    return SYK_EINVAL;
  }
}

// Device memory owned for the duration of one call.
struct DeviceBuffer {
  void* p = nullptr;
  explicit DeviceBuffer(size_t n) {
    if (n && cudaMalloc(&p, n) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error(SYK_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed");
    }
  }
  ~DeviceBuffer() {
    if (p) cudaFree(p);
  }
  DeviceBuffer(const DeviceBuffer&) = delete;
  DeviceBuffer& operator=(const DeviceBuffer&) = delete;
};

// syk_krylov_params with the library defaults filled in (zero fields:
// m = 20 for complex64 / 30 for complex128, tol = 1e-6 / 1e-12, 1000
// substeps), validated.
struct KrylovSettings {
  int m;
  double tol;
  int max_sub;
  bool reorth, two_pass;
};
inline KrylovSettings krylov_settings(int dtype, const syk_krylov_params* p) {
  KrylovSettings k;
  k.m = (p && p->m) ? p->m : default_krylov_m(dtype);
  k.tol = (p && p->tol > 0) ? p->tol : (dtype == SYK_C128 ? 1e-12 : 1e-6);
  k.max_sub = (p && p->max_substeps) ? p->max_substeps : 1000;
  k.reorth = p && p->reorth;
  k.two_pass = p && p->two_pass;
  SYK_REQUIRE(k.m >= 1 && k.m <= kMaxKrylov, "Krylov dimension m must be in [1, 64]");
  SYK_REQUIRE(std::isfinite(k.tol) && k.tol > 0, "tol must be positive");
  SYK_REQUIRE(k.max_sub >= 1, "max_substeps must be >= 1");
  SYK_REQUIRE(!(k.reorth && k.two_pass), "reorth and two_pass cannot be combined");
  return k;
}

// A handle on the current device holding `terms`: syk_build_terms with no
// terms on N_build Majoranas in representation rep (device, Majorana
// strings, D = 2^{N_build/2 - 1}), then the strings, their counts and
// sum_t max_P |coef_P|, and syk_terms_replan with the dtype's default plan
// (pass plan, records, upload).  Throws syk::Error on failure.
syk_terms_t* make_handle(int N_build, int dtype, int rep, std::vector<BlockString>&& terms, int64_t n_input,
                         int64_t n_real, int64_t n_xgroups, bool hermitian);

// The pass plan, split and complex64 records syk_terms_replan would set up
// for `terms` on L index bits (l2_budget_bytes = 0: the dtype's default
// plan), written to `out` as syk_plan_host documents (planview.cpp).
void plan_view(std::vector<BlockString>&& terms, int L, int dtype, size_t l2_budget_bytes, double straggler_ratio,
               int n_sm, syk_plan_host_out* out);

}  // namespace syk
