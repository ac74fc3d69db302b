// Shared by the extern "C" entry points that live outside capi.cu (spin
// chains, non-Hermitian SYK, host plan views): status mapping and handle
// construction from an already compiled list of block strings.
#pragma once

#include <new>
#include <string>
#include <vector>

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
