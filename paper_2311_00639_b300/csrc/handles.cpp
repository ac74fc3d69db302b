// Handle construction shared by the spin-chain and non-Hermitian entry points
// (declared in entry.h).
#include <algorithm>
#include <cmath>
#include <utility>

#include "entry.h"

namespace syk {

syk_terms_t* make_handle(int N_build, int dtype, int rep, std::vector<BlockString>&& terms, int64_t n_input,
                         int64_t n_real, int64_t n_xgroups, bool hermitian) {
  syk_terms_t* raw = nullptr;
  int rc = syk_build_terms(N_build, 0, nullptr, nullptr, dtype, rep, &raw);
  if (rc != SYK_OK) {
    char buf[512];
    syk_last_error(buf, sizeof buf);
    throw Error(rc, buf);
  }
  raw->terms = std::move(terms);
  raw->n_input = n_input;
  raw->n_real = n_real;
  raw->n_xgroups = n_xgroups;
  raw->hermitian = hermitian;
  raw->sum_abs = 0.0;
  for (const auto& t : raw->terms) raw->sum_abs += std::max(std::fabs(t.coef[0]), std::fabs(t.coef[1]));
  rc = syk_terms_replan(raw, 0, 0.0);
  if (rc != SYK_OK) {
    char buf[512];
    syk_last_error(buf, sizeof buf);
    syk_terms_destroy(raw);
    throw Error(rc, buf);
  }
  return raw;
}

}  // namespace syk
