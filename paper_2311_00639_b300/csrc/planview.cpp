// Host views of the matvec pass plan and complex64 records (no CUDA call):
// what syk_terms_replan sets up for a compiled string list, written to a
// syk_plan_host_out.  Shared by syk_plan_host (Majorana quadruples) and
// syk_plan_strings_host (any compiled strings: Pauli-string chains, complex
// couplings).
#include <cmath>
#include <cstring>

#include "entry.h"
#include "kernels.cuh"

namespace syk {

void plan_view(std::vector<BlockString>&& terms, int L, int dtype, size_t l2_budget_bytes, double straggler_ratio,
               int n_sm, syk_plan_host_out* out) {
  SYK_REQUIRE(out != nullptr, "null output");
  SYK_REQUIRE(dtype == SYK_C64 || dtype == SYK_C128, "dtype must be SYK_C64 or SYK_C128");
  SYK_REQUIRE(l2_budget_bytes == 0 || l2_budget_bytes >= 4096, "l2_budget_bytes must be 0 or >= 4096");
  SYK_REQUIRE(std::isfinite(straggler_ratio) && straggler_ratio >= 0, "straggler_ratio must be >= 0");
  SYK_REQUIRE(n_sm >= 1, "n_sm must be >= 1");
  SYK_REQUIRE(out->term_capacity >= 0 && out->pass_capacity >= 0, "negative capacity");
  if (l2_budget_bytes == 0) {
    l2_budget_bytes = default_l2_budget(dtype);
    straggler_ratio = default_hbm_ratio(dtype);
  }
  syk_terms h;  // host fields only: nothing is allocated on a device
  h.L = L;
  h.D = int64_t(1) << L;
  h.dtype = dtype;
  h.n_sm = n_sm;
  h.terms = std::move(terms);
  h.passes = plan_passes(h.terms, h.L, elem_bytes(dtype), l2_budget_bytes, straggler_ratio);
  std::vector<TermF> rec[2];
  const size_t n = h.terms.size();
  out->n_runs = build_records(h.terms, h.passes, rec, &h.n_merges);
  out->n_merges = h.n_merges;
  plan_split(&h);
  out->n_terms = static_cast<int64_t>(n);
  out->n_passes = static_cast<int64_t>(h.passes.size());
  if (out->term_capacity < out->n_terms || out->pass_capacity < out->n_passes) return;
  for (size_t p = 0; p < h.passes.size() && out->passes; ++p) {
    const PassPlan& ps = h.passes[p];
    syk_pass_info& o = out->passes[p];
    o.t0 = ps.t0;
    o.ti = ps.ti;
    o.t1 = ps.t1;
    o.emask = ps.emask;
    for (int c = 0; c < 9; ++c) o.cls[c] = ps.cls[c];
    o.split_chunks = h.split_chunks[p];
    o.split_terms = h.split_terms[p];
    std::memcpy(o.dep, ps.dep, sizeof(o.dep));
  }
  for (size_t i = 0; i < n; ++i) {
    const auto& t = h.terms[i];
    if (out->x) out->x[i] = t.x;
    if (out->z) out->z[i] = t.z;
    if (out->coef_U) out->coef_U[i] = t.coef[0];
    if (out->coef_D) out->coef_D[i] = t.coef[1];
    if (out->imag) out->imag[i] = t.imag ? 1 : 0;
    if (out->straggler) out->straggler[i] = t.straggler ? 1 : 0;
  }
  if (out->records)
    for (int b = 0; b < 2; ++b)
      std::memcpy(out->records + static_cast<size_t>(b) * (n + 1) * 4, rec[b].data(), (n + 1) * sizeof(TermF));
}

}  // namespace syk

extern "C" int syk_plan_strings_host(int L, int64_t n, const uint32_t* x, const uint32_t* z, const double* coef_U,
                                     const double* coef_D, const uint8_t* imag, int dtype, size_t l2_budget_bytes,
                                     double straggler_ratio, int n_sm, syk_plan_host_out* out) {
  return syk::guard_call("syk_plan_strings_host", [&] {
    SYK_REQUIRE(L >= 1 && L <= 31, "L must be in [1, 31]");
    SYK_REQUIRE(n >= 0 && n <= (int64_t(1) << 31) - 1, "n out of range");
    SYK_REQUIRE(n == 0 || (x && z && coef_U && coef_D && imag), "null string array");
    const uint32_t lim = (1u << L) - 1u;
    std::vector<syk::BlockString> terms(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) {
      SYK_REQUIRE((x[i] & ~lim) == 0 && (z[i] & ~lim) == 0, "string acts on a bit >= L");
      SYK_REQUIRE(std::isfinite(coef_U[i]) && std::isfinite(coef_D[i]), "non-finite coefficient");
      terms[i].x = x[i];
      terms[i].z = z[i];
      terms[i].coef[0] = coef_U[i];
      terms[i].coef[1] = coef_D[i];
      terms[i].imag = imag[i] != 0;
    }
    syk::plan_view(std::move(terms), L, dtype, l2_budget_bytes, straggler_ratio, n_sm, out);
  });
}
