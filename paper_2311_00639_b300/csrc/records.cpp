// Complex64 term records: the per-pass order and packed form in which the H psi
// kernel reads the Pauli strings of one block (TermF, internal.h).  Host code
// only; capi.cu uploads the result and syk_plan_host returns it for checks.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <tuple>

#include "internal.h"

namespace syk {

int64_t build_records(const std::vector<BlockString>& terms, const std::vector<PassPlan>& passes,
                      std::vector<TermF> rec[2], int64_t* n_merges) {
  const size_t n = terms.size();
  // Within each pass, the terms that read the same input tile (equal
  // x >> kTileBits) are made adjacent and flagged as a run.
  std::vector<size_t> rec_order(n);
  std::iota(rec_order.begin(), rec_order.end(), size_t(0));
  auto rec_key = [&](size_t i) {
    const auto& t = terms[i];
    return std::make_tuple(t.x >> kTileBits, 4 * int(t.imag) + 2 * int(t.x & 1u) + int(t.z & 1u), t.x, t.z);
  };
  for (const auto& ps : passes)
    std::stable_sort(rec_order.begin() + ps.t0, rec_order.begin() + ps.t1,
                     [&](size_t a, size_t b) { return rec_key(a) < rec_key(b); });
  std::vector<char> pass_end(n + 1, 0);
  for (const auto& ps : passes) pass_end[ps.t1] = 1;
  for (int b = 0; b < 2; ++b) rec[b].assign(n + 1, TermF{0, 0, 0.0f, 0});  // + one zero record: prefetch past the end
  // merge groups: maximal stretches of a pass with equal x and class
  // (adjacent under rec_key), split into groups of at most kTermGroupMax + 1
  // records; merge = the next record is in the same group, glen = records
  // after a group's first one
  std::vector<char> same_next(n, 0);
  for (size_t k = 0; k + 1 < n; ++k) {
    const auto& a = terms[rec_order[k]];
    const auto& b = terms[rec_order[k + 1]];
    same_next[k] = !pass_end[k + 1] && a.x == b.x && a.imag == b.imag && ((a.z ^ b.z) & 1u) == 0;
  }
  std::vector<uint32_t> glen(n, 0);
  std::vector<char> merge_next(n, 0);
  for (size_t k = 0; k < n;) {
    size_t e = k;
    while (e + 1 < n && same_next[e]) ++e;  // [k, e] is one stretch
    for (size_t a = k; a <= e; a += kTermGroupMax + 1) {
      const size_t b = std::min(e, a + kTermGroupMax);
      glen[a] = static_cast<uint32_t>(b - a);
      for (size_t i = a; i < b; ++i) merge_next[i] = 1;
    }
    k = e + 1;
  }
  int64_t n_runs = 0, merges = 0;
  for (size_t k = 0; k < n; ++k) {
    const auto& t = terms[rec_order[k]];
    const uint32_t hi = t.x >> kTileBits;
    const bool start = k == 0 || pass_end[k] || (terms[rec_order[k - 1]].x >> kTileBits) != hi;
    const bool end = k + 1 == n || pass_end[k + 1] || (terms[rec_order[k + 1]].x >> kTileBits) != hi;
    const bool merge = merge_next[k];
    n_runs += start ? 1 : 0;
    merges += merge ? 1 : 0;
    for (int b = 0; b < 2; ++b) {
      TermF& r = rec[b][k];
      r.x = t.x | (((t.z >> 7) & 1u) << 31);  // z bit 7 (row sign pattern, see TermF)
      r.z = t.z | (((t.z >> 8) & 1u) << 31);  // z bit 8
      r.c = static_cast<float>(t.coef[b]);
      r.flags = (t.straggler ? kTermStraggler : 0u) | (start ? kTermRunStart : 0u) | (end ? kTermRunEnd : 0u) |
                (merge ? kTermMerge : 0u) | (glen[k] << kTermGroupShift) |
                (t.imag ? kTermImag : 0u) | (term_body(t.x, t.z, t.imag) << kTermBodyShift) |
                (((t.z >> 6) & 1u) << 31);
    }
  }
  if (n_merges) *n_merges = merges;
  return n_runs;
}

PassPlan tail_pass(const PassPlan& last) {
  PassPlan tail = last;
  tail.t0 = tail.ti = tail.t1;
  for (int c = 0; c < 9; ++c) tail.cls[c] = tail.t1;
  return tail;
}

}  // namespace syk
