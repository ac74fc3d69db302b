// Pass planner: groups the Pauli strings so that every group can be applied
// with an L2-resident working set.
//
// The matvec walks the block in tiles of 2^kTileBits consecutive amplitudes;
// a term with flip mask x reads, for output tile T, the input tile T ^ x_hi
// (x_hi = the bits of x above the tile).  If every term of a pass leaves a
// set E of high bits untouched, the amplitudes with one fixed value of the E
// bits (a "super-tile", 2^(L-|E|) amplitudes) only read from themselves.  The
// kernel visits tiles super-tile by super-tile, so each input super-tile is
// brought from HBM once per pass and then re-read from L2 by every term.
// |E| is the smallest size whose super-tile fits the L2 budget; passes are
// chosen greedily (random restarts + swap local search) to cover as many of
// the remaining terms as possible.  Terms that no admissible E can cover go
// to a final pass in plain order.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <tuple>

#include "internal.h"

namespace syk {
namespace {

struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

int count_covered(const std::vector<uint32_t>& hx, const std::vector<int>& rem, uint32_t emask) {
  int c = 0;
  for (int t : rem) c += (hx[t] & emask) == 0;
  return c;
}

void fill_tables(PassPlan& p, int nh, uint32_t emask) {
  int pos[32];
  int n = 0;
  for (int b = 0; b < nh; ++b)
    if (!((emask >> b) & 1)) pos[n++] = b;  // inner (fast-varying) bits first
  for (int b = 0; b < nh; ++b)
    if ((emask >> b) & 1) pos[n++] = b;  // then the excluded bits: one super-tile at a time
  for (int byte = 0; byte < 3; ++byte)
    for (int v = 0; v < 256; ++v) {
      uint32_t m = 0;
      for (int k = 0; k < 8; ++k) {
        const int j = 8 * byte + k;
        if (((v >> k) & 1) && j < nh) m |= 1u << (kTileBits + pos[j]);
      }
      p.dep[byte][v] = m;
    }
  p.emask = emask << kTileBits;
}

}  // namespace

std::vector<PassPlan> plan_passes(std::vector<BlockString>& terms, int L, size_t elem_bytes, size_t l2_budget,
                                   double hbm_ratio) {
  const int nh = std::max(0, L - kTileBits);
  const size_t vec_bytes = (size_t(1) << L) * elem_bytes;
  int e = 0;
  while (e < nh && (vec_bytes >> e) > l2_budget) ++e;
  std::vector<int> pass_of(terms.size(), 0);
  std::vector<uint32_t> emasks;
  if (e == 0) {
    emasks.push_back(0);
  } else {
    std::vector<uint32_t> hx(terms.size());
    for (size_t t = 0; t < terms.size(); ++t) hx[t] = terms[t].x >> kTileBits;
    std::vector<int> rem(terms.size());
    std::iota(rem.begin(), rem.end(), 0);
    SplitMix rng{0x5EED5EEDull};
    while (!rem.empty()) {
      uint32_t best = 0;
      int best_c = -1;
      for (int trial = 0; trial < 24; ++trial) {
        int bits[32];
        for (int b = 0; b < nh; ++b) bits[b] = b;
        for (int k = 0; k < e; ++k) std::swap(bits[k], bits[k + static_cast<int>(rng.next() % (nh - k))]);
        uint32_t m = 0;
        for (int k = 0; k < e; ++k) m |= 1u << bits[k];
        int c = count_covered(hx, rem, m);
        for (bool improved = true; improved;) {  // first-improvement swaps
          improved = false;
          for (int bi = 0; bi < nh && !improved; ++bi) {
            if (!((m >> bi) & 1)) continue;
            for (int bo = 0; bo < nh && !improved; ++bo) {
              if ((m >> bo) & 1) continue;
              const uint32_t m2 = (m & ~(1u << bi)) | (1u << bo);
              const int c2 = count_covered(hx, rem, m2);
              if (c2 > c) {
                m = m2;
                c = c2;
                improved = true;
              }
            }
          }
        }
        if (c > best_c) {
          best_c = c;
          best = m;
        }
      }
      const int p = static_cast<int>(emasks.size());
      if (best_c <= 0) {  // nothing coverable: one final pass in plain order
        emasks.push_back(0);
        for (int t : rem) pass_of[t] = p;
        rem.clear();
        break;
      }
      emasks.push_back(best);
      std::vector<int> left;
      for (int t : rem) {
        if ((hx[t] & best) == 0)
          pass_of[t] = p;
        else
          left.push_back(t);
      }
      rem.swap(left);
    }
  }
  // Dissolve light passes.  A pass costs about max(L2, HBM) where, in units
  // of one block vector moved at L2 bandwidth, L2 = (terms read from the
  // resident super-tile + terms read from outside it) and HBM = kHbmRatio x
  // (its own input and output streams + one vector per outside term).  A pass
  // with few terms is dominated by its fixed output read-modify-write; its
  // terms are cheaper as "stragglers" of an L2-bound pass, whose input tiles
  // they fetch from HBM while the pass's covered terms saturate L2.
  for (auto& t : terms) t.straggler = false;
  const int P = static_cast<int>(emasks.size());
  if (P > 1 && hbm_ratio > 0.0) {
    const double kHbmRatio = hbm_ratio;  // ~ L2 / HBM bandwidth (B300: ~17.5 / ~5.8 TB/s)
    std::vector<int> covered(P, 0), extra(P, 0);
    for (size_t t = 0; t < terms.size(); ++t) covered[pass_of[t]] += 1;
    auto cost = [&](int p, int cov, int ext) {
      const double fixed = (p == 0) ? 2.0 : 3.0;
      return std::max(static_cast<double>(cov + ext), kHbmRatio * (fixed + ext));
    };
    std::vector<int> alive(P, 1);
    for (;;) {
      // lightest live pass other than pass 0
      int victim = -1;
      for (int p = 1; p < P; ++p)
        if (alive[p] && (victim < 0 || covered[p] + extra[p] < covered[victim] + extra[victim])) victim = p;
      if (victim < 0) break;
      const int moving = covered[victim] + extra[victim];
      std::vector<int> add(P, 0);
      double delta = -cost(victim, covered[victim], extra[victim]);
      for (int m = 0; m < moving; ++m) {
        int best = -1;
        double best_inc = 0.0;
        for (int p = 0; p < P; ++p) {
          if (!alive[p] || p == victim) continue;
          const double inc = cost(p, covered[p], extra[p] + add[p] + 1) - cost(p, covered[p], extra[p] + add[p]);
          if (best < 0 || inc < best_inc) {
            best = p;
            best_inc = inc;
          }
        }
        add[best] += 1;
        delta += best_inc;
      }
      if (delta >= 0.0) break;
      // Commit: hand the victim's terms to the chosen passes in order.
      std::vector<int> targets;
      for (int p = 0; p < P; ++p)
        for (int a = 0; a < add[p]; ++a) targets.push_back(p);
      size_t next = 0;
      for (size_t t = 0; t < terms.size(); ++t)
        if (pass_of[t] == victim) {
          pass_of[t] = targets[next++];
          terms[t].straggler = true;
        }
      for (int p = 0; p < P; ++p) extra[p] += add[p];
      covered[victim] = extra[victim] = 0;
      alive[victim] = 0;
    }
    // Renumber the surviving passes.
    std::vector<int> newid(P, -1);
    std::vector<uint32_t> kept_masks;
    for (int p = 0; p < P; ++p)
      if (alive[p]) {
        newid[p] = static_cast<int>(kept_masks.size());
        kept_masks.push_back(emasks[p]);
      }
    for (auto& v : pass_of) v = newid[v];
    emasks.swap(kept_masks);
  }

  // Device order: by pass, then real before imaginary, then flip mask.
  std::vector<int> order(terms.size());
  std::iota(order.begin(), order.end(), 0);
  auto cls_of = [&](int t) { return 4 * int(terms[t].imag) + 2 * int(terms[t].x & 1u) + int(terms[t].z & 1u); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return std::make_tuple(pass_of[a], cls_of(a), terms[a].x, terms[a].z) <
           std::make_tuple(pass_of[b], cls_of(b), terms[b].x, terms[b].z);
  });
  std::vector<BlockString> sorted(terms.size());
  std::vector<int> sorted_pass(terms.size());
  for (size_t i = 0; i < order.size(); ++i) {
    sorted[i] = terms[order[i]];
    sorted_pass[i] = pass_of[order[i]];
  }
  terms.swap(sorted);
  std::vector<PassPlan> out(emasks.size());
  size_t i = 0;
  auto cls_sorted = [&](size_t t) {
    return 4 * int(terms[t].imag) + 2 * int(terms[t].x & 1u) + int(terms[t].z & 1u);
  };
  for (size_t p = 0; p < emasks.size(); ++p) {
    out[p].t0 = static_cast<int>(i);
    for (int c = 0; c < 8; ++c) {
      out[p].cls[c] = static_cast<int>(i);
      if (c == 4) out[p].ti = static_cast<int>(i);
      while (i < terms.size() && sorted_pass[i] == static_cast<int>(p) && cls_sorted(i) == c) ++i;
    }
    out[p].t1 = out[p].cls[8] = static_cast<int>(i);
    fill_tables(out[p], nh, emasks[p]);
  }
  // Drop empty passes (possible only when there are no terms at all); keep one.
  std::vector<PassPlan> kept;
  for (auto& p : out)
    if (p.t1 > p.t0 || kept.empty()) kept.push_back(p);
  if (kept.size() > 1 && kept[0].t1 == kept[0].t0) kept.erase(kept.begin());
  return kept;
}

}  // namespace syk
