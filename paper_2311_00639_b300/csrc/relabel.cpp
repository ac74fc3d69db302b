// syk_relabel_majoranas: a Jordan-Wigner ordering of the Majoranas chosen for
// the locality of the blocked H psi.
//
// In the Jordan-Wigner representation the Majoranas 2s and 2s+1 share qubit s,
// and a four-Majorana term flips the qubits that hold an odd number of its
// Majoranas.  Which physical Majorana sits on which qubit is a free choice: a
// relabelling of the Majoranas is an automorphism of the Clifford algebra,
// implemented on the state space by a unitary, so spectra and traces (the
// exact-trace OTOC of Eq. (2)) do not change.  The complex64 matvec stages one
// 2^tile_bits-amplitude input tile per distinct flip pattern above the tile
// bits (per pass) for every output tile, so the number of distinct patterns
// sets its L2 -> shared-memory traffic.  This search lowers it by simulated
// annealing over swaps of two Majoranas between qubits, with the objective
// updated incrementally (only the terms of the two swapped Majoranas change).
// Majoranas N-2 and N-1 keep the top qubit (the one the block index drops),
// so chi_{N-1} and chi_{N-2} stay diagonal between the parity blocks.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "entry.h"

namespace {

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" int syk_relabel_majoranas(int N, int64_t T, const int32_t* quads, const double* J, int tile_bits,
                                     int64_t iterations, uint64_t seed, int32_t* perm, int32_t* quads_out,
                                     double* J_out, int64_t* patterns_before, int64_t* patterns_after) {
  return syk::guard_call("syk_relabel_majoranas", [&] {
    SYK_REQUIRE(N >= 6 && N <= 64 && N % 2 == 0, "N must be even and in [6, 64]");
    SYK_REQUIRE(T >= 0 && (T == 0 || (quads && J)), "bad T or null quads/J");
    SYK_REQUIRE(perm != nullptr, "null perm");
    SYK_REQUIRE(tile_bits >= 0 && tile_bits <= 31, "tile_bits must be in [0, 31]");
    SYK_REQUIRE(iterations >= 0, "iterations must be >= 0");
    const int L = N / 2 - 1;  // block index bits; qubit L is the dropped top qubit
    for (int64_t t = 0; t < T; ++t)
      for (int c = 0; c < 4; ++c) {
        SYK_REQUIRE(quads[4 * t + c] >= 0 && quads[4 * t + c] < N, "quad index out of range");
        if (c) SYK_REQUIRE(quads[4 * t + c] > quads[4 * t + c - 1], "quads must be strictly increasing");
      }
    std::vector<int> qubit(N);  // qubit of each physical Majorana
    for (int m = 0; m < N; ++m) qubit[m] = m / 2;
    std::vector<std::vector<int64_t>> terms_of(N);
    for (int64_t t = 0; t < T; ++t)
      for (int c = 0; c < 4; ++c) terms_of[quads[4 * t + c]].push_back(t);
    auto bit = [&](int q) -> uint64_t { return q < L ? (uint64_t(1) << q) : 0u; };
    auto pattern = [&](uint64_t x) { return x >> tile_bits; };
    std::vector<uint64_t> x(static_cast<size_t>(T), 0);
    for (int64_t t = 0; t < T; ++t)
      for (int c = 0; c < 4; ++c) x[static_cast<size_t>(t)] ^= bit(qubit[quads[4 * t + c]]);
    std::unordered_map<uint64_t, int> count;  // patterns with a zero count stay in the map
    for (int64_t t = 0; t < T; ++t) ++count[pattern(x[static_cast<size_t>(t)])];
    int64_t distinct = static_cast<int64_t>(count.size());
    if (patterns_before) *patterns_before = distinct;
    std::vector<int> best_qubit = qubit;
    int64_t best = distinct;
    std::vector<int> free_m;
    for (int m = 0; m < N - 2; ++m) free_m.push_back(m);
    uint64_t rs = seed ^ 0x5DEECE66Dull;
    std::vector<int64_t> touched;
    std::vector<uint64_t> newx;
    for (int64_t it = 0; it < iterations && T > 0; ++it) {
      const int a = free_m[splitmix64(rs) % free_m.size()];
      const int b = free_m[splitmix64(rs) % free_m.size()];
      if (qubit[a] == qubit[b]) continue;
      const uint64_t flip = bit(qubit[a]) ^ bit(qubit[b]);
      // terms holding exactly one of a, b change their flip mask by `flip`
      touched.clear();
      for (int64_t t : terms_of[a]) touched.push_back(t);
      for (int64_t t : terms_of[b]) touched.push_back(t);
      std::sort(touched.begin(), touched.end());
      int64_t delta = 0;
      newx.assign(touched.size(), 0);
      size_t w = 0;
      for (size_t i = 0; i < touched.size(); ++i) {
        if (i + 1 < touched.size() && touched[i + 1] == touched[i]) {  // holds both: unchanged
          ++i;
          continue;
        }
        touched[w++] = touched[i];
      }
      touched.resize(w);
      for (size_t i = 0; i < touched.size(); ++i) {
        const uint64_t xo = x[static_cast<size_t>(touched[i])];
        if (--count[pattern(xo)] == 0) --delta;
      }
      for (size_t i = 0; i < touched.size(); ++i) {
        const uint64_t xn = x[static_cast<size_t>(touched[i])] ^ flip;
        newx[i] = xn;
        if (count[pattern(xn)]++ == 0) ++delta;
      }
      const double temp = std::max(0.05, 2.0 * (1.0 - static_cast<double>(it) / static_cast<double>(iterations)));
      const double u = static_cast<double>(splitmix64(rs) >> 11) * 0x1.0p-53;
      if (delta <= 0 || u < std::exp(-static_cast<double>(delta) / temp)) {
        for (size_t i = 0; i < touched.size(); ++i) x[static_cast<size_t>(touched[i])] = newx[i];
        std::swap(qubit[a], qubit[b]);
        distinct += delta;
        if (distinct < best) {
          best = distinct;
          best_qubit = qubit;
        }
      } else {  // undo the counts
        for (size_t i = 0; i < touched.size(); ++i) --count[pattern(newx[i])];
        for (size_t i = 0; i < touched.size(); ++i) ++count[pattern(x[static_cast<size_t>(touched[i])])];
      }
    }
    if (patterns_after) *patterns_after = best;
    // Jordan-Wigner index: qubit s holds indices 2s, 2s+1, given to its two
    // Majoranas in increasing physical order
    std::vector<int> seen(N / 2, 0);
    for (int m = 0; m < N; ++m) perm[m] = 2 * best_qubit[m] + seen[best_qubit[m]]++;
    if (quads_out || J_out) {
      for (int64_t t = 0; t < T; ++t) {
        int32_t v[4];
        for (int c = 0; c < 4; ++c) v[c] = perm[quads[4 * t + c]];
        int inversions = 0;
        for (int i = 0; i < 4; ++i)
          for (int j = i + 1; j < 4; ++j) inversions += v[i] > v[j] ? 1 : 0;
        std::sort(v, v + 4);  // chi_v0 chi_v1 chi_v2 chi_v3 = (-1)^inversions x the product in the old order
        if (quads_out)
          for (int c = 0; c < 4; ++c) quads_out[4 * t + c] = v[c];
        if (J_out) J_out[t] = (inversions & 1) ? -J[t] : J[t];
      }
    }
  });
}
