// Term compiler: chi_i chi_j chi_k chi_l -> one Pauli string on a parity block.
//
// Supplement Sec. I.A represents a spin operator as a list of Pauli strings
// with coefficients; the product of two strings is the XOR of their flip
// patterns times a sign read off the pattern, and the sum of operators merges
// equal strings.  Here a string on q <= 32 qubits is kept as i^e X^x Z^z
// (Z^z acts first), for which
//   (i^a X^x1 Z^z1)(i^b X^x2 Z^z2) = i^{a+b} (-1)^{popc(z1 & x2)} X^{x1^x2} Z^{z1^z2}.
// Majoranas come from supplement Eq. (S1) (compact form, gamma_{N-1} =
// sigma_y on the block qubit) or from the Jordan-Wigner form; the block
// qubit is then folded away so the kernels act on L = N/2 - 1 bits.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <tuple>

#include "internal.h"

namespace syk {
namespace {

struct Pauli {
  uint64_t x = 0, z = 0;
  int e = 0;  // power of i
};

Pauli mul(const Pauli& a, const Pauli& b) {
  Pauli r;
  r.x = a.x ^ b.x;
  r.z = a.z ^ b.z;
  r.e = (a.e + b.e + 2 * (__builtin_popcountll(a.z & b.x) & 1)) & 3;
  return r;
}

Pauli site_op(int s, char op) {
  Pauli p;
  const uint64_t bit = 1ull << s;
  if (op == 'X') p.x = bit;
  if (op == 'Z') p.z = bit;
  if (op == 'Y') {  // Y = i X Z
    p.x = bit;
    p.z = bit;
    p.e = 1;
  }
  return p;
}

// gamma_n ({gamma, gamma} = 2 delta) as a Pauli string on N/2 qubits.
Pauli gamma_string(int N, int rep, int n) {
  const int L = N / 2 - 1;
  Pauli g;
  if (rep == SYK_REP_PAPER) {
    if (n == N - 1) return site_op(L, 'Y');  // UD = -i 1, DU = +i 1
    g = site_op(L, 'X');                     // UD = DU = A_n
    for (int s = (n + 1) / 2; s < L; ++s) g = mul(g, site_op(s, 'X'));
    if (n > 0) g = mul(g, site_op((n - 1) / 2, (n % 2) ? 'Y' : 'Z'));
  } else {
    const int s = n / 2;
    for (int r = 0; r < s; ++r) g = mul(g, site_op(r, 'Z'));
    g = mul(g, site_op(s, (n % 2) ? 'Y' : 'X'));
  }
  return g;
}

int popc(uint64_t v) { return __builtin_popcountll(v); }

}  // namespace

// Fold the block qubit (bit L) of a full string into the block form.
// Acting on block P at block index n, the full basis state has block bit
// b = P (paper rep) or b = parity(n) ^ P (JW rep), so
//   i^e X^x Z^z |b, n> = i^e (-1)^{z_top b} (-1)^{popc(z_low & n)} |b ^ x_top, n ^ x_low>.
// With zeff = z_low (paper) or z_low ^ (z_top ? all : 0) (JW) the sign is
// (-1)^{z_top P} (-1)^{popc(zeff & n)}, and in output-index form
// (-1)^{popc(zeff & m)} (-1)^{popc(zeff & x_low)} with m = n ^ x_low.
static void fold_block(int N, int rep, const Pauli& p, uint32_t& x_low, uint32_t& zeff, int& z_top) {
  const int L = N / 2 - 1;
  const uint64_t lmask = (L == 64) ? ~0ull : ((1ull << L) - 1);
  x_low = static_cast<uint32_t>(p.x & lmask);
  z_top = static_cast<int>((p.z >> L) & 1);
  uint64_t zl = p.z & lmask;
  if (rep == SYK_REP_JW && z_top) zl ^= lmask;
  zeff = static_cast<uint32_t>(zl);
}

void compile_terms(int N, int rep, int64_t T, const int32_t* quads, const double* J,
                   std::vector<BlockString>& out, int64_t& n_real, int64_t& n_xgroups) {
  const int L = N / 2 - 1;
  Pauli gam[64];
  for (int n = 0; n < N; ++n) gam[n] = gamma_string(N, rep, n);
  std::map<std::tuple<uint32_t, uint32_t, int>, size_t> index;
  out.clear();
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* q = quads + 4 * t;
    for (int k = 0; k < 4; ++k)
      SYK_REQUIRE(q[k] >= 0 && q[k] < N, "quad index out of range [0, N)");
    SYK_REQUIRE(q[0] < q[1] && q[1] < q[2] && q[2] < q[3], "quad indices must be strictly increasing");
    SYK_REQUIRE(std::isfinite(J[t]), "non-finite coupling");
    Pauli p = mul(mul(gam[q[0]], gam[q[1]]), mul(gam[q[2]], gam[q[3]]));
    const uint64_t top = 1ull << L;
    if (rep == SYK_REP_PAPER) {
      SYK_REQUIRE((p.x & top) == 0, "internal: term leaves the parity block");
    } else {
      SYK_REQUIRE((popc(p.x) & 1) == 0, "internal: term changes parity");
    }
    uint32_t x, zeff;
    int z_top;
    fold_block(N, rep, p, x, zeff, z_top);
    // Hermitian string: e is odd exactly when popc(x & z) is odd; the block
    // form keeps this with zeff (popc(x_low & zeff) has the same parity).
    const bool imag = (p.e & 1) != 0;
    SYK_REQUIRE(((popc(static_cast<uint64_t>(x) & zeff) & 1) != 0) == imag,
                "internal: non-Hermitian term string");
    const double s_e = (p.e == 0 || p.e == 1) ? 1.0 : -1.0;  // i^e = s_e * (1 or i)
    const double s_fold = (popc(static_cast<uint64_t>(x) & zeff) & 1) ? -1.0 : 1.0;
    const double c = 0.25 * J[t] * s_e * s_fold;  // chi^4 = gamma^4 / 4
    const double cU = c;
    const double cD = z_top ? -c : c;
    auto key = std::make_tuple(x, zeff, static_cast<int>(imag));
    auto it = index.find(key);
    if (it == index.end()) {
      BlockString b;
      b.x = x;
      b.z = zeff;
      b.imag = imag;
      b.coef[0] = cU;
      b.coef[1] = cD;
      index.emplace(key, out.size());
      out.push_back(b);
    } else {
      out[it->second].coef[0] += cU;
      out[it->second].coef[1] += cD;
    }
  }
  out.erase(std::remove_if(out.begin(), out.end(),
                           [](const BlockString& b) { return b.coef[0] == 0.0 && b.coef[1] == 0.0; }),
            out.end());
  std::sort(out.begin(), out.end(), [](const BlockString& a, const BlockString& b) {
    return std::make_tuple(a.imag, a.x, a.z) < std::make_tuple(b.imag, b.x, b.z);
  });
  n_real = 0;
  std::set<uint32_t> xs;
  for (const auto& b : out) {
    n_real += b.imag ? 0 : 1;
    xs.insert(b.x);
  }
  n_xgroups = static_cast<int64_t>(xs.size());
}

void compile_terms_complex(int N, int rep, int64_t T, const int32_t* quads, const double* J_re, const double* J_im,
                           std::vector<BlockString>& out, int64_t& n_real, int64_t& n_xgroups) {
  const int L = N / 2 - 1;
  Pauli gam[64];
  for (int n = 0; n < N; ++n) gam[n] = gamma_string(N, rep, n);
  std::map<std::tuple<uint32_t, uint32_t, int>, size_t> index;
  out.clear();
  auto add = [&](uint32_t x, uint32_t z, bool imag, double cU, double cD) {
    if (cU == 0.0 && cD == 0.0) return;
    auto key = std::make_tuple(x, z, static_cast<int>(imag));
    auto it = index.find(key);
    if (it == index.end()) {
      BlockString b;
      b.x = x;
      b.z = z;
      b.imag = imag;
      b.coef[0] = cU;
      b.coef[1] = cD;
      index.emplace(key, out.size());
      out.push_back(b);
    } else {
      out[it->second].coef[0] += cU;
      out[it->second].coef[1] += cD;
    }
  };
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* q = quads + 4 * t;
    for (int k = 0; k < 4; ++k)
      SYK_REQUIRE(q[k] >= 0 && q[k] < N, "quad index out of range [0, N)");
    SYK_REQUIRE(q[0] < q[1] && q[1] < q[2] && q[2] < q[3], "quad indices must be strictly increasing");
    SYK_REQUIRE(std::isfinite(J_re[t]) && std::isfinite(J_im[t]), "non-finite coupling");
    Pauli p = mul(mul(gam[q[0]], gam[q[1]]), mul(gam[q[2]], gam[q[3]]));
    const uint64_t top = 1ull << L;
    if (rep == SYK_REP_PAPER) {
      SYK_REQUIRE((p.x & top) == 0, "internal: term leaves the parity block");
    } else {
      SYK_REQUIRE((popc(p.x) & 1) == 0, "internal: term changes parity");
    }
    uint32_t x, zeff;
    int z_top;
    fold_block(N, rep, p, x, zeff, z_top);
    // value of the string in block form: 0.25 (J_re + i J_im) s_e s_fold (i if e is odd)
    const bool odd = (p.e & 1) != 0;
    const double s_e = (p.e == 0 || p.e == 1) ? 1.0 : -1.0;
    const double s_fold = (popc(static_cast<uint64_t>(x) & zeff) & 1) ? -1.0 : 1.0;
    const double g = 0.25 * s_e * s_fold;
    const double v_re = odd ? -g * J_im[t] : g * J_re[t];  // (J_re + i J_im) * (odd ? i : 1)
    const double v_im = odd ? g * J_re[t] : g * J_im[t];
    const double sD = z_top ? -1.0 : 1.0;
    add(x, zeff, false, v_re, sD * v_re);
    add(x, zeff, true, v_im, sD * v_im);
  }
  out.erase(std::remove_if(out.begin(), out.end(),
                           [](const BlockString& b) { return b.coef[0] == 0.0 && b.coef[1] == 0.0; }),
            out.end());
  std::sort(out.begin(), out.end(), [](const BlockString& a, const BlockString& b) {
    return std::make_tuple(a.imag, a.x, a.z) < std::make_tuple(b.imag, b.x, b.z);
  });
  n_real = 0;
  std::set<uint32_t> xs;
  for (const auto& b : out) {
    n_real += b.imag ? 0 : 1;
    xs.insert(b.x);
  }
  n_xgroups = static_cast<int64_t>(xs.size());
}

ChiString compile_chi(int N, int rep, int n) {
  const Pauli g = gamma_string(N, rep, n);
  const int L = N / 2 - 1;
  const bool changes = (rep == SYK_REP_PAPER) ? (((g.x >> L) & 1) != 0) : ((popc(g.x) & 1) != 0);
  SYK_REQUIRE(changes, "internal: Majorana does not change the block");
  ChiString c;
  int z_top;
  fold_block(N, rep, g, c.x, c.z, z_top);
  const double s_fold = (popc(static_cast<uint64_t>(c.x) & c.z) & 1) ? -1.0 : 1.0;
  const double r = s_fold / std::sqrt(2.0);
  for (int P = 0; P < 2; ++P) {
    const double s = (z_top && P == 1) ? -r : r;
    // i^e * s
    const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
    c.re[P] = s * re[g.e];
    c.im[P] = s * im[g.e];
  }
  return c;
}

}  // namespace syk
