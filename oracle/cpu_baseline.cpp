// Plain FP64 CPU baseline of the hot path: matrix-free H psi (Algorithm 1 of
// the supplement, Sec. I.A, on one parity block) and Lanczos propagation
// e^{-zH} x, parallelised over rows with OpenMP.  TEST INFRASTRUCTURE ONLY:
// the timed CPU baseline of the benchmark (the paper's CPU path is OpenMP,
// supplement Sec. I.A) and a cross-check of the Python oracle.  It shares no
// code with the CUDA library; nothing in the product links it.
//
// Conventions (Jordan-Wigner, full space of q = N/2 qubits, qubit s = bit s):
//   gamma_{2s}   = Z_0 ... Z_{s-1} X_s,
//   gamma_{2s+1} = Z_0 ... Z_{s-1} Y_s,   Y = i X Z on one site,
//   chi = gamma / sqrt(2).  An operator ph * X^x Z^z acts as
//   X^x Z^z |f> = (-1)^{popc(z & f)} |f ^ x>, and products follow
//   (X^a Z^b)(X^c Z^d) = (-1)^{popc(b & c)} X^{a^c} Z^{b^d}.
//   H = sum_t J_t chi_i chi_j chi_k chi_l (Eq. (1) of the main text).
//   Block U holds the full indices of even popcount, D of odd popcount; a
//   block index m drops the top qubit q-1.
// Written for plainness: one output row per loop iteration, every term in
// turn, no blocking or vector intrinsics.
#include <omp.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

using cplx = std::complex<double>;

struct PauliTerm {
  uint64_t x = 0, z = 0;
  cplx c;  // coefficient of X^x Z^z
};

int popc(uint64_t v) { return __builtin_popcountll(v); }

// chi_n as ph * X^x Z^z.
PauliTerm majorana(int n) {
  const int s = n / 2;
  PauliTerm p;
  p.x = uint64_t(1) << s;
  p.z = (uint64_t(1) << s) - 1;
  p.c = cplx(1.0 / std::sqrt(2.0), 0.0);
  if (n % 2) {  // Y_s = i X_s Z_s
    p.z |= uint64_t(1) << s;
    p.c *= cplx(0.0, 1.0);
  }
  return p;
}

PauliTerm product(const PauliTerm& a, const PauliTerm& b) {
  PauliTerm r;
  r.x = a.x ^ b.x;
  r.z = a.z ^ b.z;
  r.c = a.c * b.c * ((popc(a.z & b.x) & 1) ? -1.0 : 1.0);
  return r;
}

std::vector<PauliTerm> compile(int N, int64_t T, const int32_t* quads, const double* J) {
  std::vector<PauliTerm> out(static_cast<size_t>(T));
  for (int64_t t = 0; t < T; ++t) {
    PauliTerm p = majorana(quads[4 * t]);
    for (int k = 1; k < 4; ++k) p = product(p, majorana(quads[4 * t + k]));
    p.c *= J[t];
    out[static_cast<size_t>(t)] = p;
  }
  (void)N;
  return out;
}

// Full index of block index m of block B (0 = U even, 1 = D odd).
inline uint64_t full_index(uint64_t m, int L, int B) {
  const uint64_t top = static_cast<uint64_t>((popc(m) + B) & 1);
  return m | (top << L);
}

// out[r] = (H_BB psi)[row0 + r] for r < nrows.  in(t, m_in) gives psi at
// block index m_in for term t.
template <typename In>
void hpsi_rows(const std::vector<PauliTerm>& terms, int L, int B, uint64_t row0, int64_t nrows, In in, cplx* out) {
  const uint64_t Dm = (uint64_t(1) << L) - 1;
  const int64_t T = static_cast<int64_t>(terms.size());
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    const uint64_t fo = full_index(row0 + static_cast<uint64_t>(r), L, B);
    cplx acc(0.0, 0.0);
    for (int64_t t = 0; t < T; ++t) {
      const uint64_t f = fo ^ terms[static_cast<size_t>(t)].x;
      const double s = (popc(terms[static_cast<size_t>(t)].z & f) & 1) ? -1.0 : 1.0;
      acc += s * terms[static_cast<size_t>(t)].c * in(t, f & Dm);
    }
    out[r] = acc;
  }
}

void hpsi_full(const std::vector<PauliTerm>& terms, int L, int B, const cplx* psi, cplx* out) {
  hpsi_rows(terms, L, B, 0, int64_t(1) << L, [psi](int64_t, uint64_t m) { return psi[m]; }, out);
}

double norm2(const cplx* v, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += std::norm(v[i]);
  return s;
}

// Eigenvalues / eigenvectors of a real symmetric n x n matrix A (row-major,
// overwritten) by cyclic Jacobi rotations; Q receives the eigenvectors as
// columns.
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& Q) {
  Q.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) Q[static_cast<size_t>(i) * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[static_cast<size_t>(i) * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? tot : off) += a(i, j) * a(i, j);
    if (off <= 1e-30 * (tot + off) || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (a(p, q) == 0.0) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * a(p, q));
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A G
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- G^T A
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double& qp = Q[static_cast<size_t>(k) * n + p];
          double& qq = Q[static_cast<size_t>(k) * n + q];
          const double kp = qp, kq = qq;
          qp = c * kp - s * kq;
          qq = s * kp + c * kq;
        }
      }
  }
}

}  // namespace

extern "C" {

int cpu_threads(void) { return omp_get_max_threads(); }

// out = H_BB psi on the whole block (psi, out: interleaved complex128 [D]).
int cpu_hpsi(int N, int64_t T, const int32_t* quads, const double* J, int block, const double* psi, double* out) {
  if (N < 4 || N > 64 || N % 2 || (block != 0 && block != 1)) return -1;
  const auto terms = compile(N, T, quads, J);
  hpsi_full(terms, N / 2 - 1, block, reinterpret_cast<const cplx*>(psi), reinterpret_cast<cplx*>(out));
  return 0;
}

// Rows [row0, row0 + R) of H_BB psi, R = 2^log2R and row0 a multiple of R, for
// blocks too large to hold: term t reads psi only inside the aligned range of
// R amplitudes starting at (row0 ^ x_t) & ~(R - 1), passed as in_blocks[t]
// (interleaved complex128 [R]).  block_start[t] receives that start (call
// first with in_blocks = NULL to get the starts).
int cpu_hpsi_rows(int N, int64_t T, const int32_t* quads, const double* J, int block, uint64_t row0, int log2R,
                  const double* const* in_blocks, uint64_t* block_start, double* out) {
  const int L = N / 2 - 1;
  if (N < 4 || N > 64 || N % 2 || (block != 0 && block != 1) || log2R < 0 || log2R > L) return -1;
  const uint64_t R = uint64_t(1) << log2R;
  if (row0 & (R - 1)) return -1;
  const auto terms = compile(N, T, quads, J);
  const uint64_t Dm = (uint64_t(1) << L) - 1;
  for (int64_t t = 0; t < T; ++t)
    if (block_start) block_start[t] = (row0 ^ terms[static_cast<size_t>(t)].x) & Dm & ~(R - 1);
  if (!in_blocks) return 0;
  const cplx* const* ib = reinterpret_cast<const cplx* const*>(in_blocks);
  hpsi_rows(terms, L, block, row0, static_cast<int64_t>(R),
            [ib, R](int64_t t, uint64_t m) { return ib[t][m & (R - 1)]; }, reinterpret_cast<cplx*>(out));
  return 0;
}

// y = e^{-(tau + i t) H_BB} x (interleaved complex128 [D]; y may alias x) by
// Lanczos with m steps per substep, the projected exponential from a Jacobi
// eigendecomposition of the tridiagonal matrix, and substep halving until the
// estimate beta_m |e_m^T e^{-sZT} e_1| is at most tol * s.  Returns the number
// of matvecs, or -1 on bad arguments, -3 if no substep was accepted.
int64_t cpu_krylov_evolve(int N, int64_t T, const int32_t* quads, const double* J, int block, double tau, double t,
                          int m, double tol, const double* x, double* y) {
  const int L = N / 2 - 1;
  if (N < 4 || N > 64 || N % 2 || (block != 0 && block != 1) || m < 1 || m > 128) return -1;
  const auto terms = compile(N, T, quads, J);
  const int64_t D = int64_t(1) << L;
  m = static_cast<int>(std::min<int64_t>(m, D));
  std::vector<cplx> V(static_cast<size_t>(m + 1) * D), w(static_cast<size_t>(D));
  cplx* out = reinterpret_cast<cplx*>(y);
  if (out != reinterpret_cast<const cplx*>(x)) std::memcpy(out, x, sizeof(cplx) * D);
  cplx zrem(tau, t);
  int64_t matvecs = 0;
  for (int sub = 0; sub < 100000 && (zrem.real() != 0.0 || zrem.imag() != 0.0); ++sub) {
    const double beta0 = std::sqrt(norm2(out, D));
    if (beta0 == 0.0) break;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; ++i) V[i] = out[i] / beta0;
    std::vector<double> alpha, beta;
    int n = 0;
    for (int j = 0; j < m; ++j) {
      cplx* vj = &V[static_cast<size_t>(j) * D];
      hpsi_full(terms, L, block, vj, w.data());
      ++matvecs;
      if (j > 0) {
        const cplx* vp = &V[static_cast<size_t>(j - 1) * D];
        const double b = beta[j - 1];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < D; ++i) w[i] -= b * vp[i];
      }
      double a = 0.0;
#pragma omp parallel for reduction(+ : a) schedule(static)
      for (int64_t i = 0; i < D; ++i) a += (std::conj(vj[i]) * w[i]).real();
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < D; ++i) w[i] -= a * vj[i];
      const double b = std::sqrt(norm2(w.data(), D));
      alpha.push_back(a);
      beta.push_back(b);
      n = j + 1;
      if (b <= 1e-14 * (std::fabs(a) + 1e-300)) break;  // invariant subspace
      cplx* vn = &V[static_cast<size_t>(j + 1) * D];
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < D; ++i) vn[i] = w[i] / b;
    }
    const bool exact = n < m || beta[n - 1] <= 1e-14 * (std::fabs(alpha[n - 1]) + 1e-300);
    std::vector<double> A(static_cast<size_t>(n) * n, 0.0), Q;
    for (int i = 0; i < n; ++i) {
      A[static_cast<size_t>(i) * n + i] = alpha[i];
      if (i + 1 < n) A[static_cast<size_t>(i) * n + i + 1] = A[static_cast<size_t>(i + 1) * n + i] = beta[i];
    }
    jacobi_eig(n, A, Q);
    double s = 1.0;
    std::vector<cplx> c(static_cast<size_t>(n));
    bool ok = false;
    for (int attempt = 0; attempt < 60; ++attempt) {
      for (int i = 0; i < n; ++i) {
        cplx acc(0.0, 0.0);
        for (int k = 0; k < n; ++k)
          acc += Q[static_cast<size_t>(i) * n + k] * std::exp(-s * zrem * A[static_cast<size_t>(k) * n + k]) *
                 Q[static_cast<size_t>(k)];
        c[static_cast<size_t>(i)] = acc;
      }
      const double err = exact ? 0.0 : beta[n - 1] * std::abs(c[static_cast<size_t>(n - 1)]);
      if (err <= tol * s) {
        ok = true;
        break;
      }
      s *= 0.5;
    }
    if (!ok) return -3;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; ++i) {
      cplx acc(0.0, 0.0);
      for (int j = 0; j < n; ++j) acc += c[static_cast<size_t>(j)] * V[static_cast<size_t>(j) * D + i];
      out[i] = beta0 * acc;
    }
    zrem *= (1.0 - s);
    if (s >= 1.0) break;
  }
  return matvecs;
}

}  // extern "C"
