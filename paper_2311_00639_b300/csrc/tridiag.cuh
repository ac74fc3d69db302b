// Projected exponential of a Lanczos run (FP64, one warp): implicit QL on the
// symmetric tridiagonal T, then the substep search.  Shared by the
// single-state and batched engines.
#pragma once

#include <cfloat>

#include "kernels.cuh"

namespace syk {
namespace {

__device__ inline double2 cexp_(double re, double im) {
  double s, c;
  sincos(im, &s, &c);
  const double e = exp(re);
  return make_double2(e * c, e * s);
}

// phi_1(w) = (e^w - 1) / w for complex w.
__device__ inline double2 phi1_(double re, double im) {
  const double a = hypot(re, im);
  if (a < 1e-6) return make_double2(1.0 + 0.5 * re, 0.5 * im);
  const double2 e = cexp_(re, im);
  const double nr = e.x - 1.0, ni = e.y;
  const double d = re * re + im * im;
  return make_double2((nr * re + ni * im) / d, (ni * re - nr * im) / d);
}

// Bits of |v| (IEEE order: for non-negative doubles, integer order = value order).
__device__ inline long long abs_bits_(double v) { return __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL; }

// |e| <= eps * max(|a|, |b|), eps = 2^-52, decided on bit patterns: FP64
// instructions are costly on this part and this test runs inside the QL scan.
// Multiplying by 2^-52 subtracts 52 from the exponent field; when that would
// leave the normal range the threshold is taken as 0 (deflate only e = 0).
__device__ inline bool negligible_(double e, double a, double b) {
  const long long m = max(abs_bits_(a), abs_bits_(b));
  const long long t = m - (52LL << 52);
  return abs_bits_(e) <= (t > (1LL << 52) ? t : 0LL);
}

__device__ inline double warp_sum_(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp.  Every lane runs the same scalar QL recurrence on its own copy
// of (d, e) and rotates the eigenvector rows k = lane, lane + 32 it owns.
// Z is shared scratch of kMaxKrylov x (kMaxKrylov + 1) doubles.
__device__ void tridiag_warp(KScalars* sc, int m, double z_re, double z_im, double tol,
                             double (*Z)[kMaxKrylov + 1]) {
  const int lane = threadIdx.x & 31;
  const int n = min(sc->m_eff, m);
  if (n <= 0) {  // x = 0
    if (lane == 0) {
      sc->s_acc = 1.0;
      sc->err = 0.0;
    }
    return;
  }
  double d[kMaxKrylov], e[kMaxKrylov];
  for (int i = 0; i < n; ++i) {
    d[i] = sc->alpha[i];
    e[i] = (i < n - 1) ? sc->beta[i] : 0.0;
  }
  const double resid = sc->beta[n - 1];
  for (int k = lane; k < n; k += 32)
    for (int i = 0; i < n; ++i) Z[k][i] = (i == k) ? 1.0 : 0.0;
  __syncwarp();
  int status = 0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int mm = l;
      for (; mm < n - 1; ++mm)
        if (negligible_(e[mm], d[mm], d[mm + 1])) break;
      if (mm == l) break;
      if (++iter > 100) {
        status = 2;
        break;
      }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = mm - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        // Givens rotation from one reciprocal square root: rho = f^2 + g^2,
        // r = rho rho^{-1/2}, s = f rho^{-1/2}, c = g rho^{-1/2} (the entries of
        // a Lanczos T are far from the overflow range).
        const double rho = fma(f, f, g * g);
        if (abs_bits_(rho) == 0) {
          e[i + 1] = 0.0;
          d[i + 1] -= p;
          e[mm] = 0.0;
          deflated = true;
          break;
        }
        const double inv = rsqrt(rho);
        r = rho * inv;
        e[i + 1] = r;
        s = f * inv;
        c = g * inv;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        for (int k = lane; k < n; k += 32) {
          const double zf = Z[k][i + 1];
          Z[k][i + 1] = s * Z[k][i] + c * zf;
          Z[k][i] = c * Z[k][i] - s * zf;
        }
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
    if (status) break;
  }
  __syncwarp();
  // Substep search: largest s = 2^-k with estimated local error <= tol * s.
  // Estimates (relative to ||c||): beta_m |e_m^T e^{-hT} e_1| and
  // beta_m |h| |e_m^T phi_1(-hT) e_1| (Saad 1992, Thm. 5.1), the larger one.
  // Each lane evaluates the exponentials of its own eigenvalues (k = lane,
  // lane + 32) once per attempt; the small products then use shared memory.
  __shared__ double Er[kMaxKrylov], Ei[kMaxKrylov], Pr[kMaxKrylov], Pi[kMaxKrylov];
  double s_frac = 1.0, err = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 64 && status == 0; ++attempt) {
    const double hr = s_frac * z_re, hi = s_frac * z_im;
    for (int k = lane; k < n; k += 32) {
      const double w0 = Z[0][k];
      const double2 ex = cexp_(-hr * d[k], -hi * d[k]);
      const double2 ph = phi1_(-hr * d[k], -hi * d[k]);
      Er[k] = ex.x * w0;
      Ei[k] = ex.y * w0;
      Pr[k] = ph.x * w0;
      Pi[k] = ph.y * w0;
    }
    __syncwarp();
    double cr0 = 0, ci0 = 0, cr1 = 0, ci1 = 0;  // rows lane, lane+32
    double pr_last = 0, pi_last = 0;
    for (int k = 0; k < n; ++k) {
      const double er = Er[k], ei = Ei[k];
      if (lane < n) {
        cr0 += Z[lane][k] * er;
        ci0 += Z[lane][k] * ei;
      }
      if (lane + 32 < n) {
        cr1 += Z[lane + 32][k] * er;
        ci1 += Z[lane + 32][k] * ei;
      }
      pr_last += Z[n - 1][k] * Pr[k];
      pi_last += Z[n - 1][k] * Pi[k];
    }
    __syncwarp();
    const double nc = sqrt(warp_sum_(cr0 * cr0 + ci0 * ci0 + cr1 * cr1 + ci1 * ci1));
    // |c_{n-1}|: owned by lane (n-1) % 32 in slot (n-1) / 32.
    const int owner = (n - 1) & 31;
    const double cl_r = __shfl_sync(0xffffffffu, (n - 1) < 32 ? cr0 : cr1, owner);
    const double cl_i = __shfl_sync(0xffffffffu, (n - 1) < 32 ? ci0 : ci1, owner);
    const double e1 = resid * hypot(cl_r, cl_i);
    const double e2 = resid * hypot(hr, hi) * hypot(pr_last, pi_last);
    err = (nc > 0.0) ? fmax(e1, e2) / nc : 0.0;
    const bool exact = n < m;  // invariant subspace found (breakdown)
    if (exact || err <= tol * s_frac || !(err == err)) {
      ok = exact || (err == err);
      if (lane < n) {
        sc->c_re[lane] = cr0;
        sc->c_im[lane] = ci0;
      }
      if (lane + 32 < n) {
        sc->c_re[lane + 32] = cr1;
        sc->c_im[lane + 32] = ci1;
      }
      if (exact) err = 0.0;
      break;
    }
    s_frac *= 0.5;
  }
  if (lane == 0) {
    sc->s_acc = ok ? s_frac : 0.0;
    sc->err = err;
    sc->status = status ? status : (ok ? 0 : 1);
  }
}

}  // namespace
}  // namespace syk
