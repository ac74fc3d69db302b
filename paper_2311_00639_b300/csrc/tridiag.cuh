// Projected exponential of a Lanczos run (FP64, one warp): the eigensystem of
// the symmetric tridiagonal T, then the substep search.  Shared by the
// single-state and batched engines.
//
// Eigensystem.  FP64 instructions are scarce on this part (a warp-wide DFMA
// costs about as much as 64 cycles of issue, whatever the active lanes), so
// the default path gives every lane its own eigenvalue and eigenvector and
// keeps each lane's work to a few O(n) recurrences:
//   1. bisection on the Sturm count (sign changes along the leading minors
//      det(T_i - x), by their three-term recurrence) in FP32 locates
//      eigenvalue k of T for lane k;
//   2. Newton's method on the characteristic polynomial det(T_i - x), its
//      three-term recurrence and derivative in FP64, polishes it, safeguarded
//      by the Sturm count of the same recurrence (sign changes along the
//      leading minors: the bracket always holds eigenvalue k);
//   3. the eigenvector from the two three-term recurrences (from the top row
//      and from the bottom row), joined at the row where the product of the
//      two solutions is largest: that row maximises |[(T - x)^{-1}]_rr|, the
//      twisted-factorisation choice (Dhillon and Parlett's MRRR) that keeps
//      both halves accurate.
// The result is accepted when every lane's Newton iteration converged, the
// eigenvalues come out strictly increasing, and the eigensystem reproduces
// the first columns of T^0 and T^1 to 1e-13 (the step only needs
// c = sum_k f(lam_k) z_k z_k[0], and vectors of nearly equal eigenvalues,
// which come out mixed, err in c as in these sums); otherwise (tight
// clusters, e.g. converged Ritz values of a small block) the warp
// falls back to the implicit QL algorithm with Wilkinson shifts (the tql2
// procedure of Bowdler, Martin, Reinsch and Wilkinson, Handbook for Automatic
// Computation II), every lane running the same recurrence.
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

// phi_1(w) = (e^w - 1) / w for complex w, given e = e^w.
__device__ inline double2 phi1_(double re, double im, double2 e) {
  const double d = re * re + im * im;
  if (d < 1e-12) return make_double2(1.0 + 0.5 * re, 0.5 * im);
  const double nr = e.x - 1.0, ni = e.y;
  const double r = 1.0 / d;
  return make_double2((nr * re + ni * im) * r, (ni * re - nr * im) * r);
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

// Sign bits of two doubles / floats differ (integer test: FP64 compares
// cost as much as FP64 arithmetic on this part).
__device__ inline bool sign_differs(double a, double b) { return (__double2hiint(a) ^ __double2hiint(b)) < 0; }
__device__ inline bool is_zero(double a) { return (__double_as_longlong(a) << 1) == 0; }

// Sturm counts below three points x0 < x1 < x2 in FP32: sign changes along
// det(T_i - x), i = 0..n, by the three-term recurrence on T / ||T|| (one
// dependent FMA per row and point; the three chains share each row's loads
// and run interleaved).  With the entries scaled to at most 1 a value grows
// by at most 3 a row, so pairs of consecutive values are checked (and
// rescaled by 2^-/+64 when they leave [2^-64, 2^64]) every 8 rows only.  An
// exact zero counts as non-negative (measure zero; the FP64 stage corrects).
__device__ inline void sturm_rescale_f32(float& p0, float& p1) {
  const int ex = (__float_as_int(p1) >> 23) & 0xFF;
  if (ex > 127 + 64) {
    p0 *= 0x1p-64f;
    p1 *= 0x1p-64f;
  } else if (ex < 127 - 64 && ((__float_as_int(p0) >> 23) & 0xFF) < 127 - 64) {
    p0 *= 0x1p64f;
    p1 *= 0x1p64f;
  }
}
__device__ inline void sturm_count3_f32(int n, const float* df, const float* e2f, const float (&x)[3], int (&c)[3]) {
  float p0[3], p1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    p0[j] = 1.f;
    p1[j] = df[0] - x[j];
    c[j] = static_cast<int>(static_cast<unsigned>(__float_as_int(p1[j])) >> 31);
  }
  for (int i = 1; i < n; ++i) {
    const float d = df[i], e2 = e2f[i - 1];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float p2 = fmaf(d - x[j], p1[j], -e2 * p0[j]);
      c[j] += static_cast<int>(static_cast<unsigned>(__float_as_int(p2) ^ __float_as_int(p1[j])) >> 31);
      p0[j] = p1[j];
      p1[j] = p2;
    }
    if ((i & 7) == 7) {
#pragma unroll
      for (int j = 0; j < 3; ++j) sturm_rescale_f32(p0[j], p1[j]);
    }
  }
}

// det(T_i - x) for the leading i x i blocks by the three-term recurrence, in
// FP64: returns p_n, dp_n/dx and the number of sign changes along
// p_0 .. p_n (= eigenvalues below x).  Pairs of consecutive values are
// rescaled by 2^-/+600 when they leave [2^-600, 2^600] (the ratio p/dp is
// unchanged).
struct CharPoly {
  double p, dp;
  int below;
};
__device__ inline CharPoly char_poly(int n, const double* d, const double* e2, double x) {
  double p0 = 1.0, dp0 = 0.0;
  double p1 = d[0] - x, dp1 = -1.0;
  if (is_zero(p1)) p1 = -0x1p-900;
  int below = __double2hiint(p1) < 0 ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const double a = d[i] - x;
    double p2 = fma(a, p1, -e2[i - 1] * p0);
    const double dp2 = fma(a, dp1, -fma(e2[i - 1], dp0, p1));
    if (is_zero(p2)) p2 = -0x1p-300 * p1;  // a zero counts as a sign change
    below += sign_differs(p2, p1) ? 1 : 0;
    p0 = p1;
    dp0 = dp1;
    p1 = p2;
    dp1 = dp2;
    const int ex = (__double2hiint(p1) >> 20) & 0x7FF;
    if (ex > 1023 + 600) {
      p0 *= 0x1p-600;
      p1 *= 0x1p-600;
      dp0 *= 0x1p-600;
      dp1 *= 0x1p-600;
    } else if (ex < 1023 - 600 && ((__double2hiint(p0) >> 20) & 0x7FF) < 1023 - 600) {
      p0 *= 0x1p600;
      p1 *= 0x1p600;
      dp0 *= 0x1p600;
      dp1 *= 0x1p600;
    }
  }
  return {p1, dp1, below};
}

// Unbiased binary exponent of |v| (v != 0), from its bits.
__device__ inline int exp2_of(double v) { return ((__double2hiint(v) >> 20) & 0x7FF) - 1023; }

// Lane-parallel eigensystem of T (see the header): eigenvalue k of lane k
// (and k + 32) in lam[0] (lam[1]), eigenvector k in column k of Z.  Returns
// false when the checks fail (the caller then runs the QL path).
__device__ bool eig_lane_parallel(const KScalars* sc, int n, double (*Z)[kMaxKrylov + 1], double (&lam)[2]) {
  __shared__ double sd[kMaxKrylov], se[kMaxKrylov], se2[kMaxKrylov], sinv[kMaxKrylov];
  __shared__ float sdf[kMaxKrylov], se2f[kMaxKrylov];
  const int lane = threadIdx.x & 31;
  // Gershgorin interval in FP32, widened by 2^-16 relative (it only brackets)
  float glf = 3e38f, ghf = -3e38f;
  for (int i = lane; i < n; i += 32) {
    const double di = sc->alpha[i];
    const double ei = i < n - 1 ? sc->beta[i] : 0.0;
    const float ep = i > 0 ? static_cast<float>(sc->beta[i - 1]) : 0.f;
    sd[i] = di;
    se[i] = ei;
    se2[i] = ei * ei;
    sinv[i] = i < n - 1 ? 1.0 / ei : 0.0;
    const float df = static_cast<float>(di), ef = fabsf(static_cast<float>(ei)) + fabsf(ep);
    glf = fminf(glf, df - ef);
    ghf = fmaxf(ghf, df + ef);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    glf = fminf(glf, __shfl_xor_sync(0xffffffffu, glf, o));
    ghf = fmaxf(ghf, __shfl_xor_sync(0xffffffffu, ghf, o));
  }
  __syncwarp();
  const float padf = 0x1p-16f * fmaxf(fabsf(glf), fabsf(ghf));
  const double glo = static_cast<double>(glf - padf), ghi = static_cast<double>(ghf + padf);
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double width = ghi - glo;
  if (!(width > 0.0) || !(tnorm < 1e300)) return false;
  const double rn = 1.0 / tnorm;  // the FP32 bracketing works on T / ||T||
  for (int i = lane; i < n; i += 32) {
    sdf[i] = static_cast<float>(sd[i] * rn);
    se2f[i] = static_cast<float>(se2[i] * rn * rn);
  }
  __syncwarp();
  bool ok = true;
  for (int slot = 0; slot < 2; ++slot) {
    const int k = lane + 32 * slot;
    if (slot == 1 && n <= 32) break;
    double xk = 0.0;
    if (k < n) {
      // 1. FP32 bracketing of the k-th eigenvalue (0-based, ascending): the
      //    interval [a, b] (count(a) <= k < count(b)) is cut in four per
      //    round by three Sturm counts at once, down to FP32 resolution
      float a = static_cast<float>((glo - 1e-6 * width) * rn), b = static_cast<float>((ghi + 1e-6 * width) * rn);
      for (int it = 0; it < 16; ++it) {
        const float w = b - a;
        const float xs3[3] = {a + 0.25f * w, a + 0.5f * w, a + 0.75f * w};
        if (!(xs3[0] > a && xs3[2] < b && xs3[0] < xs3[1] && xs3[1] < xs3[2])) break;
        int cnt[3];
        sturm_count3_f32(n, sdf, se2f, xs3, cnt);
        if (cnt[0] > k) {
          b = xs3[0];
        } else if (cnt[1] > k) {
          a = xs3[0];
          b = xs3[1];
        } else if (cnt[2] > k) {
          a = xs3[1];
          b = xs3[2];
        } else {
          a = xs3[2];
        }
      }
      // 2. FP64 Newton on det(T - x), bracketed by the Sturm count
      const double af = static_cast<double>(a) * tnorm, bf = static_cast<double>(b) * tnorm;
      double A = af - 4.0 * (bf - af) - 1e-6 * width;
      double B = bf + 4.0 * (bf - af) + 1e-6 * width;
      double x = 0.5 * (af + bf);
      bool conv = false;
      for (int it = 0; it < 12 && !conv; ++it) {
        const CharPoly cp = char_poly(n, sd, se2, x);
        if (cp.below > k)
          B = x;
        else
          A = x;
        // a Newton step at rounding level ends the iteration (the iterate may
        // then sit on the bracket's end, where the count put it)
        const double step = !is_zero(cp.dp) ? cp.p / cp.dp : 1e300;
        // Newton converges quadratically here: after a step below 2^-36 of the
        // scale the error is of order step^2 / gap, far below rounding
        if (fabs(step) <= 0x1p-36 * fmax(fabs(x), 1e-3 * tnorm)) {
          conv = true;
          x -= step;
          break;
        }
        double xn = x - step;
        if (!(xn > A && xn < B)) xn = 0.5 * (A + B);
        x = xn;
      }
      ok = ok && conv;
      xk = x;
      // 3. eigenvector: x_i from the top (x_0 = 1), y_i from the bottom
      //    (y_{n-1} = 1).  When a value passes 2^600 the values stored so far
      //    are scaled by 2^-600 with it (rare; earlier entries may underflow
      //    to zero, they are negligible then).  The backward sweep picks the
      //    join row r maximising |x_r y_r| from binary exponents on the fly.
      double xv[kMaxKrylov], yv[kMaxKrylov];
      {
        double u0 = 0.0, u1 = 1.0;
        xv[0] = 1.0;
        for (int i = 0; i + 1 < n; ++i) {
          double u2 = fma(x - sd[i], u1, -(i > 0 ? se[i - 1] : 0.0) * u0) * sinv[i];
          if (exp2_of(u2) > 600) {
            u2 *= 0x1p-600;
            u1 *= 0x1p-600;
            for (int j = 0; j <= i; ++j) xv[j] *= 0x1p-600;
          }
          xv[i + 1] = u2;
          u0 = u1;
          u1 = u2;
        }
      }
      auto expsum = [](double a, double b) {
        return (is_zero(a) || is_zero(b)) ? -100000 : exp2_of(a) + exp2_of(b);
      };
      int r = n - 1;
      int best = expsum(xv[n - 1], 1.0);
      {
        double u0 = 0.0, u1 = 1.0;
        yv[n - 1] = 1.0;
        for (int i = n - 1; i > 0; --i) {
          double u2 = fma(x - sd[i], u1, -(i < n - 1 ? se[i] : 0.0) * u0) * sinv[i - 1];
          if (exp2_of(u2) > 600) {
            u2 *= 0x1p-600;
            u1 *= 0x1p-600;
            for (int j = i; j < n; ++j) yv[j] *= 0x1p-600;
            best -= 600;
          }
          yv[i - 1] = u2;
          u0 = u1;
          u1 = u2;
          const int e = expsum(xv[i - 1], u2);
          if (e > best) {
            best = e;
            r = i - 1;
          }
        }
      }
      const double ixr = 1.0 / xv[r], iyr = 1.0 / yv[r];
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) {
        const double v = (i <= r) ? xv[i] * ixr : yv[i] * iyr;
        nrm = fma(v, v, nrm);
      }
      const double inv = rsqrt(nrm);
      const double fx = ixr * inv, fy = iyr * inv;
      for (int i = 0; i < n; ++i) Z[i][k] = (i <= r) ? xv[i] * fx : yv[i] * fy;
    }
    lam[slot] = xk;
  }
  __syncwarp();
  // checks: eigenvalues strictly increasing (relative gaps >= 1e-7), and the
  // eigensystem reproduces the first column of T^0 and T^1:
  // sum_k z_k z_k[0] = e_1 and sum_k lam_k z_k z_k[0] = T e_1 to 1e-13.  The
  // step uses c = sum_k f(lam_k) z_k z_k[0]; errors of nearly equal lam_k
  // (whose vectors mix) enter c as these two sums do, so passing them bounds
  // the eigenvector part of the error of c.
  __shared__ double szl[kMaxKrylov];  // lam_k z_k[0]
  for (int slot = 0; slot < 2; ++slot) {
    const int k = lane + 32 * slot;
    if (k < n) szl[k] = lam[slot] * Z[0][k];
  }
  __syncwarp();
  const double next0 = __shfl_down_sync(0xffffffffu, lam[0], 1);
  const double next1 = __shfl_down_sync(0xffffffffu, lam[1], 1);
  const double first1 = __shfl_sync(0xffffffffu, lam[1], 0);
  for (int slot = 0; slot < 2; ++slot) {
    const int i = lane + 32 * slot;
    if (i + 1 < n) {
      const double nx = (slot == 0) ? (lane < 31 ? next0 : first1) : next1;
      if (!(nx - lam[slot] >= 1e-7 * width)) ok = false;
    }
    if (i < n) {
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < n; ++k) {
        s0 = fma(Z[i][k], Z[0][k], s0);
        s1 = fma(Z[i][k], szl[k], s1);
      }
      const double t0 = i == 0 ? 1.0 : 0.0;
      const double t1 = i == 0 ? sd[0] : (i == 1 ? se[0] : 0.0);
      if (!(fabs(s0 - t0) <= 1e-13) || !(fabs(s1 - t1) <= 1e-13 * tnorm)) ok = false;
    }
  }
  return __all_sync(0xffffffffu, ok);
}

// Implicit QL with Wilkinson shifts (tql2, see the header): every lane runs
// the same recurrence on its own copy of (d, e) and rotates the eigenvector
// rows k = lane, lane + 32 it owns.  Returns 0, or 2 if an eigenvalue needed
// more than 100 iterations.
__device__ int tridiag_ql(const KScalars* sc, int n, double (*Z)[kMaxKrylov + 1], double (&lam)[2]) {
  const int lane = threadIdx.x & 31;
  double d[kMaxKrylov], e[kMaxKrylov];
  for (int i = 0; i < n; ++i) {
    d[i] = sc->alpha[i];
    e[i] = (i < n - 1) ? sc->beta[i] : 0.0;
  }
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
  lam[0] = lane < n ? d[lane] : 0.0;
  lam[1] = lane + 32 < n ? d[lane + 32] : 0.0;
  return status;
}

// Substep search on the eigensystem (lam, Z) of T: largest s = 2^-k with
// estimated local error <= tol * s.  Estimates (relative to ||c||):
// beta_m |e_m^T e^{-hT} e_1| and beta_m |h| |e_m^T phi_1(-hT) e_1| (Saad 1992,
// Thm. 5.1), the larger one.  Each lane evaluates the exponentials of its own
// eigenvalues (k = lane, lane + 32) once per attempt; the small products then
// use shared memory.
__device__ void substep_search(KScalars* sc, int n, int m, double resid, double z_re, double z_im, double tol,
                               double (*Z)[kMaxKrylov + 1], const double (&lam)[2], int status) {
  const int lane = threadIdx.x & 31;
  __shared__ double Er[kMaxKrylov], Ei[kMaxKrylov], Pr[kMaxKrylov], Pi[kMaxKrylov];
  double s_frac = 1.0, err = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 64 && status == 0; ++attempt) {
    const double hr = s_frac * z_re, hi = s_frac * z_im;
    for (int k = lane, slot = 0; k < n; k += 32, ++slot) {
      const double w0 = Z[0][k];
      const double dk = lam[slot];
      const double2 ex = cexp_(-hr * dk, -hi * dk);
      const double2 ph = phi1_(-hr * dk, -hi * dk, ex);
      Er[k] = ex.x * w0;
      Ei[k] = ex.y * w0;
      Pr[k] = ph.x * w0;
      Pi[k] = ph.y * w0;
    }
    __syncwarp();
    double cr0 = 0, ci0 = 0, cr1 = 0, ci1 = 0;  // rows lane, lane+32
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
    }
    // last row of phi_1(-hT) e_1: each lane its own eigenvalues' terms, then a warp sum
    double pr_last = 0, pi_last = 0;
    for (int k = lane; k < n; k += 32) {
      pr_last += Z[n - 1][k] * Pr[k];
      pi_last += Z[n - 1][k] * Pi[k];
    }
    pr_last = warp_sum_(pr_last);
    pi_last = warp_sum_(pi_last);
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

// One warp.  Eigensystem by the lane-parallel path, or by implicit QL where
// every lane runs the same scalar recurrence on its own copy of (d, e) and
// rotates the eigenvector rows k = lane, lane + 32 it owns.  Z is shared
// scratch of kMaxKrylov x (kMaxKrylov + 1) doubles.
__device__ void tridiag_warp(KScalars* sc, int m, double z_re, double z_im, double tol,
                             double (*Z)[kMaxKrylov + 1], bool allow_lane_parallel = true) {
  const int lane = threadIdx.x & 31;
  const int n = min(sc->m_eff, m);
  if (n <= 0) {  // x = 0
    if (lane == 0) {
      sc->s_acc = 1.0;
      sc->err = 0.0;
    }
    return;
  }
  double lam[2] = {0.0, 0.0};
  int status = 0;
  const double resid = sc->beta[n - 1];
  if (n == 1 || !allow_lane_parallel || !eig_lane_parallel(sc, n, Z, lam)) {
    status = tridiag_ql(sc, n, Z, lam);
    if ((threadIdx.x & 31) == 0) sc->tot.ql += 1;
  }
  __syncwarp();
  substep_search(sc, n, m, resid, z_re, z_im, tol, Z, lam, status);
}

}  // namespace
}  // namespace syk
