// Lanczos propagation y = e^{-z H_P} x, z = tau + i t (supplement Sec. I.A:
// the paper re-implements a restarted Krylov method for e^{-iHt}|psi>; this
// is a Lanczos variant with the a-posteriori error estimate and substep
// control of Expokit (Sidje, ACM TOMS 24, 1998)).
//
// One substep:  beta0 = ||x||, v_0 = x / beta0; m Lanczos steps build the
// real symmetric tridiagonal T (alpha_j = Re <v_j, H v_j>, beta_j = ||w_j||)
// and the basis V; the device eigen-decomposes T (implicit QL with
// Wilkinson-type shifts), picks the largest fraction s of the remaining step
// whose error estimate passes, and forms y = beta0 V e^{-s z T} e_1.  All
// scalars are float64; vectors are complex64 or complex128.
#include <cfloat>
#include <cmath>
#include <algorithm>
#include <complex>

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

__device__ inline double warp_sum_(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp.  Every lane runs the same scalar QL recurrence on its own copy
// of (d, e) and rotates the eigenvector rows k = lane, lane + 32 it owns.
__global__ void __launch_bounds__(32) k_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  const int lane = threadIdx.x;
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
      for (; mm < n - 1; ++mm) {
        const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
        if (fabs(e[mm]) <= DBL_EPSILON * dd) break;
      }
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
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[mm] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
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
  double s_frac = 1.0, err = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 64 && status == 0; ++attempt) {
    const double hr = s_frac * z_re, hi = s_frac * z_im;
    double cr0 = 0, ci0 = 0, cr1 = 0, ci1 = 0;  // rows lane, lane+32
    double pr_last = 0, pi_last = 0;
    for (int k = 0; k < n; ++k) {
      const double2 ex = cexp_(-hr * d[k], -hi * d[k]);
      const double w0 = Z[0][k];
      if (lane < n) {
        cr0 += Z[lane][k] * ex.x * w0;
        ci0 += Z[lane][k] * ex.y * w0;
      }
      if (lane + 32 < n) {
        cr1 += Z[lane + 32][k] * ex.x * w0;
        ci1 += Z[lane + 32][k] * ex.y * w0;
      }
      const double2 ph = phi1_(-hr * d[k], -hi * d[k]);
      pr_last += Z[n - 1][k] * ph.x * w0;
      pi_last += Z[n - 1][k] * ph.y * w0;
    }
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

void launch_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol, cudaStream_t st) {
  k_tridiag<<<1, 32, 0, st>>>(sc, m, z_re, z_im, tol);
  SYK_CUDA(cudaGetLastError());
}

// Workspace layout (bytes, each region 256-aligned):
//   KScalars | partialA [G] | partialN [G] | partialR [64][G][2] | vectors
size_t krylov_ws_bytes(const syk_terms* h, int m, bool two_pass) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t G = static_cast<size_t>(std::max(vec_grid(h), matvec_grid(h)));
  size_t b = up(sizeof(KScalars)) + 2 * up(G * sizeof(double)) + up(kMaxKrylov * G * 2 * sizeof(double));
  const size_t nvec = two_pass ? 3 : static_cast<size_t>(m) + 1;
  b += nvec * up(static_cast<size_t>(h->D) * elem_bytes(h->dtype));
  return b;
}

// Evolve one state.  x and y are device vectors of D amplitudes; y may alias x.
KrylovResult krylov_evolve_one(const syk_terms* h, int block, double tau, double t, const void* x, void* y, int m,
                               double tol, int max_substeps, bool reorth, bool two_pass, void* ws, cudaStream_t st) {
  KrylovResult res;
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t G = static_cast<size_t>(std::max(vec_grid(h), matvec_grid(h)));
  char* p = static_cast<char*>(ws);
  KScalars* sc = reinterpret_cast<KScalars*>(p);
  p += up(sizeof(KScalars));
  double* partialA = reinterpret_cast<double*>(p);
  p += up(G * sizeof(double));
  double* partialN = reinterpret_cast<double*>(p);
  p += up(G * sizeof(double));
  double* partialR = reinterpret_cast<double*>(p);
  p += up(kMaxKrylov * G * 2 * sizeof(double));
  const size_t vb = up(static_cast<size_t>(h->D) * elem_bytes(h->dtype));
  char* vecs = p;
  const size_t esz = elem_bytes(h->dtype);
  const int npA = matvec_grid(h), npN = vec_grid(h);
  m = static_cast<int>(std::min<int64_t>(m, h->D));
  const double brk = 1e-14 * std::max(h->sum_abs, 1e-300);

  if (tau == 0.0 && t == 0.0) {
    if (x != y) SYK_CUDA(cudaMemcpyAsync(y, x, h->D * esz, cudaMemcpyDeviceToDevice, st));
    return res;
  }
  std::complex<double> zrem(tau, t);
  const void* xin = x;
  for (;;) {
    if (res.substeps >= max_substeps)
      throw Error(SYK_ENOCONV, "Krylov evolve: max_substeps reached before the step was complete");
    if (!two_pass) {
      auto V = [&](int j) { return static_cast<void*>(vecs + static_cast<size_t>(j) * vb); };
      launch_norm_partials(h, xin, partialN, st);
      launch_scale_first(h, xin, V(0), partialN, sc, m, st);
      for (int j = 0; j < m; ++j) {
        launch_lanczos_matvec(h, block, V(j), j ? V(j - 1) : nullptr, V(j + 1), partialA, sc, j, st);
        launch_axpy_norm(h, V(j + 1), V(j), partialA, npA, partialN, sc, j, st);
        if (reorth) launch_reorth(h, V(j + 1), V(0), j, partialR, partialN, sc, st);
        launch_scale_next(h, V(j + 1), partialN, npN, sc, j, brk, st);
      }
      res.matvecs += m;
      launch_tridiag(sc, m, zrem.real(), zrem.imag(), tol, st);
      launch_combine(h, V(0), y, sc, m, st);
    } else {
      void* B[3] = {vecs, vecs + vb, vecs + 2 * vb};
      // pass 1: scalars only (ring of three vectors)
      launch_norm_partials(h, xin, partialN, st);
      launch_scale_first(h, xin, B[0], partialN, sc, m, st);
      int cur = 0, prv = 2, nxt = 1;
      for (int j = 0; j < m; ++j) {
        launch_lanczos_matvec(h, block, B[cur], j ? B[prv] : nullptr, B[nxt], partialA, sc, j, st);
        launch_axpy_norm(h, B[nxt], B[cur], partialA, npA, partialN, sc, j, st);
        launch_scale_next(h, B[nxt], partialN, npN, sc, j, brk, st);
        prv = cur;
        cur = nxt;
        nxt = 3 - prv - cur;
      }
      launch_tridiag(sc, m, zrem.real(), zrem.imag(), tol, st);
      // pass 2: regenerate v_j and accumulate y
      launch_recur_first(h, xin, B[0], y, sc, st);
      cur = 0;
      prv = 2;
      nxt = 1;
      for (int j = 0; j + 1 < m; ++j) {
        launch_lanczos_recur(h, block, B[cur], j ? B[prv] : nullptr, B[nxt], y, sc, j, st);
        prv = cur;
        cur = nxt;
        nxt = 3 - prv - cur;
      }
      res.matvecs += 2 * m - 1;
    }
    struct {
      double s_acc, err;
      int status;
    } hv;
    SYK_CUDA(cudaMemcpyAsync(&hv.s_acc, &sc->s_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaMemcpyAsync(&hv.err, &sc->err, sizeof(double), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaMemcpyAsync(&hv.status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaStreamSynchronize(st));
    res.substeps += 1;
    if (hv.status == 2) throw Error(SYK_ENOCONV, "Krylov evolve: tridiagonal eigensolver did not converge");
    if (hv.status != 0 || !(hv.s_acc > 0.0))
      throw Error(SYK_ENOCONV, "Krylov evolve: no acceptable substep (increase m or tol)");
    res.err += hv.err * hv.s_acc;
    if (hv.s_acc >= 1.0) break;
    zrem *= (1.0 - hv.s_acc);
    xin = y;
  }
  return res;
}

}  // namespace syk
