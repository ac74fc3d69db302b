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
#include "tridiag.cuh"

namespace syk {
namespace {

__global__ void __launch_bounds__(32) k_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  tridiag_warp(sc, m, z_re, z_im, tol, Z);
}

}  // namespace

void launch_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol, cudaStream_t st) {
  k_tridiag<<<1, 32, 0, st>>>(sc, m, z_re, z_im, tol);
  SYK_CUDA(cudaGetLastError());
}

// Workspace layout (bytes, each region 256-aligned):
//   KScalars | partialA [G] | partialN [G] | partialR [64][G][2] | vectors
size_t krylov_ws_bytes(const syk_terms* h, int m, bool two_pass) {
  if (!h->hermitian) return arnoldi_ws_bytes(h, m);
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
  if (!h->hermitian) {  // complex couplings: full orthogonalisation (Arnoldi) instead of the three-term recurrence
    SYK_REQUIRE(!reorth && !two_pass, "a non-Hermitian H needs the stored Arnoldi basis (no reorth / two_pass)");
    return arnoldi_evolve_one(h, block, tau, t, x, y, m, tol, max_substeps, ws, st);
  }
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
  // basis vectors back to back: the combine and re-orthogonalisation kernels
  // index vector j at j * D amplitudes
  const size_t vb = static_cast<size_t>(h->D) * elem_bytes(h->dtype);
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
