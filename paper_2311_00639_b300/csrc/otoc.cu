// OTOC driver: the parity-block single-state formula of the supplement,
//   F_P(t) = <psi_P| e^{(it-b/8)H_PP} chi_a e^{-(it+b/4)H_QQ} chi_b
//            e^{(it-b/4)H_PP} chi_a e^{-(it+b/4)H_QQ} chi_b e^{-bH_PP/8} |psi_P>,
// F = F_U + F_D (Eq. (2) of the main text evaluated on a typical state, or
// summed over all basis states for the exact trace).
//
// Per state and block P the host loop keeps four vectors of the block:
//   u0  = e^{-b H/8} psi_P                  (computed once),
//   bra = e^{-(it_n + b/8) H} psi_P          (advanced by e^{-i dt H} per grid point),
//   k1, k2: the ket chain, rebuilt for every t (it depends on t in all four evolutions).
#include <algorithm>
#include <memory>
#include <vector>

#include "kernels.cuh"

namespace syk {

namespace {
struct DevBuf {
  void* p = nullptr;
  explicit DevBuf(size_t n) {
    if (n && cudaMalloc(&p, n) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error(SYK_ENOMEM, "syk_otoc: device allocation of " + std::to_string(n) + " bytes failed");
    }
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};
}  // namespace

void otoc_run(const syk_terms* h, int a, int b, double beta, const double* tg, int n_t, int mode, int n_states,
              uint64_t seed, const void* psi_opt, int m, double tol, int max_sub, bool reorth, bool two_pass,
              double* F_raw, double* otoc, KrylovResult& tot, cudaStream_t st) {
  SYK_REQUIRE(h->hermitian, "syk_otoc needs a Hermitian H (complex couplings: use syk_otoc_nonhermitian)");
  const size_t esz = elem_bytes(h->dtype);
  const size_t vb = (static_cast<size_t>(h->D) * esz + 255) & ~size_t(255);
  const bool exact = mode == SYK_OTOC_EXACT_TRACE;
  const int rows = exact ? 1 : n_states;
  const int G = vec_grid(h);
  DevBuf vecs(4 * vb);
  DevBuf ws(krylov_ws_bytes(h, m, two_pass));
  DevBuf small((2 * static_cast<size_t>(G) + 8) * sizeof(double) + static_cast<size_t>(rows) * n_t * 2 * sizeof(double));
  char* vp = static_cast<char*>(vecs.p);
  void* u0 = vp;
  void* bra = vp + vb;
  void* k1 = vp + 2 * vb;
  void* k2 = vp + 3 * vb;
  double* partial = static_cast<double*>(small.p);
  double* n2 = partial + 2 * G;
  double* Fdev = n2 + 8;
  SYK_CUDA(cudaMemsetAsync(Fdev, 0, static_cast<size_t>(rows) * n_t * 2 * sizeof(double), st));
  krylov_totals_reset(ws.p, st);

  auto evolve = [&](int blk, double tau, double t, void* x) {
    KrylovResult r = krylov_evolve_one(h, blk, tau, t, x, x, m, tol, max_sub, reorth, two_pass, ws.p, st);
    tot.matvecs += r.matvecs;
    tot.substeps += r.substeps;
    tot.err += r.err;
  };

  const int64_t n_outer = exact ? 2 * h->D : n_states;
  const double scale = exact ? 1.0 / (2.0 * static_cast<double>(h->D)) : 1.0;
  for (int64_t s = 0; s < n_outer; ++s) {
    const int row = exact ? 0 : static_cast<int>(s);
    if (!exact && !psi_opt) {  // ||psi_U||^2 + ||psi_D||^2 of the Philox state
      for (int P = 0; P < 2; ++P) {
        launch_random_state(h, seed, static_cast<uint64_t>(s), P, u0, st);
        launch_norm_partials(h, u0, partial, st);
        launch_sum_finalize(partial, G, n2, P, st);
      }
    }
    for (int P = 0; P < 2; ++P) {
      const int Q = 1 - P;
      if (exact) {
        if (s / h->D != P) continue;  // basis state lives in the other block: F_P = 0
        launch_basis_vector(h, u0, s % h->D, st);
      } else if (psi_opt) {
        const char* src = static_cast<const char*>(psi_opt) + (static_cast<size_t>(s) * 2 + P) * h->D * esz;
        SYK_CUDA(cudaMemcpyAsync(u0, src, h->D * esz, cudaMemcpyDeviceToDevice, st));
      } else {
        launch_random_state(h, seed, static_cast<uint64_t>(s), P, u0, st);
        launch_scale_inv_sqrt(h, u0, n2, st);
      }
      evolve(P, beta / 8.0, 0.0, u0);
      SYK_CUDA(cudaMemcpyAsync(bra, u0, h->D * esz, cudaMemcpyDeviceToDevice, st));
      double tprev = 0.0;
      for (int n = 0; n < n_t; ++n) {
        const double t = tg[n];
        if (t != tprev) evolve(P, 0.0, t - tprev, bra);
        tprev = t;
        launch_apply_chi(h, b, P, u0, k1, 1, st);
        evolve(Q, beta / 4.0, t, k1);
        launch_apply_chi(h, a, Q, k1, k2, 1, st);
        evolve(P, beta / 4.0, -t, k2);
        launch_apply_chi(h, b, P, k2, k1, 1, st);
        evolve(Q, beta / 4.0, t, k1);
        launch_apply_chi(h, a, Q, k1, k2, 1, st);
        launch_zdot_partials(h, bra, k2, partial, st);
        launch_zdot_finalize(partial, G, Fdev + (static_cast<size_t>(row) * n_t + n) * 2, scale, 1, st);
      }
    }
  }
  std::vector<double> Fh(static_cast<size_t>(rows) * n_t * 2);
  SYK_CUDA(cudaMemcpyAsync(Fh.data(), Fdev, Fh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SYK_CUDA(cudaStreamSynchronize(st));
  krylov_totals_collect(ws.p, st, tot);  // counts and failures of the queued Lanczos evolves
  if (F_raw) std::copy(Fh.begin(), Fh.end(), F_raw);
  if (otoc) {
    std::vector<double> mean(n_t, 0.0);
    for (int r = 0; r < rows; ++r)
      for (int n = 0; n < n_t; ++n) mean[n] += Fh[(static_cast<size_t>(r) * n_t + n) * 2] / rows;
    for (int n = 0; n < n_t; ++n) otoc[n] = mean[n] / mean[0];
  }
}

}  // namespace syk
