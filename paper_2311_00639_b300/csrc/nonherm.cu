// Non-Hermitian sparse SYK: H = sum_t (J_t + i M_t) chi_i chi_j chi_k chi_l,
// the other model the paper's conclusions name for OTOC studies.  The terms
// compile to the same block strings as Eq. (1) -- the value of each splits into
// a real-class and an imaginary-class string with the same masks -- so H psi
// runs on the unchanged matvec kernels; Krylov propagation of such a handle
// uses the Arnoldi engine (arnoldi.cu).
//
// OTOC reading (the paper gives no formula): Eq. (2) at infinite temperature
// with the Heisenberg-picture operator W(t) = e^{iH^dag t} W e^{-iHt}, i.e.
//   F_P(t) = <psi_P| e^{iH^dag t} chi_a e^{-iH_QQ t} chi_b e^{iH^dag_PP t}
//            chi_a e^{-iH_QQ t} chi_b |psi_P>,   F = F_U + F_D,
// which is the beta = 0 OTOC of syk_otoc when M = 0.  H^dag is a second handle
// built from the first by syk_terms_adjoint: a block string
// A = w S, S[m, m ^ x] = (-1)^{popc(z & m)}, has A^dag = conj(w) (-1)^{popc(x & z)} S.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "entry.h"
#include "kernels.cuh"

namespace syk {
namespace {

void check_args(int N, int64_t T, const int32_t* quads, const double* J_re, const double* J_im, int rep) {
  SYK_REQUIRE(N >= 4 && N <= 64 && N % 2 == 0, "N must be even and in [4, 64]");
  SYK_REQUIRE(T >= 0 && T <= (int64_t(1) << 31) - 1, "T out of range");
  SYK_REQUIRE(T == 0 || (quads && J_re && J_im), "null quads, J_re or J_im");
  SYK_REQUIRE(rep == SYK_REP_JW || rep == SYK_REP_PAPER, "rep must be SYK_REP_JW or SYK_REP_PAPER");
}

struct HandleGuard {
  syk_terms_t* h = nullptr;
  ~HandleGuard() {
    if (h) syk_terms_destroy(h);
  }
};

syk_terms_t* build_adjoint(const syk_terms* h) {
  std::vector<BlockString> terms = h->terms;
  for (auto& t : terms) {
    const double sg = (__builtin_popcount(t.x & t.z) & 1) ? -1.0 : 1.0;
    const double f = t.imag ? -sg : sg;  // conj(i c) = -i c
    t.coef[0] *= f;
    t.coef[1] *= f;
    t.straggler = false;
  }
  const bool pauli = h->rep == SYK_REP_PAULI;
  syk_terms_t* a = make_handle(pauli ? 2 * h->L + 2 : h->N, h->dtype, pauli ? SYK_REP_JW : h->rep,
                               std::move(terms), h->n_input, h->n_real, h->n_xgroups, h->hermitian);
  if (pauli) {
    a->N = 0;
    a->rep = SYK_REP_PAULI;
  }
  return a;
}

void otoc_nh_run(const syk_terms* h, const syk_terms* hd, int a, int b, const double* tg, int n_t, int mode,
                 int n_states, uint64_t seed, const void* psi_opt, int m, double tol, int max_sub, double* F_raw,
                 double* otoc, KrylovResult& tot, cudaStream_t st) {
  const size_t esz = elem_bytes(h->dtype);
  const size_t vb = (static_cast<size_t>(h->D) * esz + 255) & ~size_t(255);
  const bool exact = mode == SYK_OTOC_EXACT_TRACE;
  const int rows = exact ? 1 : n_states;
  const int G = vec_grid(h);
  DeviceBuffer vecs(4 * vb);
  DeviceBuffer ws(std::max(krylov_ws_bytes(h, m, false), krylov_ws_bytes(hd, m, false)));
  DeviceBuffer small((2 * static_cast<size_t>(G) + 8) * sizeof(double) + static_cast<size_t>(rows) * n_t * 2 * sizeof(double));
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
  auto evolve = [&](const syk_terms* hh, int blk, double t, void* x) {
    KrylovResult r = krylov_evolve_one(hh, blk, 0.0, t, x, x, m, tol, max_sub, false, false, ws.p, st);
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
        if (s / h->D != P) continue;
        launch_basis_vector(h, u0, s % h->D, st);
      } else if (psi_opt) {
        const char* src = static_cast<const char*>(psi_opt) + (static_cast<size_t>(s) * 2 + P) * h->D * esz;
        SYK_CUDA(cudaMemcpyAsync(u0, src, h->D * esz, cudaMemcpyDeviceToDevice, st));
      } else {
        launch_random_state(h, seed, static_cast<uint64_t>(s), P, u0, st);
        launch_scale_inv_sqrt(h, u0, n2, st);
      }
      SYK_CUDA(cudaMemcpyAsync(bra, u0, h->D * esz, cudaMemcpyDeviceToDevice, st));
      double tprev = 0.0;
      for (int n = 0; n < n_t; ++n) {
        const double t = tg[n];
        if (t != tprev) evolve(h, P, t - tprev, bra);  // bra = e^{-iH t} psi_P
        tprev = t;
        launch_apply_chi(h, b, P, u0, k1, 1, st);
        evolve(h, Q, t, k1);    // e^{-iHt}
        launch_apply_chi(h, a, Q, k1, k2, 1, st);
        evolve(hd, P, -t, k2);  // e^{iH^dag t}
        launch_apply_chi(h, b, P, k2, k1, 1, st);
        evolve(h, Q, t, k1);
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

}  // namespace
}  // namespace syk

extern "C" {

int syk_compile_terms_complex_host(int N, int64_t T, const int32_t* quads, const double* J_re, const double* J_im,
                                   int rep, int64_t capacity, int64_t* n_terms, uint32_t* x, uint32_t* z,
                                   double* coef_U, double* coef_D, uint8_t* imag) {
  return syk::guard_call("syk_compile_terms_complex_host", [&] {
    syk::check_args(N, T, quads, J_re, J_im, rep);
    SYK_REQUIRE(n_terms != nullptr, "null n_terms");
    SYK_REQUIRE(capacity >= 0, "negative capacity");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_terms_complex(N, rep, T, quads, J_re, J_im, terms, n_real, n_x);
    *n_terms = static_cast<int64_t>(terms.size());
    const int64_t n = std::min<int64_t>(capacity, *n_terms);
    for (int64_t i = 0; i < n; ++i) {
      if (x) x[i] = terms[i].x;
      if (z) z[i] = terms[i].z;
      if (coef_U) coef_U[i] = terms[i].coef[0];
      if (coef_D) coef_D[i] = terms[i].coef[1];
      if (imag) imag[i] = terms[i].imag ? 1 : 0;
    }
  });
}

int syk_build_terms_complex(int N, int64_t T, const int32_t* quads, const double* J_re, const double* J_im, int dtype,
                            int rep, syk_terms_t** out) {
  return syk::guard_call("syk_build_terms_complex", [&] {
    SYK_REQUIRE(out != nullptr, "null output handle pointer");
    *out = nullptr;
    syk::check_args(N, T, quads, J_re, J_im, rep);
    SYK_REQUIRE(dtype == SYK_C64 || dtype == SYK_C128, "dtype must be SYK_C64 or SYK_C128");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_terms_complex(N, rep, T, quads, J_re, J_im, terms, n_real, n_x);
    bool hermitian = true;
    for (int64_t t = 0; t < T; ++t) hermitian = hermitian && J_im[t] == 0.0;
    *out = syk::make_handle(N, dtype, rep, std::move(terms), T, n_real, n_x, hermitian);
  });
}

int syk_terms_is_hermitian(const syk_terms_t* h, int* hermitian) {
  return syk::guard_call("syk_terms_is_hermitian", [&] {
    SYK_REQUIRE(h && hermitian, "null argument");
    *hermitian = h->hermitian ? 1 : 0;
  });
}

int syk_terms_adjoint(const syk_terms_t* h, syk_terms_t** out) {
  return syk::guard_call("syk_terms_adjoint", [&] {
    SYK_REQUIRE(h && out, "null argument");
    *out = nullptr;
    int dev = -1;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_REQUIRE(dev == h->device, "the current CUDA device is not the one the terms were built on");
    *out = syk::build_adjoint(h);
  });
}

int syk_otoc_nonhermitian(const syk_terms_t* h, int a, int b, const double* t_grid, int n_t, int mode, int n_states,
                          uint64_t seed, const void* psi_opt, const syk_krylov_params* p, double* F_raw, double* otoc,
                          syk_krylov_stats* stats, syk_stream_t stream) {
  return syk::guard_call("syk_otoc_nonhermitian", [&] {
    SYK_REQUIRE(h != nullptr, "null terms handle");
    int dev = -1;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_REQUIRE(dev == h->device, "the current CUDA device is not the one the terms were built on");
    SYK_REQUIRE(a >= 0 && a < h->N && b >= 0 && b < h->N, "Majorana index out of range [0, N)");
    SYK_REQUIRE(t_grid != nullptr && n_t >= 1, "need a time grid");
    for (int n = 0; n < n_t; ++n) {
      SYK_REQUIRE(std::isfinite(t_grid[n]), "non-finite time");
      if (n) SYK_REQUIRE(t_grid[n] >= t_grid[n - 1], "time grid must be non-decreasing");
    }
    SYK_REQUIRE(mode == SYK_OTOC_TYPICAL || mode == SYK_OTOC_EXACT_TRACE, "bad mode");
    if (mode == SYK_OTOC_TYPICAL) SYK_REQUIRE(n_states >= 1, "n_states must be >= 1");
    if (psi_opt) SYK_REQUIRE((reinterpret_cast<uintptr_t>(psi_opt) & 15) == 0, "psi_opt not 16-byte aligned");
    const syk::KrylovSettings k = syk::krylov_settings(h->dtype, p);
    SYK_REQUIRE(!k.reorth && !k.two_pass, "reorth and two_pass are not available here");
    syk::HandleGuard adj;
    adj.h = syk::build_adjoint(h);
    syk::KrylovResult tot;
    syk::otoc_nh_run(h, adj.h, a, b, t_grid, n_t, mode, n_states, seed, psi_opt, k.m, k.tol, k.max_sub, F_raw, otoc,
                     tot, reinterpret_cast<cudaStream_t>(stream));
    if (stats) {
      stats->matvecs = tot.matvecs;
      stats->substeps = tot.substeps;
      stats->err_est = tot.err;
    }
  });
}

}  // extern "C"
