// Pauli-string Hamiltonians on L qubits: the spin chains that the paper's
// conclusions name as the next use of its GPU machinery (e.g. the random-field
// Heisenberg chain of many-body-localisation studies), run through the same
// H psi, Lanczos and OTOC kernels as the SYK handles.  The supplement
// (Sec. I.A) keeps every operator as a list of Pauli strings with
// coefficients; here that list is given directly instead of being compiled
// from Majorana quadruples.
//
// A string is two masks (x, z): on qubit q, x_q alone = sigma_x, z_q alone =
// sigma_z, both = sigma_y = i sigma_x sigma_z.  So P(x, z) = i^k X^x Z^z with
// k = popc(x & z), and in the output-index form every kernel uses
//   (P psi)[m] = i^k (-1)^{popc(z & (m ^ x))} psi[m ^ x]
//              = (-i)^k (-1)^{popc(z & m)} psi[m ^ x].
//
// A Pauli handle is an ordinary handle (make_handle: syk_build_terms with no
// terms on N = 2L + 2, so D = 2^L, then the compiled strings and a re-plan
// that builds and uploads the pass plan and records).  It holds no Majoranas
// (N = 0), so the Majorana entry points refuse it, and its two block slots
// carry the same coefficients; every call here uses block 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "device_common.cuh"
#include "entry.h"
#include "kernels.cuh"

namespace syk {
namespace {

uint32_t qubit_mask(int L) { return L >= 32 ? 0xFFFFFFFFu : ((1u << L) - 1u); }

// (-i)^k for k = popc(x & z): real +1, imag -1, real -1, imag +1.
void string_phase(uint32_t x, uint32_t z, bool& imag, double& sign) {
  const int k = __builtin_popcount(x & z) & 3;
  imag = (k & 1) != 0;
  sign = (k == 0 || k == 3) ? 1.0 : -1.0;
}

void compile_pauli(int L, int64_t T, const uint32_t* x, const uint32_t* z, const double* h,
                   std::vector<BlockString>& out, int64_t& n_real, int64_t& n_xgroups) {
  SYK_REQUIRE(L >= 1 && L <= 31, "n_qubits must be in [1, 31]");
  SYK_REQUIRE(T >= 0 && T <= (int64_t(1) << 31) - 1, "T out of range");
  SYK_REQUIRE(T == 0 || (x && z && h), "null x, z or h");
  const uint32_t lim = qubit_mask(L);
  std::map<std::pair<uint32_t, uint32_t>, size_t> index;  // (x, z) -> string (imag follows from x & z)
  out.clear();
  for (int64_t t = 0; t < T; ++t) {
    SYK_REQUIRE((x[t] & ~lim) == 0 && (z[t] & ~lim) == 0, "Pauli string acts on a qubit >= n_qubits");
    SYK_REQUIRE(std::isfinite(h[t]), "non-finite coefficient");
    bool imag;
    double sign;
    string_phase(x[t], z[t], imag, sign);
    const double c = sign * h[t];
    auto key = std::make_pair(x[t], z[t]);
    auto it = index.find(key);
    if (it == index.end()) {
      BlockString b;
      b.x = x[t];
      b.z = z[t];
      b.imag = imag;
      b.coef[0] = b.coef[1] = c;
      index.emplace(key, out.size());
      out.push_back(b);
    } else {
      out[it->second].coef[0] += c;
      out[it->second].coef[1] += c;
    }
  }
  out.erase(std::remove_if(out.begin(), out.end(), [](const BlockString& b) { return b.coef[0] == 0.0; }),
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

void check_pauli_handle(const syk_terms* h) {
  SYK_REQUIRE(h != nullptr, "null terms handle");
  SYK_REQUIRE(h->rep == SYK_REP_PAULI, "not a Pauli-string handle (build it with syk_build_pauli_terms)");
  int dev = -1;
  SYK_CUDA(cudaGetDevice(&dev));
  SYK_REQUIRE(dev == h->device, "the current CUDA device is not the one the terms were built on");
}

void check_ptr(const void* p, const char* what) {
  SYK_REQUIRE(p != nullptr, std::string("null pointer: ") + what);
  SYK_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0, std::string("pointer not 16-byte aligned: ") + what);
}

bool overlaps(const void* a, const void* b, size_t n) {
  const char* p = static_cast<const char*>(a);
  const char* q = static_cast<const char*>(b);
  return p < q + n && q < p + n;
}

// out[m] = (cre + i cim) (-1)^{popc(z & m)} psi[m ^ x], one state per blockIdx.y.
template <typename Real>
__global__ void k_pauli(const typename CT<Real>::T* psi, typename CT<Real>::T* out, uint64_t D, uint32_t x,
                        uint32_t z, double cre, double cim) {
  using C = typename CT<Real>::T;
  const uint64_t soff = static_cast<uint64_t>(blockIdx.y) * D;
  const Real re = static_cast<Real>(cre), im = static_cast<Real>(cim);
  for (uint64_t m = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; m < D;
       m += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t mm = static_cast<uint32_t>(m);
    const C v = psi[soff + (mm ^ x)];
    const uint32_t s = __popc(z & mm) & 1u;
    const Real a = sgnflip(re, s), b = sgnflip(im, s);
    C o;
    o.x = fma_(a, v.x, -mul_(b, v.y));
    o.y = fma_(a, v.y, mul_(b, v.x));
    out[soff + m] = o;
  }
}

void launch_pauli(const syk_terms* h, uint32_t x, uint32_t z, const void* psi, void* out, int64_t nstates,
                  cudaStream_t st) {
  bool imag;
  double sign;
  string_phase(x, z, imag, sign);
  const double cre = imag ? 0.0 : sign, cim = imag ? sign : 0.0;
  const int grid = vec_grid(h);
  for (int64_t s0 = 0; s0 < nstates; s0 += 65535) {
    const unsigned gy = static_cast<unsigned>(std::min<int64_t>(65535, nstates - s0));
    const uint64_t off = static_cast<uint64_t>(s0) * h->D;
    if (h->dtype == SYK_C128)
      k_pauli<double><<<dim3(grid, gy), 256, 0, st>>>(static_cast<const double2*>(psi) + off,
                                                      static_cast<double2*>(out) + off, h->D, x, z, cre, cim);
    else
      k_pauli<float><<<dim3(grid, gy), 256, 0, st>>>(static_cast<const float2*>(psi) + off,
                                                     static_cast<float2*>(out) + off, h->D, x, z, cre, cim);
  }
  SYK_CUDA(cudaGetLastError());
}

// The single-state chain of Eq. (2) with W, V for each state (or basis state),
// on the handle's one state space (block 0):
//   u0  = e^{-bH/8} psi                     (once per state),
//   bra = e^{-(it_n + b/8)H} psi             (advanced by e^{-i dt H}),
//   ket = W e^{-(it+b/4)H} V e^{(it-b/4)H} W e^{-(it+b/4)H} V u0  (per t),
//   F(t_n) = <bra|ket>.
void pauli_otoc_run(const syk_terms* h, uint32_t wx, uint32_t wz, uint32_t vx, uint32_t vz, double beta,
                    const double* tg, int n_t, int mode, int n_states, uint64_t seed, const void* psi_opt, int m,
                    double tol, int max_sub, bool reorth, bool two_pass, double* F_raw, double* otoc,
                    KrylovResult& tot, cudaStream_t st) {
  const size_t esz = elem_bytes(h->dtype);
  const size_t vb = (static_cast<size_t>(h->D) * esz + 255) & ~size_t(255);
  const bool exact = mode == SYK_OTOC_EXACT_TRACE;
  const int rows = exact ? 1 : n_states;
  const int G = vec_grid(h);
  DeviceBuffer vecs(4 * vb);
  DeviceBuffer ws(krylov_ws_bytes(h, m, two_pass));
  DeviceBuffer small((2 * static_cast<size_t>(G) + 8) * sizeof(double) +
                     static_cast<size_t>(rows) * n_t * 2 * sizeof(double));
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

  auto evolve = [&](double tau, double t, void* x) {
    KrylovResult r = krylov_evolve_one(h, 0, tau, t, x, x, m, tol, max_sub, reorth, two_pass, ws.p, st);
    tot.matvecs += r.matvecs;
    tot.substeps += r.substeps;
    tot.err += r.err;
  };

  const int64_t n_outer = exact ? h->D : n_states;
  const double scale = exact ? 1.0 / static_cast<double>(h->D) : 1.0;
  for (int64_t s = 0; s < n_outer; ++s) {
    const int row = exact ? 0 : static_cast<int>(s);
    if (exact) {
      launch_basis_vector(h, u0, s, st);
    } else if (psi_opt) {
      const char* src = static_cast<const char*>(psi_opt) + static_cast<size_t>(s) * h->D * esz;
      SYK_CUDA(cudaMemcpyAsync(u0, src, h->D * esz, cudaMemcpyDeviceToDevice, st));
    } else {
      launch_random_state(h, seed, static_cast<uint64_t>(s), 0, u0, st);
      launch_norm_partials(h, u0, partial, st);
      launch_sum_finalize(partial, G, n2, 0, st);
      launch_scale_inv_sqrt(h, u0, n2, st);
    }
    evolve(beta / 8.0, 0.0, u0);
    SYK_CUDA(cudaMemcpyAsync(bra, u0, h->D * esz, cudaMemcpyDeviceToDevice, st));
    double tprev = 0.0;
    for (int n = 0; n < n_t; ++n) {
      const double t = tg[n];
      if (t != tprev) evolve(0.0, t - tprev, bra);
      tprev = t;
      launch_pauli(h, vx, vz, u0, k1, 1, st);
      evolve(beta / 4.0, t, k1);
      launch_pauli(h, wx, wz, k1, k2, 1, st);
      evolve(beta / 4.0, -t, k2);
      launch_pauli(h, vx, vz, k2, k1, 1, st);
      evolve(beta / 4.0, t, k1);
      launch_pauli(h, wx, wz, k1, k2, 1, st);
      launch_zdot_partials(h, bra, k2, partial, st);
      launch_zdot_finalize(partial, G, Fdev + (static_cast<size_t>(row) * n_t + n) * 2, scale, 1, st);
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

int syk_compile_pauli_host(int n_qubits, int64_t T, const uint32_t* x, const uint32_t* z, const double* h,
                           int64_t capacity, int64_t* n_terms, uint32_t* x_out, uint32_t* z_out, double* coef,
                           uint8_t* imag) {
  return syk::guard_call("syk_compile_pauli_host", [&] {
    SYK_REQUIRE(n_terms != nullptr, "null n_terms");
    SYK_REQUIRE(capacity >= 0, "negative capacity");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_pauli(n_qubits, T, x, z, h, terms, n_real, n_x);
    *n_terms = static_cast<int64_t>(terms.size());
    const int64_t n = std::min<int64_t>(capacity, *n_terms);
    for (int64_t i = 0; i < n; ++i) {
      if (x_out) x_out[i] = terms[i].x;
      if (z_out) z_out[i] = terms[i].z;
      if (coef) coef[i] = terms[i].coef[0];
      if (imag) imag[i] = terms[i].imag ? 1 : 0;
    }
  });
}

int syk_build_pauli_terms(int n_qubits, int64_t T, const uint32_t* x, const uint32_t* z, const double* h,
                          int dtype, syk_terms_t** out) {
  return syk::guard_call("syk_build_pauli_terms", [&] {
    SYK_REQUIRE(out != nullptr, "null output handle pointer");
    *out = nullptr;
    SYK_REQUIRE(dtype == SYK_C64 || dtype == SYK_C128, "dtype must be SYK_C64 or SYK_C128");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_pauli(n_qubits, T, x, z, h, terms, n_real, n_x);
    // N = 2 n_qubits + 2 Majoranas give D = 2^{N/2 - 1} = 2^n_qubits amplitudes
    syk_terms_t* raw = syk::make_handle(2 * n_qubits + 2, dtype, SYK_REP_JW, std::move(terms), T, n_real, n_x, true);
    raw->N = 0;  // no Majoranas: the chi / OTOC / batch entry points refuse the handle
    raw->rep = SYK_REP_PAULI;
    *out = raw;
  });
}

int syk_apply_pauli(const syk_terms_t* h, uint32_t x, uint32_t z, const void* psi, void* out, int64_t nstates,
                    syk_stream_t stream) {
  return syk::guard_call("syk_apply_pauli", [&] {
    syk::check_pauli_handle(h);
    const uint32_t lim = syk::qubit_mask(h->L);
    SYK_REQUIRE((x & ~lim) == 0 && (z & ~lim) == 0, "Pauli string acts on a qubit >= n_qubits");
    SYK_REQUIRE(nstates >= 1, "nstates must be >= 1");
    syk::check_ptr(psi, "psi");
    syk::check_ptr(out, "out");
    const size_t bytes = static_cast<size_t>(nstates) * h->D * syk::elem_bytes(h->dtype);
    if (x != 0 || psi != out)
      SYK_REQUIRE(!syk::overlaps(psi, out, bytes), "out may alias psi only exactly and only for x = 0");
    syk::launch_pauli(h, x, z, psi, out, nstates, reinterpret_cast<cudaStream_t>(stream));
  });
}

int syk_pauli_otoc(const syk_terms_t* h, uint32_t w_x, uint32_t w_z, uint32_t v_x, uint32_t v_z, double beta,
                   const double* t_grid, int n_t, int mode, int n_states, uint64_t seed, const void* psi_opt,
                   const syk_krylov_params* p, double* F_raw, double* otoc, syk_krylov_stats* stats,
                   syk_stream_t stream) {
  return syk::guard_call("syk_pauli_otoc", [&] {
    syk::check_pauli_handle(h);
    const uint32_t lim = syk::qubit_mask(h->L);
    SYK_REQUIRE(((w_x | w_z | v_x | v_z) & ~lim) == 0, "Pauli string acts on a qubit >= n_qubits");
    SYK_REQUIRE(std::isfinite(beta) && beta >= 0, "beta must be finite and >= 0");
    SYK_REQUIRE(t_grid != nullptr && n_t >= 1, "need a time grid");
    for (int n = 0; n < n_t; ++n) {
      SYK_REQUIRE(std::isfinite(t_grid[n]), "non-finite time");
      if (n) SYK_REQUIRE(t_grid[n] >= t_grid[n - 1], "time grid must be non-decreasing");
    }
    SYK_REQUIRE(mode == SYK_OTOC_TYPICAL || mode == SYK_OTOC_EXACT_TRACE, "bad mode");
    if (mode == SYK_OTOC_TYPICAL) SYK_REQUIRE(n_states >= 1, "n_states must be >= 1");
    if (psi_opt) syk::check_ptr(psi_opt, "psi_opt");
    const syk::KrylovSettings k = syk::krylov_settings(h->dtype, p);
    syk::KrylovResult tot;
    syk::pauli_otoc_run(h, w_x, w_z, v_x, v_z, beta, t_grid, n_t, mode, n_states, seed, psi_opt, k.m, k.tol,
                        k.max_sub, k.reorth, k.two_pass, F_raw, otoc, tot, reinterpret_cast<cudaStream_t>(stream));
    if (stats) {
      stats->matvecs = tot.matvecs;
      stats->substeps = tot.substeps;
      stats->err_est = tot.err;
    }
  });
}

}  // extern "C"
