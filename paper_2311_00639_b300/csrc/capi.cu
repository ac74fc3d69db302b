// extern "C" entry points of libsyk (declared in include/syk.h).  Every call
// validates its arguments, runs inside a try block and maps failures to a
// status code plus a per-thread message; no exception crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "entry.h"
#include "kernels.cuh"

namespace syk {
void otoc_run(const syk_terms* h, int a, int b, double beta, const double* tg, int n_t, int mode, int n_states,
              uint64_t seed, const void* psi_opt, int m, double tol, int max_sub, bool reorth, bool two_pass,
              double* F_raw, double* otoc, KrylovResult& tot, cudaStream_t st);
}

namespace {

thread_local std::string g_last_error;

template <typename F>
int guarded(const char* fn, F&& f) {
  try {
    f();
    return SYK_OK;
  } catch (const syk::Error& e) {
    g_last_error = std::string(fn) + ": " + e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = std::string(fn) + ": host allocation failed";
    return SYK_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = std::string(fn) + ": " + e.what();
    return SYK_EINVAL;
  } catch (...) {
    g_last_error = std::string(fn) + ": unknown failure";
    return SYK_EINVAL;
  }
}

void check_handle(const syk_terms* h) {
  SYK_REQUIRE(h != nullptr, "null terms handle");
  int dev = -1;
  SYK_CUDA(cudaGetDevice(&dev));
  SYK_REQUIRE(dev == h->device, "the current CUDA device is not the one the terms were built on");
}

void check_vec(const void* p, const char* what) {
  SYK_REQUIRE(p != nullptr, std::string("null pointer: ") + what);
  SYK_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0, std::string("pointer not 16-byte aligned: ") + what);
}

bool overlap(const void* a, const void* b, size_t n) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + n && y < x + n;
}

struct Params {
  int m;
  double tol;
  int max_sub;
  bool reorth, two_pass;
};

Params resolve(const syk_terms* h, const syk_krylov_params* p) {
  const syk::KrylovSettings k = syk::krylov_settings(h->dtype, p);  // defaults and checks (entry.h)
  Params r;
  r.m = k.m;
  r.tol = k.tol;
  r.max_sub = k.max_sub;
  r.reorth = k.reorth;
  r.two_pass = k.two_pass;
  return r;
}

}  // namespace

namespace {
void upload_table(syk_terms* h) {
    const size_t n = h->terms.size();
    const size_t rb = h->dtype == SYK_C128 ? 8 : 4;
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    std::vector<syk::TermF> rec[2];
    h->n_runs = syk::build_records(h->terms, h->passes, rec, &h->n_merges);
    syk::plan_split(h);  // its CTA count depends on whether the records merge terms
    // the passes, then one more: the last pass's tile order with no terms, run
    // for the epilogue after a split last pass
    const size_t pass_bytes = up((h->passes.size() + 1) * sizeof(syk::PassPlan));
    const size_t rec_bytes = up((n + 1) * sizeof(syk::TermF));  // + one zero record: prefetch past the end
    const size_t zi_bytes = up(std::max<size_t>(n, 1) * 4);
    const size_t bytes = 2 * up(std::max<size_t>(n, 1) * 4) + 2 * up(std::max<size_t>(n, 1) * rb) + pass_bytes + 256 +
                         2 * rec_bytes + zi_bytes;
    std::vector<char> host(bytes, 0);
    char* p = host.data();
    uint32_t* hx = reinterpret_cast<uint32_t*>(p);
    uint32_t* hz = reinterpret_cast<uint32_t*>(p + up(std::max<size_t>(n, 1) * 4));
    char* hc0 = p + 2 * up(std::max<size_t>(n, 1) * 4);
    char* hc1 = hc0 + up(std::max<size_t>(n, 1) * rb);
    char* hp = hc1 + up(std::max<size_t>(n, 1) * rb);
    std::memcpy(hp, h->passes.data(), h->passes.size() * sizeof(syk::PassPlan));
    if (!h->passes.empty()) {
      const syk::PassPlan tail = syk::tail_pass(h->passes.back());
      std::memcpy(hp + h->passes.size() * sizeof(syk::PassPlan), &tail, sizeof(tail));
    }
    char* hr0 = hp + pass_bytes + 256;
    char* hr1 = hr0 + rec_bytes;
    uint32_t* hzi = reinterpret_cast<uint32_t*>(hr1 + rec_bytes);
    for (size_t i = 0; i < n; ++i) hzi[i] = h->terms[i].z | (h->terms[i].imag ? 0x80000000u : 0u);
    std::memcpy(hr0, rec[0].data(), (n + 1) * sizeof(syk::TermF));
    std::memcpy(hr1, rec[1].data(), (n + 1) * sizeof(syk::TermF));
    for (size_t i = 0; i < n; ++i) {
      hx[i] = h->terms[i].x;
      hz[i] = h->terms[i].z;
      for (int b = 0; b < 2; ++b) {
        char* dst = (b ? hc1 : hc0) + i * rb;
        if (h->dtype == SYK_C128) {
          const double v = h->terms[i].coef[b];
          std::memcpy(dst, &v, 8);
        } else {
          const float v = static_cast<float>(h->terms[i].coef[b]);
          std::memcpy(dst, &v, 4);
        }
      }
    }
    if (h->d_mem) {
      SYK_CUDA(cudaDeviceSynchronize());
      cudaFree(h->d_mem);
      h->d_mem = nullptr;
    }
    h->clear_graphs();  // captured evolves point into the old table
    if (cudaMalloc(&h->d_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw syk::Error(SYK_ENOMEM, "device allocation of the term table failed");
    }
    SYK_CUDA(cudaMemcpy(h->d_mem, host.data(), bytes, cudaMemcpyHostToDevice));
    char* d = static_cast<char*>(h->d_mem);
    h->d_x = reinterpret_cast<uint32_t*>(d);
    h->d_z = reinterpret_cast<uint32_t*>(d + (reinterpret_cast<char*>(hz) - p));
    h->d_coef[0] = d + (hc0 - p);
    h->d_coef[1] = d + (hc1 - p);
    h->d_passes = reinterpret_cast<syk::PassPlan*>(d + (hp - p));
    h->d_pass_tail = h->d_passes + h->passes.size();
    if (h->d_split_ws) {
      cudaFree(h->d_split_ws);
      h->d_split_ws = nullptr;
    }
    if (h->split_ws_bytes && cudaMalloc(&h->d_split_ws, h->split_ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      throw syk::Error(SYK_ENOMEM, "device allocation of the split-pass workspace failed");
    }
    h->d_err = reinterpret_cast<int*>(d + (hp - p) + pass_bytes);  // zeroed with the host image
    h->d_sched = reinterpret_cast<unsigned long long*>(d + (hp - p) + pass_bytes + 64);  // likewise
    h->d_termf[0] = reinterpret_cast<syk::TermF*>(d + (hr0 - p));
    h->d_termf[1] = reinterpret_cast<syk::TermF*>(d + (hr1 - p));
    h->d_zi = reinterpret_cast<uint32_t*>(d + (reinterpret_cast<char*>(hzi) - p));
}

}  // namespace

namespace syk {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace syk

extern "C" {

const char* syk_version(void) { return "libsyk 0.1 (sm_103a)"; }

int syk_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return SYK_EINVAL;
  std::strncpy(buf, g_last_error.c_str(), n - 1);
  buf[n - 1] = '\0';
  return SYK_OK;
}

int syk_build_terms(int N, int64_t T, const int32_t* quads, const double* J, int dtype, int rep,
                    syk_terms_t** out) {
  return guarded("syk_build_terms", [&] {
    SYK_REQUIRE(out != nullptr, "null output handle pointer");
    *out = nullptr;
    SYK_REQUIRE(N >= 4 && N <= 64 && N % 2 == 0, "N must be even and in [4, 64]");
    SYK_REQUIRE(T >= 0 && T <= (int64_t(1) << 31) - 1, "T out of range");
    SYK_REQUIRE(T == 0 || (quads && J), "null quads or J");
    SYK_REQUIRE(dtype == SYK_C64 || dtype == SYK_C128, "dtype must be SYK_C64 or SYK_C128");
    SYK_REQUIRE(rep == SYK_REP_JW || rep == SYK_REP_PAPER, "rep must be SYK_REP_JW or SYK_REP_PAPER");
    auto h = std::make_unique<syk_terms>();
    h->N = N;
    h->L = N / 2 - 1;
    h->D = int64_t(1) << h->L;
    h->dtype = dtype;
    h->rep = rep;
    h->n_input = T;
    syk::compile_terms(N, rep, T, quads, J, h->terms, h->n_real, h->n_xgroups);
    for (const auto& t : h->terms) h->sum_abs += std::max(std::fabs(t.coef[0]), std::fabs(t.coef[1]));
    for (int n = 0; n < N; ++n) h->chi[n] = syk::compile_chi(N, rep, n);
    h->passes = syk::plan_passes(h->terms, h->L, syk::elem_bytes(dtype), syk::default_l2_budget(dtype),
                                   syk::default_hbm_ratio(dtype));
    SYK_CUDA(cudaGetDevice(&h->device));
    SYK_CUDA(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device));
    upload_table(h.get());
    *out = h.release();
  });
}

int syk_terms_destroy(syk_terms_t* h) {
  return guarded("syk_terms_destroy", [&] {
    delete h;  // frees the device table
  });
}

int syk_terms_get_info(const syk_terms_t* h, syk_terms_info* info) {
  return guarded("syk_terms_get_info", [&] {
    SYK_REQUIRE(h && info, "null argument");
    info->N = h->N;
    info->L = h->L;
    info->dtype = h->dtype;
    info->rep = h->rep;
    info->D = h->D;
    info->n_input = h->n_input;
    info->n_terms = static_cast<int64_t>(h->terms.size());
    info->n_real = h->n_real;
    info->n_xgroups = h->n_xgroups;
    info->sum_abs_coef = h->sum_abs;
    info->n_passes = static_cast<int64_t>(h->passes.size());
    int e = 0;
    SYK_CUDA(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    info->device_error = e;
    info->n_tile_reads = h->dtype == SYK_C64 ? h->n_runs : static_cast<int64_t>(h->terms.size());
    info->n_merged = h->dtype == SYK_C64 ? h->n_merges : 0;
  });
}

int syk_terms_replan(syk_terms_t* h, size_t l2_budget_bytes, double straggler_ratio) {
  return guarded("syk_terms_replan", [&] {
    check_handle(h);
    SYK_REQUIRE(l2_budget_bytes == 0 || l2_budget_bytes >= 4096, "l2_budget_bytes must be 0 or >= 4096");
    SYK_REQUIRE(std::isfinite(straggler_ratio) && straggler_ratio >= 0, "straggler_ratio must be >= 0");
    if (l2_budget_bytes == 0) {  // the default plan of the handle's dtype
      l2_budget_bytes = syk::default_l2_budget(h->dtype);
      straggler_ratio = syk::default_hbm_ratio(h->dtype);
    }
    h->passes = syk::plan_passes(h->terms, h->L, syk::elem_bytes(h->dtype), l2_budget_bytes, straggler_ratio);
    upload_table(h);
  });
}

int syk_terms_export(const syk_terms_t* h, uint32_t* x, uint32_t* z, double* cU, double* cD, uint8_t* imag) {
  return guarded("syk_terms_export", [&] {
    SYK_REQUIRE(h, "null terms handle");
    for (size_t i = 0; i < h->terms.size(); ++i) {
      const auto& t = h->terms[i];
      if (x) x[i] = t.x;
      if (z) z[i] = t.z;
      if (cU) cU[i] = t.coef[0];
      if (cD) cD[i] = t.coef[1];
      if (imag) imag[i] = t.imag ? 1 : 0;
    }
  });
}

int syk_compile_terms_host(int N, int64_t T, const int32_t* quads, const double* J, int rep, int64_t capacity,
                           int64_t* n_terms, uint32_t* x, uint32_t* z, double* cU, double* cD, uint8_t* imag) {
  return guarded("syk_compile_terms_host", [&] {
    SYK_REQUIRE(N >= 4 && N <= 64 && N % 2 == 0, "N must be even and in [4, 64]");
    SYK_REQUIRE(T >= 0 && (T == 0 || (quads && J)), "bad T or null quads/J");
    SYK_REQUIRE(rep == SYK_REP_JW || rep == SYK_REP_PAPER, "rep must be SYK_REP_JW or SYK_REP_PAPER");
    SYK_REQUIRE(n_terms != nullptr, "null n_terms");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_terms(N, rep, T, quads, J, terms, n_real, n_x);
    *n_terms = static_cast<int64_t>(terms.size());
    const int64_t n = std::min<int64_t>(capacity, *n_terms);
    for (int64_t i = 0; i < n; ++i) {
      if (x) x[i] = terms[i].x;
      if (z) z[i] = terms[i].z;
      if (cU) cU[i] = terms[i].coef[0];
      if (cD) cD[i] = terms[i].coef[1];
      if (imag) imag[i] = terms[i].imag ? 1 : 0;
    }
  });
}

int syk_plan_host(int N, int64_t T, const int32_t* quads, const double* J, int dtype, int rep,
                  size_t l2_budget_bytes, double straggler_ratio, int n_sm, syk_plan_host_out* out) {
  return guarded("syk_plan_host", [&] {
    SYK_REQUIRE(N >= 4 && N <= 64 && N % 2 == 0, "N must be even and in [4, 64]");
    SYK_REQUIRE(T >= 0 && T <= (int64_t(1) << 31) - 1, "T out of range");
    SYK_REQUIRE(T == 0 || (quads && J), "null quads or J");
    SYK_REQUIRE(rep == SYK_REP_JW || rep == SYK_REP_PAPER, "rep must be SYK_REP_JW or SYK_REP_PAPER");
    std::vector<syk::BlockString> terms;
    int64_t n_real = 0, n_x = 0;
    syk::compile_terms(N, rep, T, quads, J, terms, n_real, n_x);
    syk::plan_view(std::move(terms), N / 2 - 1, dtype, l2_budget_bytes, straggler_ratio, n_sm, out);
  });
}

int syk_compile_chi_host(int N, int rep, int n, uint32_t* x, uint32_t* z, double* re, double* im) {
  return guarded("syk_compile_chi_host", [&] {
    SYK_REQUIRE(N >= 4 && N <= 64 && N % 2 == 0, "N must be even and in [4, 64]");
    SYK_REQUIRE(n >= 0 && n < N, "Majorana index out of range [0, N)");
    SYK_REQUIRE(rep == SYK_REP_JW || rep == SYK_REP_PAPER, "rep must be SYK_REP_JW or SYK_REP_PAPER");
    SYK_REQUIRE(x && z && re && im, "null output");
    const syk::ChiString c = syk::compile_chi(N, rep, n);
    *x = c.x;
    *z = c.z;
    for (int P = 0; P < 2; ++P) {
      re[P] = c.re[P];
      im[P] = c.im[P];
    }
  });
}

int syk_apply_H(const syk_terms_t* h, int block, const void* psi, void* out, int64_t nstates,
                syk_stream_t stream) {
  return guarded("syk_apply_H", [&] {
    check_handle(h);
    SYK_REQUIRE(block == 0 || block == 1, "block must be SYK_BLOCK_U or SYK_BLOCK_D");
    SYK_REQUIRE(nstates >= 1, "nstates must be >= 1");
    check_vec(psi, "psi");
    check_vec(out, "out");
    const size_t bytes = static_cast<size_t>(nstates) * h->D * syk::elem_bytes(h->dtype);
    SYK_REQUIRE(!overlap(psi, out, bytes), "out must not overlap psi");
    syk::launch_apply_H(h, block, psi, out, nstates, reinterpret_cast<cudaStream_t>(stream));
  });
}

int syk_apply_chi(const syk_terms_t* h, int i, int from_block, const void* psi, void* out, int64_t nstates,
                  syk_stream_t stream) {
  return guarded("syk_apply_chi", [&] {
    check_handle(h);
    SYK_REQUIRE(i >= 0 && i < h->N, "Majorana index out of range [0, N)");
    SYK_REQUIRE(from_block == 0 || from_block == 1, "from_block must be SYK_BLOCK_U or SYK_BLOCK_D");
    SYK_REQUIRE(nstates >= 1, "nstates must be >= 1");
    check_vec(psi, "psi");
    check_vec(out, "out");
    const size_t bytes = static_cast<size_t>(nstates) * h->D * syk::elem_bytes(h->dtype);
    if (h->chi[i].x != 0 || psi != out)
      SYK_REQUIRE(!overlap(psi, out, bytes), "out may alias psi only exactly and only for a diagonal Majorana");
    syk::launch_apply_chi(h, i, from_block, psi, out, nstates, reinterpret_cast<cudaStream_t>(stream));
  });
}

int syk_random_state(const syk_terms_t* h, uint64_t seed, uint64_t state_id, void* psi_U, void* psi_D,
                     syk_stream_t stream) {
  return guarded("syk_random_state", [&] {
    check_handle(h);
    if (psi_U) check_vec(psi_U, "psi_U");
    if (psi_D) check_vec(psi_D, "psi_D");
    if (psi_U) syk::launch_random_state(h, seed, state_id, 0, psi_U, reinterpret_cast<cudaStream_t>(stream));
    if (psi_D) syk::launch_random_state(h, seed, state_id, 1, psi_D, reinterpret_cast<cudaStream_t>(stream));
  });
}

size_t syk_krylov_workspace_bytes(const syk_terms_t* h, const syk_krylov_params* p) {
  size_t out = 0;
  const int rc = guarded("syk_krylov_workspace_bytes", [&] {
    SYK_REQUIRE(h, "null terms handle");
    const Params r = resolve(h, p);
    out = syk::krylov_ws_bytes(h, r.m, r.two_pass);
  });
  return rc == SYK_OK ? out : 0;
}

int syk_krylov_evolve(const syk_terms_t* h, int block, double tau, double t, const void* x, void* y,
                      int64_t nstates, const syk_krylov_params* p, void* workspace, size_t ws_bytes,
                      syk_krylov_stats* stats, syk_stream_t stream) {
  return guarded("syk_krylov_evolve", [&] {
    check_handle(h);
    SYK_REQUIRE(block == 0 || block == 1, "block must be SYK_BLOCK_U or SYK_BLOCK_D");
    SYK_REQUIRE(std::isfinite(tau) && std::isfinite(t), "tau and t must be finite");
    SYK_REQUIRE(nstates >= 1, "nstates must be >= 1");
    check_vec(x, "x");
    check_vec(y, "y");
    const Params r = resolve(h, p);
    SYK_REQUIRE(workspace != nullptr, "null workspace");
    SYK_REQUIRE(ws_bytes >= syk::krylov_ws_bytes(h, r.m, r.two_pass), "workspace too small");
    const size_t vb = static_cast<size_t>(h->D) * syk::elem_bytes(h->dtype);
    SYK_REQUIRE(x == y || !overlap(x, y, nstates * vb), "y must either equal x or not overlap it");
    SYK_REQUIRE(!overlap(workspace, x, nstates * vb) && !overlap(workspace, y, nstates * vb),
                "workspace overlaps x or y");
    syk::KrylovResult tot;
    auto st = reinterpret_cast<cudaStream_t>(stream);
    syk::krylov_totals_reset(workspace, st);
    for (int64_t s = 0; s < nstates; ++s) {
      const char* xs = static_cast<const char*>(x) + s * vb;
      char* ys = static_cast<char*>(y) + s * vb;
      auto r1 = syk::krylov_evolve_one(h, block, tau, t, xs, ys, r.m, r.tol, r.max_sub, r.reorth, r.two_pass,
                                       workspace, st);
      tot.matvecs += r1.matvecs;
      tot.substeps += r1.substeps;
      tot.err += r1.err;
    }
    syk::krylov_totals_collect(workspace, st, tot);  // one synchronisation for the whole call
    if (stats) {
      stats->matvecs = tot.matvecs;
      stats->substeps = tot.substeps;
      stats->err_est = tot.err;
    }
  });
}

int syk_otoc(const syk_terms_t* h, int a, int b, double beta, const double* t_grid, int n_t, int mode,
             int n_states, uint64_t seed, const void* psi_opt, const syk_krylov_params* p, double* F_raw,
             double* otoc, syk_krylov_stats* stats, syk_stream_t stream) {
  return guarded("syk_otoc", [&] {
    check_handle(h);
    SYK_REQUIRE(a >= 0 && a < h->N && b >= 0 && b < h->N, "Majorana index out of range [0, N)");
    SYK_REQUIRE(std::isfinite(beta) && beta >= 0, "beta must be finite and >= 0");
    SYK_REQUIRE(t_grid != nullptr && n_t >= 1, "need a time grid");
    for (int n = 0; n < n_t; ++n) {
      SYK_REQUIRE(std::isfinite(t_grid[n]), "non-finite time");
      if (n) SYK_REQUIRE(t_grid[n] >= t_grid[n - 1], "time grid must be non-decreasing");
    }
    SYK_REQUIRE(mode == SYK_OTOC_TYPICAL || mode == SYK_OTOC_EXACT_TRACE, "bad mode");
    if (mode == SYK_OTOC_TYPICAL) SYK_REQUIRE(n_states >= 1, "n_states must be >= 1");
    if (psi_opt) check_vec(psi_opt, "psi_opt");
    const Params r = resolve(h, p);
    syk::KrylovResult tot;
    syk::otoc_run(h, a, b, beta, t_grid, n_t, mode, n_states, seed, psi_opt, r.m, r.tol, r.max_sub, r.reorth,
                  r.two_pass, F_raw, otoc, tot, reinterpret_cast<cudaStream_t>(stream));
    if (stats) {
      stats->matvecs = tot.matvecs;
      stats->substeps = tot.substeps;
      stats->err_est = tot.err;
    }
  });
}

}  // extern "C"
