// syk_otoc_exact_trace_batched: the exact trace of Eq. (2) as the sum of the
// single-state OTOC over all 2D basis states of both parity blocks, each basis
// state one job of the batched engine (basis_index = g).  The per-job curves
// are kept and summed on the host in the order g = 0 .. 2D-1 (FP64), so the
// result does not depend on the order in which jobs finish.
#include <algorithm>
#include <cmath>
#include <vector>

#include "entry.h"

extern "C" int syk_otoc_exact_trace_batched(const syk_terms_t* h, int n_pairs, const int32_t* pairs, double beta,
                                            const double* t_grid, int n_t, int max_slots, size_t max_bytes,
                                            const syk_krylov_params* p, double* F_out, double* otoc_out,
                                            syk_krylov_stats* stats) {
  syk_batch_t* b = nullptr;
  const int rc = syk::guard_call("syk_otoc_exact_trace_batched", [&] {
    SYK_REQUIRE(h != nullptr && pairs != nullptr && t_grid != nullptr, "null argument");
    SYK_REQUIRE(n_pairs >= 1 && n_t >= 1, "need at least one pair and one time");
    SYK_REQUIRE(max_slots >= 1, "max_slots must be >= 1");
    for (int i = 0; i < n_pairs; ++i)
      SYK_REQUIRE(pairs[2 * i] >= 0 && pairs[2 * i] < h->N && pairs[2 * i + 1] >= 0 && pairs[2 * i + 1] < h->N,
                  "Majorana index out of range [0, N)");
    const int64_t G = 2 * h->D;
    const int64_t n_jobs = static_cast<int64_t>(n_pairs) * G;
    std::vector<double> Fj(static_cast<size_t>(n_jobs) * n_t * 2, 0.0);
    std::vector<int> status(static_cast<size_t>(n_jobs), SYK_OK);
    std::vector<syk_krylov_stats> st(static_cast<size_t>(n_jobs));
    auto ck = [](int r) {
      if (r != SYK_OK) throw syk::Error(r, "batched engine call failed");
    };
    ck(syk_batch_create(h->dtype, static_cast<int>(std::min<int64_t>(max_slots, n_jobs)), max_bytes, p, &b));
    std::vector<int64_t> done(static_cast<size_t>(std::min<int64_t>(max_slots, n_jobs)));
    int64_t next = 0, finished = 0;
    while (finished < n_jobs) {
      while (next < n_jobs) {
        syk_otoc_job job{};
        job.h = h;
        job.a = pairs[2 * (next / G)];
        job.b = pairs[2 * (next / G) + 1];
        job.beta = beta;
        job.t_grid = t_grid;
        job.n_t = n_t;
        job.tag = next;
        job.F_out = &Fj[static_cast<size_t>(next) * n_t * 2];
        job.stats = &st[static_cast<size_t>(next)];
        job.status_out = &status[static_cast<size_t>(next)];
        job.basis_index = next % G;
        job.kind = SYK_JOB_OTOC;
        const int r = syk_batch_submit(b, &job);
        if (r == SYK_EAGAIN) break;
        ck(r);
        ++next;
      }
      int nf = 0;
      ck(syk_batch_run(b, 1 << 20, 16, &nf, done.data(), static_cast<int>(done.size())));
      finished += nf;
    }
    syk_batch_destroy(b);
    b = nullptr;
    int64_t mv = 0, ss = 0;
    for (int64_t j = 0; j < n_jobs; ++j) {
      if (status[static_cast<size_t>(j)] != SYK_OK)
        throw syk::Error(SYK_ENOCONV, "a basis-state job did not converge (increase m or tol)");
      mv += st[static_cast<size_t>(j)].matvecs;
      ss += st[static_cast<size_t>(j)].substeps;
    }
    for (int i = 0; i < n_pairs; ++i) {
      std::vector<double> acc(static_cast<size_t>(n_t) * 2, 0.0);
      for (int64_t g = 0; g < G; ++g) {
        const double* f = &Fj[static_cast<size_t>(i * G + g) * n_t * 2];
        for (int k = 0; k < 2 * n_t; ++k) acc[static_cast<size_t>(k)] += f[k];
      }
      for (double& v : acc) v /= static_cast<double>(G);
      if (F_out) std::copy(acc.begin(), acc.end(), F_out + static_cast<size_t>(i) * n_t * 2);
      if (otoc_out)
        for (int n = 0; n < n_t; ++n) otoc_out[static_cast<size_t>(i) * n_t + n] = acc[2 * n] / acc[0];
    }
    if (stats) {
      stats->matvecs = mv;
      stats->substeps = ss;
      stats->err_est = 0.0;
    }
  });
  if (b) syk_batch_destroy(b);
  return rc;
}
