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
//
// The substep control stays on the device: one substep is captured once per
// (block, output vector, workspace, m, reorth, two_pass) as the body of a
// CUDA-graph while-loop, and the tridiagonal kernel decides after each
// substep whether another one runs (cudaGraphSetConditional).  A call queues
// the loop and returns; counts and failures accumulate in the workspace's
// device scalars and are read once by the caller at the end of its work.
#include <cfloat>
#include <cmath>
#include <algorithm>
#include <complex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "tridiag.cuh"

namespace syk {
namespace {

__global__ void __launch_bounds__(32) k_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  tridiag_warp(sc, m, z_re, z_im, tol, Z);
}

__global__ void __launch_bounds__(32) k_tridiag_test(KScalars* sc, int m, double z_re, double z_im, double tol,
                                                    int allow_lane_parallel) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  tridiag_warp(sc, m, z_re, z_im, tol, Z, allow_lane_parallel != 0);
}

// Start of one evolve: the remaining step is all of z, no substep taken yet.
__global__ void k_evolve_init(KScalars* sc, double tau, double t, double tol, int max_sub) {
  sc->z_re = tau;
  sc->z_im = t;
  sc->tol = tol;
  sc->max_sub = max_sub;
  sc->n_sub = 0;
  sc->fail = 0;
}

// The substep's projected exponential plus the loop control of a captured
// evolve: accept the fraction s of the remaining step (or record a failure),
// count the substep, and set the while-loop condition: 1 runs another substep,
// 0 ends the loop once this substep's combine has run.
__global__ void __launch_bounds__(32) k_tridiag_ctl(KScalars* sc, int m, long long matvecs_per_substep,
                                                   cudaGraphConditionalHandle loop) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  const double zr = sc->z_re, zi = sc->z_im, tol = sc->tol;
  tridiag_warp(sc, m, zr, zi, tol, Z);
  __syncwarp();
  if (threadIdx.x == 0) {
    sc->n_sub += 1;
    sc->tot.substeps += 1;
    sc->tot.matvecs += matvecs_per_substep;
    unsigned int again = 0;
    const double s = sc->s_acc;
    if (sc->status != 0 || !(s > 0.0)) {
      sc->fail = sc->status == 2 ? 2 : 1;
    } else {
      sc->tot.err += sc->err * s;
      if (s < 1.0) {
        sc->z_re = zr * (1.0 - s);
        sc->z_im = zi * (1.0 - s);
        if (sc->n_sub >= sc->max_sub)
          sc->fail = 3;
        else
          again = 1;
      }
    }
    if (sc->fail && !sc->tot.fail) sc->tot.fail = sc->fail;
    cudaGraphSetConditional(loop, again);
  }
}

// Captured evolves kept per handle (least recently used dropped first).
constexpr size_t kMaxGraphs = 64;

struct WsLayout {
  KScalars* sc;
  double *partialA, *partialN, *partialR;
  char* vecs;
};

WsLayout ws_layout(const syk_terms* h, void* ws) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t G = static_cast<size_t>(std::max(vec_grid(h), matvec_grid(h)));
  WsLayout L;
  char* p = static_cast<char*>(ws);
  L.sc = reinterpret_cast<KScalars*>(p);
  p += up(sizeof(KScalars));
  L.partialA = reinterpret_cast<double*>(p);
  p += up(G * sizeof(double));
  L.partialN = reinterpret_cast<double*>(p);
  p += up(G * sizeof(double));
  L.partialR = reinterpret_cast<double*>(p);
  p += up(kMaxKrylov * G * 2 * sizeof(double));
  L.vecs = p;
  return L;
}

// One Lanczos substep on y (input and output), queued on st: the body of the
// captured while-loop.
void record_substep(const syk_terms* h, int block, void* y, void* ws, int m, bool reorth, bool two_pass,
                    cudaGraphConditionalHandle loop, cudaStream_t st) {
  const WsLayout L = ws_layout(h, ws);
  KScalars* sc = L.sc;
  // basis vectors back to back: the combine and re-orthogonalisation kernels
  // index vector j at j * D amplitudes
  const size_t vb = static_cast<size_t>(h->D) * elem_bytes(h->dtype);
  const int npA = matvec_grid(h), npN = vec_grid(h);
  const double brk = 1e-14 * std::max(h->sum_abs, 1e-300);
  if (!two_pass) {
    auto V = [&](int j) { return static_cast<void*>(L.vecs + static_cast<size_t>(j) * vb); };
    launch_norm_partials(h, y, L.partialN, st);
    launch_scale_first(h, y, V(0), L.partialN, sc, m, st);
    for (int j = 0; j < m; ++j) {
      launch_lanczos_matvec(h, block, V(j), j ? V(j - 1) : nullptr, V(j + 1), L.partialA, sc, j, st);
      launch_axpy_norm(h, V(j + 1), V(j), L.partialA, npA, L.partialN, sc, j, st);
      if (reorth) launch_reorth(h, V(j + 1), V(0), j, L.partialR, L.partialN, sc, st);
      launch_scale_next(h, V(j + 1), L.partialN, npN, sc, j, brk, st);
    }
    k_tridiag_ctl<<<1, 32, 0, st>>>(sc, m, m, loop);
    SYK_CUDA(cudaGetLastError());
    launch_combine(h, V(0), y, sc, m, st);
  } else {
    void* B[3] = {L.vecs, L.vecs + vb, L.vecs + 2 * vb};
    // pass 1: scalars only (ring of three vectors)
    launch_norm_partials(h, y, L.partialN, st);
    launch_scale_first(h, y, B[0], L.partialN, sc, m, st);
    int cur = 0, prv = 2, nxt = 1;
    for (int j = 0; j < m; ++j) {
      launch_lanczos_matvec(h, block, B[cur], j ? B[prv] : nullptr, B[nxt], L.partialA, sc, j, st);
      launch_axpy_norm(h, B[nxt], B[cur], L.partialA, npA, L.partialN, sc, j, st);
      launch_scale_next(h, B[nxt], L.partialN, npN, sc, j, brk, st);
      prv = cur;
      cur = nxt;
      nxt = 3 - prv - cur;
    }
    k_tridiag_ctl<<<1, 32, 0, st>>>(sc, m, 2 * m - 1, loop);
    SYK_CUDA(cudaGetLastError());
    // pass 2: regenerate v_j and accumulate y (y is read once, elementwise, before it is written)
    launch_recur_first(h, y, B[0], y, sc, st);
    cur = 0;
    prv = 2;
    nxt = 1;
    for (int j = 0; j + 1 < m; ++j) {
      launch_lanczos_recur(h, block, B[cur], j ? B[prv] : nullptr, B[nxt], y, sc, j, st);
      prv = cur;
      cur = nxt;
      nxt = 3 - prv - cur;
    }
  }
}

// The instantiated evolve graph for (block, y, ws, m, reorth, two_pass):
// [while (condition) { substep }], the condition 1 at every launch.
cudaGraphExec_t evolve_graph(const syk_terms* h, int block, void* y, void* ws, int m, bool reorth, bool two_pass) {
  for (auto& g : h->kgraphs)
    if (g.block == block && g.y == y && g.ws == ws && g.m == m && g.reorth == reorth && g.two_pass == two_pass) {
      g.used = ++h->kg_clock;
      return g.exec;
    }
  if (!h->cap_stream) SYK_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (h->kgraphs.size() >= kMaxGraphs) {
    auto lru = std::min_element(h->kgraphs.begin(), h->kgraphs.end(),
                                [](const KrylovGraph& a, const KrylovGraph& b) { return a.used < b.used; });
    SYK_CUDA(cudaStreamSynchronize(h->cap_stream));
    if (lru->exec) cudaGraphExecDestroy(lru->exec);
    if (lru->graph) cudaGraphDestroy(lru->graph);
    h->kgraphs.erase(lru);
  }
  KrylovGraph g;
  g.block = block;
  g.y = y;
  g.ws = ws;
  g.m = m;
  g.reorth = reorth;
  g.two_pass = two_pass;
  SYK_CUDA(cudaGraphCreate(&g.graph, 0));
  try {
    cudaGraphConditionalHandle loop;
    SYK_CUDA(cudaGraphConditionalHandleCreate(&loop, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    SYK_CUDA(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    SYK_CUDA(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    try {
      record_substep(h, block, y, ws, m, reorth, two_pass, loop, h->cap_stream);
    } catch (...) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(h->cap_stream, &dummy);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t captured = nullptr;
    SYK_CUDA(cudaStreamEndCapture(h->cap_stream, &captured));
    SYK_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
  } catch (...) {
    cudaGraphDestroy(g.graph);
    throw;
  }
  g.used = ++h->kg_clock;
  h->kgraphs.push_back(g);
  return g.exec;
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

void krylov_totals_reset(void* ws, cudaStream_t st) {
  SYK_CUDA(cudaMemsetAsync(&static_cast<KScalars*>(ws)->tot, 0, sizeof(KTotals), st));
}

void krylov_totals_collect(void* ws, cudaStream_t st, KrylovResult& acc) {
  KTotals t{};
  SYK_CUDA(cudaMemcpyAsync(&t, &static_cast<KScalars*>(ws)->tot, sizeof(KTotals), cudaMemcpyDeviceToHost, st));
  SYK_CUDA(cudaStreamSynchronize(st));
  acc.matvecs += t.matvecs;
  acc.substeps += t.substeps;
  acc.err += t.err;
  if (t.fail == 2) throw Error(SYK_ENOCONV, "Krylov evolve: tridiagonal eigensolver did not converge");
  if (t.fail == 3) throw Error(SYK_ENOCONV, "Krylov evolve: max_substeps reached before the step was complete");
  if (t.fail) throw Error(SYK_ENOCONV, "Krylov evolve: no acceptable substep (increase m or tol)");
}

// Evolve one state.  x and y are device vectors of D amplitudes; y may alias
// x.  The Lanczos path queues [copy x -> y] [init] [captured substep loop] on
// st and returns without synchronising: its counts and any failure are in
// the workspace's device totals (krylov_totals_collect).
KrylovResult krylov_evolve_one(const syk_terms* h, int block, double tau, double t, const void* x, void* y, int m,
                               double tol, int max_substeps, bool reorth, bool two_pass, void* ws, cudaStream_t st) {
  if (!h->hermitian) {  // complex couplings: full orthogonalisation (Arnoldi) instead of the three-term recurrence
    SYK_REQUIRE(!reorth && !two_pass, "a non-Hermitian H needs the stored Arnoldi basis (no reorth / two_pass)");
    return arnoldi_evolve_one(h, block, tau, t, x, y, m, tol, max_substeps, ws, st);
  }
  const size_t esz = elem_bytes(h->dtype);
  m = static_cast<int>(std::min<int64_t>(m, h->D));
  if (x != y) SYK_CUDA(cudaMemcpyAsync(y, x, h->D * esz, cudaMemcpyDeviceToDevice, st));
  if (tau == 0.0 && t == 0.0) return KrylovResult{};
  cudaGraphExec_t exec = evolve_graph(h, block, y, ws, m, reorth, two_pass);
  KScalars* sc = static_cast<KScalars*>(ws);
  k_evolve_init<<<1, 1, 0, st>>>(sc, tau, t, tol, max_substeps);
  SYK_CUDA(cudaGetLastError());
  SYK_CUDA(cudaGraphLaunch(exec, st));
  return KrylovResult{};
}

}  // namespace syk

extern "C" int syk_tridiag_exp(int m, const double* alpha, const double* beta, double z_re, double z_im, double tol,
                               int force_ql, double* c, double* s_acc, double* err, int* used_ql, double* kernel_ms) {
  syk::KScalars* d = nullptr;
  int rc = SYK_OK;
  try {
    SYK_REQUIRE(m >= 1 && m <= syk::kMaxKrylov, "m must be in [1, 64]");
    SYK_REQUIRE(alpha && beta && c && s_acc && err, "null argument");
    SYK_REQUIRE(std::isfinite(z_re) && std::isfinite(z_im) && std::isfinite(tol) && tol > 0, "bad z or tol");
    syk::KScalars h{};
    for (int i = 0; i < m; ++i) {
      SYK_REQUIRE(std::isfinite(alpha[i]) && std::isfinite(beta[i]) && beta[i] >= 0.0, "bad alpha or beta");
      h.alpha[i] = alpha[i];
      h.beta[i] = beta[i];
    }
    h.m_eff = m;
    if (cudaMalloc(&d, sizeof(syk::KScalars)) != cudaSuccess) {
      cudaGetLastError();
      d = nullptr;
      throw syk::Error(SYK_ENOMEM, "device allocation failed");
    }
    SYK_CUDA(cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice));
    syk::k_tridiag_test<<<1, 32>>>(d, m, z_re, z_im, tol, force_ql ? 0 : 1);
    SYK_CUDA(cudaGetLastError());
    SYK_CUDA(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost));
    if (kernel_ms) {  // median of 5 timed launches on the same input (each recomputes the step)
      cudaEvent_t e0, e1;
      SYK_CUDA(cudaEventCreate(&e0));
      SYK_CUDA(cudaEventCreate(&e1));
      std::vector<float> t(5);
      for (auto& v : t) {
        SYK_CUDA(cudaEventRecord(e0));
        syk::k_tridiag_test<<<1, 32>>>(d, m, z_re, z_im, tol, force_ql ? 0 : 1);
        SYK_CUDA(cudaEventRecord(e1));
        SYK_CUDA(cudaEventSynchronize(e1));
        SYK_CUDA(cudaEventElapsedTime(&v, e0, e1));
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::sort(t.begin(), t.end());
      *kernel_ms = t[2];
    }
    for (int i = 0; i < m; ++i) {
      c[2 * i] = h.c_re[i];
      c[2 * i + 1] = h.c_im[i];
    }
    *s_acc = h.s_acc;
    *err = h.err;
    if (used_ql) *used_ql = h.tot.ql;
    if (h.status == 2) throw syk::Error(SYK_ENOCONV, "tridiagonal eigensolver did not converge");
  } catch (const syk::Error& e) {
    syk::set_last_error(std::string("syk_tridiag_exp: ") + e.what());
    rc = e.code;
  }
  if (d) cudaFree(d);
  return rc;
}
