// Arnoldi propagation y = e^{-zH} x, z = tau + i t, for a non-Hermitian H
// (complex couplings: the non-Hermitian SYK of the paper's outlook).  The
// paper's restarted Krylov method (supplement Sec. I.A) with the Hermitian
// three-term recurrence replaced by full orthogonalisation:
//
//   beta0 = ||x||, v_0 = x / beta0;  for j < m:
//     w = H v_j;  classical Gram-Schmidt against v_0..v_j, twice
//     (h_{ij} accumulates both passes);  h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j};
//   y = beta0 V e^{-s z H_m} e_1 for the largest s = 2^-k whose local error
//   estimate passes, as in the Lanczos engine (Expokit, Sidje 1998; Saad 1992).
//
// The small exponential runs on the device in FP64 (one CTA): the augmented
// matrix A = [[-s z H_m, e_1], [0, 0]] gives e^{-s z H_m} e_1 in its first
// column and phi_1(-s z H_m) e_1 in its last (Saad 1992), by scaling and
// squaring with the diagonal [6/6] Pade approximant of e^x (Moler & Van Loan,
// "Nineteen dubious ways", method 3): with ||A||_1 <= 1/2 after scaling, the
// approximant's relative error is below 2^{3-2q} (q!)^2 / ((2q)! (2q+1)!) =
// 3.4e-16 for q = 6.  Its coefficients are computed from their closed form
// c_k = (2q-k)! q! / ((2q)! k! (q-k)!).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>

#include "device_common.cuh"
#include "kernels.cuh"

namespace syk {
namespace {

constexpr int kLd = kMaxKrylov + 1;  // leading dimension of the Hessenberg and Pade matrices
constexpr int kPadeQ = 6;
constexpr int kExpmMats = 9;          // scratch matrices of kLd x kLd complex doubles

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// partial[(i * G + b) * 2 + {0, 1}] = (Re, Im) of sum over block b's amplitudes
// of conj(V_i) w, for i < nvec (G = gridDim.x, blockDim.x = 256).  Eight basis
// vectors per pass over w; the 16 sums of a pass are reduced together (warp
// shuffles, then one barrier and a fixed-order sum over the 8 warps).
template <typename Real>
__global__ void __launch_bounds__(256) k_arn_dots(const typename CT<Real>::T* __restrict__ V,
                                                  const typename CT<Real>::T* __restrict__ w, uint64_t D, int nvec,
                                                  double* partial, const KScalars* sc, int j) {
  using C = typename CT<Real>::T;
  __shared__ double red[8][16];
  if (sc->m_eff <= j) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nvec; i0 += 8) {
    const int nb = min(8, nvec - i0);
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
      const C ww = w[k];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < nb) {
          const C v = V[static_cast<uint64_t>(i0 + q) * D + k];
          acc[2 * q] += static_cast<double>(v.x) * ww.x + static_cast<double>(v.y) * ww.y;
          acc[2 * q + 1] += static_cast<double>(v.x) * ww.y - static_cast<double>(v.y) * ww.x;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double v = warp_sum(acc[q]);
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * nb) {
      double t = 0.0;
      for (int wi = 0; wi < 8; ++wi) t += red[wi][threadIdx.x];
      partial[(static_cast<uint64_t>(i0 + (threadIdx.x >> 1)) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = t;
    }
    __syncthreads();
  }
}

// h_i = sum over the G dot partials of vector i (one warp per (i, Re/Im)
// pair, fixed order): written to hbuf and added to the Hessenberg column
// (the two Gram-Schmidt passes accumulate).  One block of 256 threads.
__global__ void __launch_bounds__(256) k_arn_reduce(const double* partial, int G, int nvec, double2* hcol,
                                                    double2* hbuf, const KScalars* sc, int j) {
  if (sc->m_eff <= j) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pr = warp; pr < 2 * nvec; pr += 8) {
    const int i = pr >> 1, comp = pr & 1;
    double t = 0.0;
    for (int b = lane; b < G; b += 32) t += partial[(static_cast<uint64_t>(i) * G + b) * 2 + comp];
    t = warp_sum(t);
    if (lane == 0) {
      if (comp) {
        hbuf[i].y = t;
        hcol[i].y += t;
      } else {
        hbuf[i].x = t;
        hcol[i].x += t;
      }
    }
  }
}

// w -= sum_i h_i V_i with h from k_arn_reduce; partialN[b] = sum |w|^2.
template <typename Real>
__global__ void k_arn_sub(typename CT<Real>::T* w, const typename CT<Real>::T* __restrict__ V, uint64_t D, int nvec,
                          const double2* hbuf, double* partialN, const KScalars* sc, int j) {
  using C = typename CT<Real>::T;
  if (sc->m_eff <= j) return;
  __shared__ Real hr[kMaxKrylov], hi[kMaxKrylov];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    hr[i] = static_cast<Real>(hbuf[i].x);
    hi[i] = static_cast<Real>(hbuf[i].y);
  }
  __syncthreads();
  double s = 0.0;
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
    C ww = w[k];
    for (int i = 0; i < nvec; ++i) {
      const C v = V[static_cast<uint64_t>(i) * D + k];
      const Real a = hr[i], b = hi[i];
      ww.x = fma_(-a, v.x, fma_(b, v.y, ww.x));
      ww.y = fma_(-a, v.y, fma_(-b, v.x, ww.y));
    }
    w[k] = ww;
    s += static_cast<double>(ww.x) * ww.x + static_cast<double>(ww.y) * ww.y;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partialN[blockIdx.x] = s;
}

// h_{j+1,j} = ||w||; v_{j+1} = w / ||w||, or a breakdown (invariant subspace):
// m_eff = j + 1.
template <typename Real>
__global__ void k_arn_next(typename CT<Real>::T* w, uint64_t D, const double* partialN, int npN, double2* hsub,
                           KScalars* sc, int j, double brk) {
  using C = typename CT<Real>::T;
  if (sc->m_eff <= j) return;
  const double nrm = sqrt(sum_partials(partialN, npN));
  const bool ok = nrm > brk;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *hsub = make_double2(nrm, 0.0);
    if (!ok) sc->m_eff = j + 1;
  }
  if (!ok) return;
  const Real inv = static_cast<Real>(1.0 / nrm);
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
    C v = w[k];
    v.x = mul_(v.x, inv);
    v.y = mul_(v.y, inv);
    w[k] = v;
  }
}

// ---- small dense complex matrices (one CTA, row-major, leading dimension kLd) ----
__device__ void mat_mul(const double2* A, const double2* B, double2* Cm, int P) {
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    const int r = e / P, c = e % P;
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < P; ++l) {
      const double2 a = A[r * kLd + l], b = B[l * kLd + c];
      s.x = fma(a.x, b.x, fma(-a.y, b.y, s.x));
      s.y = fma(a.x, b.y, fma(a.y, b.x, s.y));
    }
    Cm[r * kLd + c] = s;
  }
  __syncthreads();
}

// X = e^A (A is overwritten by its scaled copy).  S: kExpmMats - 1 scratch
// matrices; returns the matrix holding the result.
__device__ double2* mat_expm(double2* A, double2* const* S, int P, bool& singular) {
  __shared__ double colsum[kLd];
  __shared__ int sh_s, sh_piv;
  __shared__ double2 fac[kLd];
  // 1-norm and the scaling 2^-s with ||A / 2^s||_1 <= 1/2
  for (int c = threadIdx.x; c < P; c += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < P; ++r) t += hypot(A[r * kLd + c].x, A[r * kLd + c].y);
    colsum[c] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int c = 0; c < P; ++c) nrm = fmax(nrm, colsum[c]);
    int s = 0;
    while (nrm > 0.5 && s < 1000) {
      nrm *= 0.5;
      ++s;
    }
    sh_s = s;
  }
  __syncthreads();
  const int sq = sh_s;
  const double scale = ldexp(1.0, -sq);
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    const int r = e / P, c = e % P;
    A[r * kLd + c].x *= scale;
    A[r * kLd + c].y *= scale;
  }
  __syncthreads();
  // Pade coefficients c_k = (2q-k)! q! / ((2q)! k! (q-k)!)
  double fct[2 * kPadeQ + 1];
  fct[0] = 1.0;
  for (int k = 1; k <= 2 * kPadeQ; ++k) fct[k] = fct[k - 1] * k;
  double cf[kPadeQ + 1];
  for (int k = 0; k <= kPadeQ; ++k)
    cf[k] = fct[2 * kPadeQ - k] * fct[kPadeQ] / (fct[2 * kPadeQ] * fct[k] * fct[kPadeQ - k]);
  double2 *A2 = S[0], *A4 = S[1], *A6 = S[2], *T = S[3], *U = S[4], *Nm = S[5], *Dm = S[6], *X = S[7];
  mat_mul(A, A, A2, P);
  mat_mul(A2, A2, A4, P);
  mat_mul(A4, A2, A6, P);
  // T = c1 I + c3 A2 + c5 A4;  V (in Nm) = c0 I + c2 A2 + c4 A4 + c6 A6
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    const int r = e / P, c = e % P, o = r * kLd + c;
    const double d = (r == c) ? 1.0 : 0.0;
    T[o] = make_double2(cf[1] * d + cf[3] * A2[o].x + cf[5] * A4[o].x, cf[3] * A2[o].y + cf[5] * A4[o].y);
    Nm[o] = make_double2(cf[0] * d + cf[2] * A2[o].x + cf[4] * A4[o].x + cf[6] * A6[o].x,
                         cf[2] * A2[o].y + cf[4] * A4[o].y + cf[6] * A6[o].y);
  }
  __syncthreads();
  mat_mul(A, T, U, P);  // U = A (c1 I + c3 A2 + c5 A4)
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    const int r = e / P, c = e % P, o = r * kLd + c;
    const double2 v = Nm[o], u = U[o];
    Nm[o] = make_double2(v.x + u.x, v.y + u.y);  // numerator V + U
    Dm[o] = make_double2(v.x - u.x, v.y - u.y);  // denominator V - U
  }
  __syncthreads();
  // Solve Dm X = Nm: Gaussian elimination with partial pivoting, then back substitution.
  bool sing = false;
  for (int k = 0; k < P; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = hypot(Dm[k * kLd + k].x, Dm[k * kLd + k].y);
      for (int r = k + 1; r < P; ++r) {
        const double v = hypot(Dm[r * kLd + k].x, Dm[r * kLd + k].y);
        if (v > best) {
          best = v;
          p = r;
        }
      }
      sh_piv = (best > 0.0) ? p : -1;
    }
    __syncthreads();
    const int p = sh_piv;
    if (p < 0) {
      sing = true;
      break;
    }
    if (p != k)
      for (int c = threadIdx.x; c < P; c += blockDim.x) {
        double2 t = Dm[k * kLd + c];
        Dm[k * kLd + c] = Dm[p * kLd + c];
        Dm[p * kLd + c] = t;
        t = Nm[k * kLd + c];
        Nm[k * kLd + c] = Nm[p * kLd + c];
        Nm[p * kLd + c] = t;
      }
    __syncthreads();
    for (int r = k + 1 + threadIdx.x; r < P; r += blockDim.x) fac[r] = cdiv(Dm[r * kLd + k], Dm[k * kLd + k]);
    __syncthreads();
    const int rows = P - k - 1;
    for (int e = threadIdx.x; e < rows * P; e += blockDim.x) {
      const int r = k + 1 + e / P, c = e % P;
      const double2 f = fac[r];
      if (c >= k) {
        const double2 t = cmul(f, Dm[k * kLd + c]);
        Dm[r * kLd + c].x -= t.x;
        Dm[r * kLd + c].y -= t.y;
      }
      const double2 t2 = cmul(f, Nm[k * kLd + c]);
      Nm[r * kLd + c].x -= t2.x;
      Nm[r * kLd + c].y -= t2.y;
    }
    __syncthreads();
  }
  if (sing) {
    singular = true;
    return Nm;
  }
  for (int k = P - 1; k >= 0; --k) {
    for (int c = threadIdx.x; c < P; c += blockDim.x) X[k * kLd + c] = cdiv(Nm[k * kLd + c], Dm[k * kLd + k]);
    __syncthreads();
    for (int e = threadIdx.x; e < k * P; e += blockDim.x) {
      const int r = e / P, c = e % P;
      const double2 t = cmul(Dm[r * kLd + k], X[k * kLd + c]);
      Nm[r * kLd + c].x -= t.x;
      Nm[r * kLd + c].y -= t.y;
    }
    __syncthreads();
  }
  // square sq times
  double2 *cur = X, *nxt = T;
  for (int i = 0; i < sq; ++i) {
    mat_mul(cur, cur, nxt, P);
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  singular = false;
  return cur;
}

// Substep search on the Arnoldi Hessenberg matrix (column-major hess, column j
// at hess + j * kLd): writes c = e^{-s z H_m} e_1 (first n entries), s_acc, err,
// status into sc.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_hess_expm(KScalars* sc, const double2* hess, int m, double z_re, double z_im,
                                                   double tol, double2* scratch) {
  __shared__ double sh_err;
  __shared__ int sh_done;
  const int n = min(sc->m_eff, m);
  if (n <= 0) {
    if (threadIdx.x == 0) {
      sc->s_acc = 1.0;
      sc->err = 0.0;
      sc->status = 0;
    }
    return;
  }
  const int P = n + 1;
  const bool exact = n < m;
  const double resid = exact ? 0.0 : hypot(hess[(n - 1) * kLd + n].x, hess[(n - 1) * kLd + n].y);
  double2* A = scratch;
  double2* S[kExpmMats - 1];
  for (int i = 0; i < kExpmMats - 1; ++i) S[i] = scratch + static_cast<size_t>(i + 1) * kLd * kLd;
  double s_frac = 1.0;
  bool ok = false;
  int status = 1;
  for (int attempt = 0; attempt < 64; ++attempt) {
    const double hr = s_frac * z_re, hi = s_frac * z_im;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
      const int r = e / P, c = e % P;
      double2 v = make_double2(0.0, 0.0);
      if (r < n && c < n && r <= c + 1) {
        const double2 hv = hess[c * kLd + r];
        v = make_double2(-(hr * hv.x - hi * hv.y), -(hr * hv.y + hi * hv.x));
      } else if (c == n && r == 0) {
        v = make_double2(1.0, 0.0);
      }
      A[r * kLd + c] = v;
    }
    __syncthreads();
    bool singular = false;
    const double2* E = mat_expm(A, S, P, singular);
    if (singular) {
      status = 3;
      break;
    }
    if (threadIdx.x == 0) {
      double nc2 = 0.0;
      for (int k = 0; k < n; ++k) nc2 += E[k * kLd].x * E[k * kLd].x + E[k * kLd].y * E[k * kLd].y;
      const double nc = sqrt(nc2);
      const double e1 = resid * hypot(E[(n - 1) * kLd].x, E[(n - 1) * kLd].y);
      const double e2 = resid * hypot(hr, hi) * hypot(E[(n - 1) * kLd + n].x, E[(n - 1) * kLd + n].y);
      const double err = (nc > 0.0) ? fmax(e1, e2) / nc : 0.0;
      sh_err = exact ? 0.0 : err;
      sh_done = (exact || err <= tol * s_frac || !(err == err)) ? ((err == err || exact) ? 1 : 2) : 0;
      if (sh_done == 1)
        for (int k = 0; k < n; ++k) {
          sc->c_re[k] = E[k * kLd].x;
          sc->c_im[k] = E[k * kLd].y;
        }
    }
    __syncthreads();
    if (sh_done) {
      ok = sh_done == 1;
      status = ok ? 0 : 1;
      break;
    }
    s_frac *= 0.5;
  }
  if (threadIdx.x == 0) {
    sc->s_acc = ok ? s_frac : 0.0;
    sc->err = ok ? sh_err : 0.0;
    sc->status = status;
  }
}

template <typename F>
void dispatch_real(int dtype, F&& f) {
  if (dtype == SYK_C128)
    f(double());
  else
    f(float());
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// Workspace: KScalars | dot partials [kMaxKrylov][G][2] | norm partials [G] |
// Hessenberg kLd x kLd | projection coefficients kLd | Pade scratch
// kExpmMats x kLd x kLd | m + 1 vectors.
size_t arnoldi_ws_bytes(const syk_terms* h, int m) {
  const size_t G = static_cast<size_t>(vec_grid(h));
  size_t b = up256(sizeof(KScalars)) + up256(kMaxKrylov * G * 2 * sizeof(double)) + up256(G * sizeof(double));
  b += up256(kLd * kLd * sizeof(double2)) + up256(kLd * sizeof(double2)) +
       up256(static_cast<size_t>(kExpmMats) * kLd * kLd * sizeof(double2));
  b += up256((static_cast<size_t>(m) + 1) * static_cast<size_t>(h->D) * elem_bytes(h->dtype));
  return b;
}

KrylovResult arnoldi_evolve_one(const syk_terms* h, int block, double tau, double t, const void* x, void* y, int m,
                                double tol, int max_substeps, void* ws, cudaStream_t st) {
  KrylovResult res;
  const size_t G = static_cast<size_t>(vec_grid(h));
  char* p = static_cast<char*>(ws);
  KScalars* sc = reinterpret_cast<KScalars*>(p);
  p += up256(sizeof(KScalars));
  double* partialD = reinterpret_cast<double*>(p);
  p += up256(kMaxKrylov * G * 2 * sizeof(double));
  double* partialN = reinterpret_cast<double*>(p);
  p += up256(G * sizeof(double));
  double2* hess = reinterpret_cast<double2*>(p);
  p += up256(kLd * kLd * sizeof(double2));
  double2* hbuf = reinterpret_cast<double2*>(p);
  p += up256(kLd * sizeof(double2));
  double2* scratch = reinterpret_cast<double2*>(p);
  p += up256(static_cast<size_t>(kExpmMats) * kLd * kLd * sizeof(double2));
  const size_t esz = elem_bytes(h->dtype);
  const size_t vb = static_cast<size_t>(h->D) * esz;  // back to back: kernels index vector j at j * D
  char* vecs = p;
  auto V = [&](int j) { return static_cast<void*>(vecs + static_cast<size_t>(j) * vb); };
  m = static_cast<int>(std::min<int64_t>(m, h->D));
  const double brk = 1e-14 * std::max(h->sum_abs, 1e-300);
  const int Gi = static_cast<int>(G);

  if (tau == 0.0 && t == 0.0) {
    if (x != y) SYK_CUDA(cudaMemcpyAsync(y, x, h->D * esz, cudaMemcpyDeviceToDevice, st));
    return res;
  }
  std::complex<double> zrem(tau, t);
  const void* xin = x;
  for (;;) {
    if (res.substeps >= max_substeps)
      throw Error(SYK_ENOCONV, "Arnoldi evolve: max_substeps reached before the step was complete");
    launch_norm_partials(h, xin, partialN, st);
    launch_scale_first(h, xin, V(0), partialN, sc, m, st);
    SYK_CUDA(cudaMemsetAsync(hess, 0, kLd * kLd * sizeof(double2), st));
    for (int j = 0; j < m; ++j) {
      launch_apply_H(h, block, V(j), V(j + 1), 1, st);
      dispatch_real(h->dtype, [&](auto r) {
        using Real = decltype(r);
        using C = typename CT<Real>::T;
        C* w = static_cast<C*>(V(j + 1));
        const C* Vb = static_cast<const C*>(V(0));
        for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
          k_arn_dots<Real><<<Gi, 256, 0, st>>>(Vb, w, h->D, j + 1, partialD, sc, j);
          k_arn_reduce<<<1, 256, 0, st>>>(partialD, Gi, j + 1, hess + static_cast<size_t>(j) * kLd, hbuf, sc, j);
          k_arn_sub<Real><<<Gi, 256, 0, st>>>(w, Vb, h->D, j + 1, hbuf, partialN, sc, j);
        }
        k_arn_next<Real><<<Gi, 256, 0, st>>>(w, h->D, partialN, Gi, hess + static_cast<size_t>(j) * kLd + j + 1, sc,
                                            j, brk);
      });
      SYK_CUDA(cudaGetLastError());
    }
    res.matvecs += m;
    k_hess_expm<<<1, 256, 0, st>>>(sc, hess, m, zrem.real(), zrem.imag(), tol, scratch);
    SYK_CUDA(cudaGetLastError());
    launch_combine(h, V(0), y, sc, m, st);
    struct {
      double s_acc, err;
      int status;
    } hv;
    SYK_CUDA(cudaMemcpyAsync(&hv.s_acc, &sc->s_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaMemcpyAsync(&hv.err, &sc->err, sizeof(double), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaMemcpyAsync(&hv.status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SYK_CUDA(cudaStreamSynchronize(st));
    res.substeps += 1;
    if (hv.status == 3) throw Error(SYK_ENOCONV, "Arnoldi evolve: singular Pade denominator");
    if (hv.status != 0 || !(hv.s_acc > 0.0))
      throw Error(SYK_ENOCONV, "Arnoldi evolve: no acceptable substep (increase m or tol)");
    res.err += hv.err * hv.s_acc;
    if (hv.s_acc >= 1.0) break;
    zrem *= (1.0 - hv.s_acc);
    xin = y;
  }
  return res;
}

}  // namespace syk
