// Device kernels of the sparse-SYK hot path.
//
//  * k_matvec      — H_P psi, the matrix-free Pauli-string action of
//                    Algorithm 1 (supplement Sec. I.A), with optional fused
//                    Lanczos epilogues;
//  * k_chi         — one Majorana between parity blocks;
//  * k_random      — Philox4x32-10 + Box-Muller typical-state amplitudes;
//  * vector kernels for the Lanczos recurrence and the OTOC inner products.
//
// Matvec layout.  A warp owns 32*R consecutive output amplitudes
// m = base + 32 r + lane (r < R).  For a term (x, z, c) the input of lane
// `lane` in row r is psi[(row ^ x_hi) | (lane ^ x_lo)] with x_lo = x & 31,
// so every load instruction of the warp reads one contiguous, aligned
// 32-amplitude segment (coalesced).  The sign (-1)^{popc(z & m)} splits into
// a per-lane part (popc(z & lane), once per term) and a per-row part
// (popc(z & row), warp-uniform), both folded into the coefficient's sign bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace syk {
namespace {

template <typename Real>
struct CT;
template <>
struct CT<float> {
  using T = float2;
};
template <>
struct CT<double> {
  using T = double2;
};

__device__ __forceinline__ float sgnflip(float c, uint32_t s) {
  return __uint_as_float(__float_as_uint(c) ^ (s << 31));
}
__device__ __forceinline__ double sgnflip(double c, uint32_t s) {
  return __hiloint2double(__double2hiint(c) ^ static_cast<int>(s << 31), __double2loint(c));
}
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block-wide sum (fixed tree); every thread gets the result.
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  __shared__ double res;
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double u = lane < nw ? sh[lane] : 0.0;
    u = warp_sum(u);
    if (lane == 0) res = u;
  }
  __syncthreads();
  return res;
}

__device__ double sum_partials(const double* p, int np, int stride = 1) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += p[i * stride];
  return block_sum(s);
}

enum { EPI_STORE = 0, EPI_LANCZOS = 1, EPI_RECUR = 2 };

template <typename Real>
struct MV {
  TermsView<Real> tv;
  const typename CT<Real>::T* psi;
  typename CT<Real>::T* out;
  uint64_t D;
  const typename CT<Real>::T* vprev;  // Lanczos: v_{j-1} (null for j = 0)
  typename CT<Real>::T* y;            // second pass: accumulated result
  double* partial;                    // Lanczos: Re <v_j, w> per block
  const KScalars* sc;
  int j;
};

// Epilogue shared by the first Lanczos pass and the second (regenerating)
// pass, so that both produce bit-identical basis vectors:
//   w1 = acc - beta_{j-1} v_{j-1}; (later) w2 = w1 - alpha_j v_j; v_{j+1} = w2 * (1/beta_j).
template <typename Real, typename C>
__device__ __forceinline__ C lanczos_w1(Real ar, Real ai, Real bprev, C vp) {
  C w;
  w.x = fma_(-bprev, vp.x, ar);
  w.y = fma_(-bprev, vp.y, ai);
  return w;
}

template <typename Real, int R, int EPI>
__global__ void __launch_bounds__(256) k_matvec(MV<Real> p) {
  using C = typename CT<Real>::T;
  if (EPI == EPI_LANCZOS && p.sc->m_eff <= p.j) return;
  if (EPI == EPI_RECUR && p.j + 1 >= p.sc->m_eff) return;
  const uint64_t soff = static_cast<uint64_t>(blockIdx.y) * p.D;
  const C* __restrict__ psi = p.psi + soff;
  C* __restrict__ out = p.out + soff;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t nw = blockDim.x >> 5;
  const uint32_t tile = 32u * R * nw;
  const uint32_t ntiles = static_cast<uint32_t>(p.D / tile);
  Real bprev = 0, alpha = 0, rbeta = 0;
  C cy = {0, 0};
  if (EPI != EPI_STORE && p.j > 0) bprev = static_cast<Real>(p.sc->beta[p.j - 1]);
  if (EPI == EPI_RECUR) {
    alpha = static_cast<Real>(p.sc->alpha[p.j]);
    rbeta = static_cast<Real>(1.0 / p.sc->beta[p.j]);
    cy.x = static_cast<Real>(p.sc->beta0 * p.sc->c_re[p.j + 1]);
    cy.y = static_cast<Real>(p.sc->beta0 * p.sc->c_im[p.j + 1]);
  }
  double part = 0.0;
  for (uint32_t bt = blockIdx.x; bt < ntiles; bt += gridDim.x) {
    const uint32_t base = bt * tile + warp * 32u * R;
    Real ar[R], ai[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ar[r] = ai[r] = Real(0);
    for (int t = 0; t < p.tv.n_real; ++t) {
      const uint32_t x = __ldg(p.tv.x + t), z = __ldg(p.tv.z + t);
      const Real cl = sgnflip(__ldg(p.tv.coef + t), __popc(z & lane) & 1u);
      const uint32_t off = lane ^ (x & 31u), xh = x & ~31u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t row = base + 32u * r;
        const Real cc = sgnflip(cl, __popc(z & row) & 1u);
        const C v = psi[(row ^ xh) | off];
        ar[r] = fma_(cc, v.x, ar[r]);
        ai[r] = fma_(cc, v.y, ai[r]);
      }
    }
    for (int t = p.tv.n_real; t < p.tv.n; ++t) {  // coefficient i * c
      const uint32_t x = __ldg(p.tv.x + t), z = __ldg(p.tv.z + t);
      const Real cl = sgnflip(__ldg(p.tv.coef + t), __popc(z & lane) & 1u);
      const uint32_t off = lane ^ (x & 31u), xh = x & ~31u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t row = base + 32u * r;
        const Real cc = sgnflip(cl, __popc(z & row) & 1u);
        const C v = psi[(row ^ xh) | off];
        ar[r] = fma_(-cc, v.y, ar[r]);
        ai[r] = fma_(cc, v.x, ai[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t m = base + 32u * r + lane;
      if (EPI == EPI_STORE) {
        C o;
        o.x = ar[r];
        o.y = ai[r];
        out[m] = o;
      } else {
        C vp = {0, 0};
        if (p.j > 0) vp = p.vprev[soff + m];
        const C w1 = lanczos_w1<Real, C>(ar[r], ai[r], bprev, vp);
        const C v = psi[m];
        if (EPI == EPI_LANCZOS) {
          out[m] = w1;
          part += static_cast<double>(v.x * w1.x + v.y * w1.y);
        } else {
          C vn;
          vn.x = mul_(fma_(-alpha, v.x, w1.x), rbeta);
          vn.y = mul_(fma_(-alpha, v.y, w1.y), rbeta);
          out[m] = vn;
          C yy = p.y[soff + m];
          yy.x = fma_(cy.x, vn.x, fma_(-cy.y, vn.y, yy.x));
          yy.y = fma_(cy.x, vn.y, fma_(cy.y, vn.x, yy.y));
          p.y[soff + m] = yy;
        }
      }
    }
  }
  if (EPI == EPI_LANCZOS) {
    part = block_sum(part);
    if (threadIdx.x == 0) p.partial[blockIdx.y * gridDim.x + blockIdx.x] = part;
  }
}

// D < 32: one thread per amplitude, one warp.
template <typename Real, int EPI>
__global__ void k_matvec_tiny(MV<Real> p) {
  using C = typename CT<Real>::T;
  if (EPI == EPI_LANCZOS && p.sc->m_eff <= p.j) return;
  if (EPI == EPI_RECUR && p.j + 1 >= p.sc->m_eff) return;
  const uint64_t soff = static_cast<uint64_t>(blockIdx.y) * p.D;
  const C* psi = p.psi + soff;
  const uint32_t m = threadIdx.x;
  double part = 0.0;
  if (m < p.D) {
    Real ar = 0, ai = 0;
    for (int t = 0; t < p.tv.n; ++t) {
      const uint32_t x = p.tv.x[t], z = p.tv.z[t];
      const Real cc = sgnflip(p.tv.coef[t], __popc(z & m) & 1u);
      const C v = psi[m ^ x];
      if (t < p.tv.n_real) {
        ar = fma_(cc, v.x, ar);
        ai = fma_(cc, v.y, ai);
      } else {
        ar = fma_(-cc, v.y, ar);
        ai = fma_(cc, v.x, ai);
      }
    }
    if (EPI == EPI_STORE) {
      C o;
      o.x = ar;
      o.y = ai;
      p.out[soff + m] = o;
    } else {
      Real bprev = p.j > 0 ? static_cast<Real>(p.sc->beta[p.j - 1]) : Real(0);
      C vp = {0, 0};
      if (p.j > 0) vp = p.vprev[soff + m];
      const C w1 = lanczos_w1<Real, C>(ar, ai, bprev, vp);
      const C v = psi[m];
      if (EPI == EPI_LANCZOS) {
        p.out[soff + m] = w1;
        part = static_cast<double>(v.x * w1.x + v.y * w1.y);
      } else {
        const Real alpha = static_cast<Real>(p.sc->alpha[p.j]);
        const Real rbeta = static_cast<Real>(1.0 / p.sc->beta[p.j]);
        C cy;
        cy.x = static_cast<Real>(p.sc->beta0 * p.sc->c_re[p.j + 1]);
        cy.y = static_cast<Real>(p.sc->beta0 * p.sc->c_im[p.j + 1]);
        C vn;
        vn.x = mul_(fma_(-alpha, v.x, w1.x), rbeta);
        vn.y = mul_(fma_(-alpha, v.y, w1.y), rbeta);
        p.out[soff + m] = vn;
        C yy = p.y[soff + m];
        yy.x = fma_(cy.x, vn.x, fma_(-cy.y, vn.y, yy.x));
        yy.y = fma_(cy.x, vn.y, fma_(cy.y, vn.x, yy.y));
        p.y[soff + m] = yy;
      }
    }
  }
  if (EPI == EPI_LANCZOS) {
    part = block_sum(part);
    if (threadIdx.x == 0) p.partial[blockIdx.y * gridDim.x + blockIdx.x] = part;
  }
}

template <typename Real>
__global__ void k_chi(const typename CT<Real>::T* __restrict__ psi, typename CT<Real>::T* out, uint64_t D,
                      uint32_t x, uint32_t z, double cre, double cim) {
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

// Philox4x32-10 (Salmon et al., SC'11), written from the published round
// function: two 32x32->64 multiplies per round, key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

template <typename Real>
__global__ void k_random(typename CT<Real>::T* out, uint64_t D, uint64_t g0, uint64_t seed, uint64_t sid) {
  using C = typename CT<Real>::T;
  for (uint64_t m = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; m < D;
       m += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t g = g0 + m;
    uint32_t c[4] = {static_cast<uint32_t>(g), static_cast<uint32_t>(g >> 32), static_cast<uint32_t>(sid),
                     static_cast<uint32_t>(sid >> 32)};
    philox4x32_10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    const uint64_t a = ((static_cast<uint64_t>(c[1]) << 32) | c[0]) >> 11;
    const uint64_t b = ((static_cast<uint64_t>(c[3]) << 32) | c[2]) >> 11;
    const double u1 = (static_cast<double>(a) + 1.0) * 0x1.0p-53;
    const double u2 = static_cast<double>(b) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    C o;
    o.x = static_cast<Real>(r * cs);
    o.y = static_cast<Real>(r * sn);
    out[m] = o;
  }
}

// ---- streaming vector kernels (grid-stride, 256 threads) ----
template <typename Real>
__global__ void k_norm_partials(const typename CT<Real>::T* __restrict__ x, uint64_t D, double* partial) {
  double s = 0.0;
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    const auto v = x[i];
    s += static_cast<double>(v.x * v.x + v.y * v.y);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename Real>
__global__ void k_scale_first(const typename CT<Real>::T* x, typename CT<Real>::T* v0, uint64_t D,
                              const double* partial, int np, KScalars* sc, int m) {
  using C = typename CT<Real>::T;
  const double n2 = sum_partials(partial, np);
  const double b0 = sqrt(n2);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->beta0 = b0;
    sc->m_eff = (b0 > 0.0) ? m : 0;
    sc->status = 0;
  }
  const Real inv = b0 > 0.0 ? static_cast<Real>(1.0 / b0) : Real(0);
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    const C v = x[i];
    C o;
    o.x = mul_(v.x, inv);
    o.y = mul_(v.y, inv);
    v0[i] = o;
  }
}

template <typename Real>
__global__ void k_axpy_norm(typename CT<Real>::T* w, const typename CT<Real>::T* __restrict__ v, uint64_t D,
                            const double* partialA, int npA, double* partialN, KScalars* sc, int j) {
  using C = typename CT<Real>::T;
  if (sc->m_eff <= j) return;
  const double a = sum_partials(partialA, npA);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->alpha[j] = a;
  const Real al = static_cast<Real>(a);
  double s = 0.0;
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    C ww = w[i];
    const C vv = v[i];
    ww.x = fma_(-al, vv.x, ww.x);
    ww.y = fma_(-al, vv.y, ww.y);
    w[i] = ww;
    s += static_cast<double>(ww.x * ww.x + ww.y * ww.y);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partialN[blockIdx.x] = s;
}

template <typename Real>
__global__ void k_scale_next(typename CT<Real>::T* w, uint64_t D, const double* partialN, int np, KScalars* sc,
                             int j, double brk) {
  using C = typename CT<Real>::T;
  if (sc->m_eff <= j) return;
  const double b = sqrt(sum_partials(partialN, np));
  const bool breakdown = !(b > brk);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->beta[j] = b;
    if (breakdown) sc->m_eff = j + 1;
  }
  if (breakdown) return;
  const Real inv = static_cast<Real>(1.0 / b);
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    C ww = w[i];
    ww.x = mul_(ww.x, inv);
    ww.y = mul_(ww.y, inv);
    w[i] = ww;
  }
}

// partialR[(i * G + b) * 2 + {0,1}] = sum conj(V_i) w over block b.
template <typename Real>
__global__ void k_dots(const typename CT<Real>::T* __restrict__ V, const typename CT<Real>::T* __restrict__ w,
                       uint64_t D, double* partialR, const KScalars* sc, int j) {
  if (sc->m_eff <= j) return;
  const int i = blockIdx.y;
  const auto* Vi = V + static_cast<uint64_t>(i) * D;
  double sr = 0.0, si = 0.0;
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
    const auto a = Vi[k];
    const auto b = w[k];
    sr += static_cast<double>(a.x * b.x + a.y * b.y);
    si += static_cast<double>(a.x * b.y - a.y * b.x);
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) {
    partialR[(static_cast<uint64_t>(i) * gridDim.x + blockIdx.x) * 2 + 0] = sr;
    partialR[(static_cast<uint64_t>(i) * gridDim.x + blockIdx.x) * 2 + 1] = si;
  }
}

template <typename Real>
__global__ void k_reorth_sub(typename CT<Real>::T* w, const typename CT<Real>::T* __restrict__ V, uint64_t D,
                             int nvec, const double* partialR, double* partialN, const KScalars* sc, int j) {
  using C = typename CT<Real>::T;
  if (sc->m_eff <= j) return;
  __shared__ Real hr[kMaxKrylov], hi[kMaxKrylov];
  for (int i = 0; i < nvec; ++i) {
    const double a = sum_partials(partialR + static_cast<uint64_t>(i) * gridDim.x * 2, gridDim.x, 2);
    const double b = sum_partials(partialR + static_cast<uint64_t>(i) * gridDim.x * 2 + 1, gridDim.x, 2);
    if (threadIdx.x == 0) {
      hr[i] = static_cast<Real>(a);
      hi[i] = static_cast<Real>(b);
    }
  }
  __syncthreads();
  double s = 0.0;
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
    C ww = w[k];
    for (int i = 0; i < nvec; ++i) {
      const C v = V[static_cast<uint64_t>(i) * D + k];
      ww.x = fma_(-hr[i], v.x, fma_(hi[i], v.y, ww.x));
      ww.y = fma_(-hr[i], v.y, fma_(-hi[i], v.x, ww.y));
    }
    w[k] = ww;
    s += static_cast<double>(ww.x * ww.x + ww.y * ww.y);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partialN[blockIdx.x] = s;
}

template <typename Real>
__global__ void k_combine(const typename CT<Real>::T* __restrict__ V, typename CT<Real>::T* y, uint64_t D,
                          const KScalars* sc, int m) {
  using C = typename CT<Real>::T;
  __shared__ Real cr[kMaxKrylov], ci[kMaxKrylov];
  const int n = min(sc->m_eff, m);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cr[i] = static_cast<Real>(sc->beta0 * sc->c_re[i]);
    ci[i] = static_cast<Real>(sc->beta0 * sc->c_im[i]);
  }
  __syncthreads();
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < D; k += gridDim.x * 256ull) {
    Real a = 0, b = 0;
    for (int i = 0; i < n; ++i) {
      const C v = V[static_cast<uint64_t>(i) * D + k];
      a = fma_(cr[i], v.x, fma_(-ci[i], v.y, a));
      b = fma_(cr[i], v.y, fma_(ci[i], v.x, b));
    }
    C o;
    o.x = a;
    o.y = b;
    y[k] = o;
  }
}

template <typename Real>
__global__ void k_recur_first(const typename CT<Real>::T* x, typename CT<Real>::T* v0, typename CT<Real>::T* y,
                              uint64_t D, const KScalars* sc) {
  using C = typename CT<Real>::T;
  const double b0 = sc->beta0;
  const Real inv = b0 > 0.0 ? static_cast<Real>(1.0 / b0) : Real(0);
  const bool any = sc->m_eff > 0;
  const Real cr = any ? static_cast<Real>(b0 * sc->c_re[0]) : Real(0);
  const Real ci = any ? static_cast<Real>(b0 * sc->c_im[0]) : Real(0);
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    const C v = x[i];
    C o;
    o.x = mul_(v.x, inv);
    o.y = mul_(v.y, inv);
    v0[i] = o;
    C yy;
    yy.x = fma_(cr, o.x, -mul_(ci, o.y));
    yy.y = fma_(cr, o.y, mul_(ci, o.x));
    y[i] = yy;
  }
}

template <typename Real>
__global__ void k_zdot_partials(const typename CT<Real>::T* __restrict__ a, const typename CT<Real>::T* __restrict__ b,
                                uint64_t D, double* partial) {
  double sr = 0.0, si = 0.0;
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    const auto u = a[i];
    const auto v = b[i];
    sr += static_cast<double>(u.x) * v.x + static_cast<double>(u.y) * v.y;
    si += static_cast<double>(u.x) * v.y - static_cast<double>(u.y) * v.x;
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sr;
    partial[2 * blockIdx.x + 1] = si;
  }
}

__global__ void k_zdot_finalize(const double* partial, int np, double* out, double scale, int accumulate) {
  const double a = sum_partials(partial, np, 2) * scale;
  const double b = sum_partials(partial + 1, np, 2) * scale;
  if (threadIdx.x == 0) {
    out[0] = accumulate ? out[0] + a : a;
    out[1] = accumulate ? out[1] + b : b;
  }
}

__global__ void k_sum_finalize(const double* partial, int np, double* acc, int accumulate) {
  const double a = sum_partials(partial, np);
  if (threadIdx.x == 0) *acc = accumulate ? *acc + a : a;
}

template <typename Real>
__global__ void k_scale_inv_sqrt(typename CT<Real>::T* x, uint64_t D, const double* n2) {
  const Real inv = static_cast<Real>(1.0 / sqrt(*n2));
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    auto v = x[i];
    v.x = mul_(v.x, inv);
    v.y = mul_(v.y, inv);
    x[i] = v;
  }
}

template <typename Real>
__global__ void k_basis(typename CT<Real>::T* x, uint64_t D, int64_t k) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < D; i += gridDim.x * 256ull) {
    typename CT<Real>::T o;
    o.x = (static_cast<int64_t>(i) == k) ? Real(1) : Real(0);
    o.y = 0;
    x[i] = o;
  }
}

template <typename Real>
TermsView<Real> view(const syk_terms* h, int block) {
  TermsView<Real> v;
  v.x = h->d_x;
  v.z = h->d_z;
  v.coef = static_cast<const Real*>(h->d_coef[block]);
  v.n_real = static_cast<int>(h->n_real);
  v.n = static_cast<int>(h->terms.size());
  return v;
}

struct Shape {
  int R, warps, grid;
};

Shape shape_of(const syk_terms* h) {
  Shape s;
  const uint64_t D = static_cast<uint64_t>(h->D);
  if (D < 32) return {0, 1, 1};
  if (D >= 2048) {
    s.R = 8;
    s.warps = 8;
  } else {
    s.R = 1;
    s.warps = static_cast<int>(std::min<uint64_t>(8, D / 32));
  }
  const uint64_t ntiles = D / (32ull * s.R * s.warps);
  s.grid = static_cast<int>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(h->n_sm) * 8));
  return s;
}

template <typename Real, int EPI>
void run_matvec(const syk_terms* h, const MV<Real>& p, int64_t nstates, cudaStream_t st) {
  const Shape s = shape_of(h);
  for (int64_t s0 = 0; s0 < nstates; s0 += 65535) {
    MV<Real> q = p;
    const uint64_t off = static_cast<uint64_t>(s0) * h->D;
    q.psi += off;
    q.out += off;
    const unsigned gy = static_cast<unsigned>(std::min<int64_t>(65535, nstates - s0));
    if (s.R == 0) {
      k_matvec_tiny<Real, EPI><<<dim3(1, gy), 32, 0, st>>>(q);
    } else if (s.R == 8) {
      k_matvec<Real, 8, EPI><<<dim3(s.grid, gy), 32 * s.warps, 0, st>>>(q);
    } else {
      k_matvec<Real, 1, EPI><<<dim3(s.grid, gy), 32 * s.warps, 0, st>>>(q);
    }
  }
  SYK_CUDA(cudaGetLastError());
}

template <typename F>
void dispatch(int dtype, F&& f) {
  if (dtype == SYK_C128)
    f(double());
  else
    f(float());
}

}  // namespace

int vec_grid(const syk_terms* h) {
  const uint64_t need = (static_cast<uint64_t>(h->D) + 255) / 256;
  return static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(need, static_cast<uint64_t>(h->n_sm) * 4)));
}

int matvec_grid(const syk_terms* h) { return shape_of(h).grid; }

void launch_apply_H(const syk_terms* h, int block, const void* psi, void* out, int64_t nstates,
                    cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    MV<Real> p{};
    p.tv = view<Real>(h, block);
    p.psi = static_cast<const C*>(psi);
    p.out = static_cast<C*>(out);
    p.D = static_cast<uint64_t>(h->D);
    run_matvec<Real, EPI_STORE>(h, p, nstates, st);
  });
}

void launch_apply_chi(const syk_terms* h, int n, int from_block, const void* psi, void* out, int64_t nstates,
                      cudaStream_t st) {
  const ChiString& c = h->chi[n];
  const int grid = vec_grid(h);
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    for (int64_t s0 = 0; s0 < nstates; s0 += 65535) {
      const unsigned gy = static_cast<unsigned>(std::min<int64_t>(65535, nstates - s0));
      const uint64_t off = static_cast<uint64_t>(s0) * h->D;
      k_chi<Real><<<dim3(grid, gy), 256, 0, st>>>(static_cast<const C*>(psi) + off, static_cast<C*>(out) + off,
                                                  h->D, c.x, c.z, c.re[from_block], c.im[from_block]);
    }
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_random_state(const syk_terms* h, uint64_t seed, uint64_t state_id, int block, void* psi,
                         cudaStream_t st) {
  const int grid = vec_grid(h);
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_random<Real><<<grid, 256, 0, st>>>(static_cast<C*>(psi), h->D, static_cast<uint64_t>(block) * h->D, seed,
                                         state_id);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_norm_partials(const syk_terms* h, const void* x, double* partial, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    k_norm_partials<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<const typename CT<Real>::T*>(x), h->D, partial);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_scale_first(const syk_terms* h, const void* x, void* v0, const double* partial, KScalars* sc, int m,
                        cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_scale_first<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<const C*>(x), static_cast<C*>(v0), h->D, partial,
                                                     vec_grid(h), sc, m);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_lanczos_matvec(const syk_terms* h, int block, const void* v, const void* vprev, void* w,
                           double* partial, KScalars* sc, int j, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    MV<Real> p{};
    p.tv = view<Real>(h, block);
    p.psi = static_cast<const C*>(v);
    p.out = static_cast<C*>(w);
    p.vprev = static_cast<const C*>(vprev);
    p.D = static_cast<uint64_t>(h->D);
    p.partial = partial;
    p.sc = sc;
    p.j = j;
    run_matvec<Real, EPI_LANCZOS>(h, p, 1, st);
  });
}

void launch_axpy_norm(const syk_terms* h, void* w, const void* v, const double* partialA, int npA,
                      double* partialN, KScalars* sc, int j, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_axpy_norm<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<C*>(w), static_cast<const C*>(v), h->D, partialA, npA,
                                                   partialN, sc, j);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_reorth(const syk_terms* h, void* w, const void* V, int j, double* partialR, double* partialN,
                   KScalars* sc, cudaStream_t st) {
  const int G = vec_grid(h);
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    for (int pass = 0; pass < 2; ++pass) {
      k_dots<Real><<<dim3(G, j + 1), 256, 0, st>>>(static_cast<const C*>(V), static_cast<const C*>(w), h->D,
                                                   partialR, sc, j);
      k_reorth_sub<Real><<<G, 256, 0, st>>>(static_cast<C*>(w), static_cast<const C*>(V), h->D, j + 1, partialR,
                                            partialN, sc, j);
    }
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_scale_next(const syk_terms* h, void* w, const double* partialN, int npN, KScalars* sc, int j,
                       double brk, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    k_scale_next<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<typename CT<Real>::T*>(w), h->D, partialN, npN, sc,
                                                    j, brk);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_combine(const syk_terms* h, const void* V, void* y, const KScalars* sc, int m, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_combine<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<const C*>(V), static_cast<C*>(y), h->D, sc, m);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_recur_first(const syk_terms* h, const void* x, void* v0, void* y, const KScalars* sc,
                        cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_recur_first<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<const C*>(x), static_cast<C*>(v0),
                                                     static_cast<C*>(y), h->D, sc);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_lanczos_recur(const syk_terms* h, int block, const void* v, const void* vprev, void* vnext, void* y,
                          const KScalars* sc, int j, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    MV<Real> p{};
    p.tv = view<Real>(h, block);
    p.psi = static_cast<const C*>(v);
    p.out = static_cast<C*>(vnext);
    p.vprev = static_cast<const C*>(vprev);
    p.y = static_cast<C*>(y);
    p.D = static_cast<uint64_t>(h->D);
    p.sc = sc;
    p.j = j;
    run_matvec<Real, EPI_RECUR>(h, p, 1, st);
  });
}

void launch_zdot_partials(const syk_terms* h, const void* a, const void* b, double* partial, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    using C = typename CT<Real>::T;
    k_zdot_partials<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<const C*>(a), static_cast<const C*>(b), h->D,
                                                       partial);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_zdot_finalize(const double* partial, int np, double* out, double scale, int accumulate,
                          cudaStream_t st) {
  k_zdot_finalize<<<1, 256, 0, st>>>(partial, np, out, scale, accumulate);
  SYK_CUDA(cudaGetLastError());
}

void launch_sum_finalize(const double* partial, int np, double* acc, int accumulate, cudaStream_t st) {
  k_sum_finalize<<<1, 256, 0, st>>>(partial, np, acc, accumulate);
  SYK_CUDA(cudaGetLastError());
}

void launch_scale_inv_sqrt(const syk_terms* h, void* x, const double* n2, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    k_scale_inv_sqrt<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<typename CT<Real>::T*>(x), h->D, n2);
  });
  SYK_CUDA(cudaGetLastError());
}

void launch_basis_vector(const syk_terms* h, void* x, int64_t k, cudaStream_t st) {
  dispatch(h->dtype, [&](auto r) {
    using Real = decltype(r);
    k_basis<Real><<<vec_grid(h), 256, 0, st>>>(static_cast<typename CT<Real>::T*>(x), h->D, k);
  });
  SYK_CUDA(cudaGetLastError());
}

}  // namespace syk
