// Batched OTOC engine: many (realisation, state) OTOC curves advanced
// together on one GPU.
//
// Every job runs the parity-block OTOC of the supplement (OTOC paragraph;
// the same chain as syk_otoc) as a device-resident state machine in a
// "slot".  One tick advances every live slot by one Krylov substep:
//
//   control   (one block per slot)  finish the previous substep; when an
//             evolution is complete, run the chain's elementwise steps (typical
//             state, chi_a / chi_b, copies, F(t_n) += <bra|ket>) up to the
//             next evolution, or mark the job done;
//   norm, scale_first, m x (matvec+epilogue, axpy_norm), tridiag (one warp
//   per slot), combine  — the Lanczos substep of syk_krylov_evolve, batched
//             over slots, on an unnormalised basis (basis_scale below): the
//             last block of a slot to leave axpy_norm finishes the step's beta.
//
// The slots of a tick form one flattened grid: slot s owns blocks
// [blk0[s], blk0[s+1]) (up to 256 blocks of 256 threads, grid-striding over
// its D amplitudes), so small and large realisations share a launch.  The tick
// is captured once into a CUDA graph and replayed; the host only admits jobs
// into free slots (device memory from an arena, admitted by footprint) and
// collects finished ones.  Reductions are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "kernels.cuh"
#include "tma_common.cuh"
#include "tridiag.cuh"

namespace syk {

namespace {

constexpr int kBlk = 256;          // threads per block
constexpr int kCtlBlk = 1024;      // threads of the per-slot control block (its vector stages run on one SM)
// Tick groups: two balance the served latency and the batch throughput on
// B300 (1000 served requests at half load, p50 / p99 / batched realisations
// per s: 2 groups 3.9 s / 13.3 s / 33.5; 3 groups 2.2 s / 15.7 s / 29.4;
// 4 groups 1.7 s / 17.7 s / 27.1).
#ifndef SYK_BATCH_GROUPS
#define SYK_BATCH_GROUPS 2
#endif
constexpr int kGroups = SYK_BATCH_GROUPS;  // tick groups (graphs on their own streams)
constexpr double kMaxTickRatio = 16.0;     // most ticks of a light group per tick of the heaviest
constexpr int kMaxBlkPerSlot = 256;  // blocks per slot (partials summed per slot)

enum Stage { S_INIT = 0, S_PART, S_AFTER_U0, S_POINT, S_K1, S_K2, S_K3, S_K4, S_G1, S_G2, S_DONE };

// Device-resident slot descriptor.
struct BSlot {
  // Hamiltonian of the job (device table of its syk_terms handle)
  const uint32_t* x;
  const uint32_t* zi;  // z | imag << 31
  const void* coef[2];
  const TermF* rec[2];       // complex64: packed records per block
  const PassPlan* passes;    // class ranges of the records (all passes, in table order)
  int n_passes;
  int n_terms;
  uint32_t D;
  uint32_t cx[2], cz[2];         // chi strings: [0] = chi_a, [1] = chi_b
  double cre[2][2], cim[2][2];   // [which][from block]
  // job
  double beta;
  int n_t;
  const double* tg;  // device [n_t]
  double* F;         // device [n_t][2]
  uint64_t seed, state_id;
  long long basis;  // < 0: Philox typical state; else basis state index g = block*D + m
  int kind;         // SYK_JOB_OTOC or SYK_JOB_GREEN
  void* vec[4];  // u0, bra, k1, k2
  void* V;       // basis, (m+1) x D
  // state machine
  int live, done, stage, part, n;
  double tprev, n2;
  int ev, ev_block, ev_vec;
  double z_re, z_im;
  long long matvecs, substeps;
  int status;
};

struct BatchArgs {
  BSlot* slots;
  KScalars* sc;
  const int* blk_slot;    // flattened block -> slot
  const int2* blk_range;  // per slot: (first block, number of blocks)
  int m;
  double tol;
  double* partA;  // [total blocks]
  double* partN;  // [total blocks]
  int* err;       // set when a bounded wait expires
  double brk;     // Lanczos breakdown threshold, relative to |alpha_j| + beta_{j-1}
  int* slot_cnt;  // [max slots] blocks of the slot done with k_b_axpy_norm (0 between launches)
  int* alpha_cnt;  // [max slots] blocks of the slot done with the matvec (0 between launches)
  double* lsc;    // [max slots][2] for the next matvec: s_j = 1 / beta_{j-1}, beta_{j-1} s_{j-1}
  const int* slot_group;  // [max slots] tick group of each live slot (-1: dead)
  int group;              // the group this tick's graph advances
};

template <typename Real>
__device__ __forceinline__ const typename CT<Real>::T* cvec(const BSlot& s, int i) {
  return static_cast<const typename CT<Real>::T*>(s.vec[i]);
}
template <typename Real>
__device__ __forceinline__ typename CT<Real>::T* mvec(const BSlot& s, int i) {
  return static_cast<typename CT<Real>::T*>(s.vec[i]);
}
template <typename Real>
__device__ __forceinline__ typename CT<Real>::T* basis(const BSlot& s, int j) {
  return static_cast<typename CT<Real>::T*>(s.V) + static_cast<size_t>(j) * s.D;
}

__device__ __forceinline__ double slot_sum(const double* part, int2 r) { return sum_partials(part + r.x, r.y); }

// The batched Lanczos keeps its basis unnormalised: basis[0] = v_0 (unit) and,
// for j >= 1, basis[j] = w_{j-1} = beta_{j-1} v_j, so that no pass over the
// vectors is spent on v_{j+1} = w_j / beta_j.  Every reader folds the scale
// s_j = 1 / beta_{j-1} (s_0 = 1) into a scalar it applies anyway.  Only call
// this for betas written by an earlier launch.
__device__ __forceinline__ double basis_scale(const KScalars* sc, int j) { return j > 0 ? 1.0 / sc->beta[j - 1] : 1.0; }

// Finish the matvec of Lanczos step j: the last block of the slot to get here
// (after every block's alpha partial is visible) sums the partials once, in
// the fixed order of slot_sum, into alpha_j, which k_b_axpy_norm then reads.
// Thread 0 has written this block's partial.  All threads of the block call it.
__device__ __forceinline__ void matvec_finish_alpha(const BatchArgs& a, KScalars* sc, int si, int j, int2 rg) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // the partial is visible before this block counts itself done
    last = atomicAdd(a.alpha_cnt + si, 1) == rg.y - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const double al = slot_sum(a.partA, rg);
    if (threadIdx.x == 0) {
      sc->alpha[j] = al;
      a.alpha_cnt[si] = 0;
    }
  }
}

// Finish Lanczos step j (run by the last block of the slot to leave
// k_b_axpy_norm(j), after every block's norm partial is visible):
// beta_j = ||w_j||, the breakdown test (m_eff = j + 1 on breakdown), and the
// scalars step j + 1's matvec applies: s_{j+1} = 1 / beta_j and
// beta_j s_j (the coefficient of basis[j]).  All threads of the block call it.
__device__ __forceinline__ void lanczos_finish_step(const BatchArgs& a, KScalars* sc, int si, int j, int2 rg) {
  const double b = sqrt(slot_sum(a.partN, rg));
  if (threadIdx.x == 0) {
    const double scale = fabs(sc->alpha[j]) + (j > 0 ? sc->beta[j - 1] : 0.0);
    sc->beta[j] = b;
    if (!(b > a.brk * fmax(scale, 1e-300))) sc->m_eff = j + 1;
    a.lsc[2 * si] = 1.0 / b;
    a.lsc[2 * si + 1] = b * basis_scale(sc, j);
  }
}


// ----------------------------------------------------------------- control --
// out = chi (which) in, from block P: out[m] = c (-1)^{popc(z&m)} in[m ^ x].
template <typename Real>
__device__ void blk_chi(const BSlot& s, int which, int P, const typename CT<Real>::T* in, typename CT<Real>::T* out) {
  const Real re = static_cast<Real>(s.cre[which][P]), im = static_cast<Real>(s.cim[which][P]);
  for (uint32_t m = threadIdx.x; m < s.D; m += blockDim.x) {
    const auto v = in[m ^ s.cx[which]];
    const uint32_t sg = __popc(s.cz[which] & m) & 1u;
    const Real a = sgnflip(re, sg), b = sgnflip(im, sg);
    typename CT<Real>::T o;
    o.x = fma_(a, v.x, -mul_(b, v.y));
    o.y = fma_(a, v.y, mul_(b, v.x));
    out[m] = o;
  }
  __syncthreads();
}

// Philox typical state of block P, unnormalised (same definition as k_random).
__device__ __forceinline__ double2 philox_amp(uint64_t g, uint64_t seed, uint64_t sid) {
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
  return make_double2(r * cs, r * sn);
}

template <typename Real>
__global__ void __launch_bounds__(kCtlBlk) k_b_control(BatchArgs a) {
  if (a.slot_group[blockIdx.x] != a.group) return;
  BSlot& g = a.slots[blockIdx.x];
  __shared__ BSlot s;
  __shared__ int stop;
  if (threadIdx.x == 0) {
    s = g;
    stop = (!s.live || s.done) ? 1 : 0;
  }
  __syncthreads();
  if (stop) return;
  using C = typename CT<Real>::T;
  if (threadIdx.x == 0 && s.ev) {  // the substep run in the previous tick
    const KScalars& k = a.sc[blockIdx.x];
    s.substeps += 1;
    s.matvecs += a.m;
    if (k.status != 0 || !(k.s_acc > 0.0)) {
      s.status = k.status ? k.status : 1;
      s.done = 1;
      s.stage = S_DONE;
    } else if (k.s_acc < 1.0) {
      s.z_re *= (1.0 - k.s_acc);
      s.z_im *= (1.0 - k.s_acc);
    } else {
      s.ev = 0;
    }
  }
  __syncthreads();
  // Advance the chain until the next evolution (or the end).  All threads
  // follow the same (shared) state.
  for (int guard = 0; guard < 64 && !s.ev && s.stage != S_DONE; ++guard) {
    const int P = s.part, Q = 1 - P;
    auto start_evolve = [&](int vec, int blk, double zr, double zi, int next) {
      __syncthreads();
      if (threadIdx.x == 0) {
        s.stage = next;
        if (zr != 0.0 || zi != 0.0) {
          s.ev = 1;
          s.ev_vec = vec;
          s.ev_block = blk;
          s.z_re = zr;
          s.z_im = zi;
        }
      }
      __syncthreads();
    };
    const int stage = s.stage;
    if (stage == S_INIT && s.basis >= 0) {  // basis state: already normalised
      __syncthreads();
      if (threadIdx.x == 0) {
        s.n2 = 1.0;
        s.part = 0;
        s.stage = S_PART;
      }
      __syncthreads();
    } else if (stage == S_PART && s.basis >= 0 && s.basis / s.D != static_cast<long long>(P)) {
      __syncthreads();  // the basis state has no component in this block: F_P = 0
      if (threadIdx.x == 0) {
        s.part += 1;
        s.stage = (s.part >= 2) ? S_DONE : S_PART;
      }
      __syncthreads();
    } else if (stage == S_INIT) {  // norm of the Philox state over both blocks
      double acc = 0.0;
      for (uint64_t g2 = threadIdx.x; g2 < 2ull * s.D; g2 += blockDim.x) {
        const double2 v = philox_amp(g2, s.seed, s.state_id);
        acc += v.x * v.x + v.y * v.y;
      }
      acc = block_sum(acc);
      if (threadIdx.x == 0) {
        s.n2 = acc;
        s.part = 0;
        s.stage = S_PART;
      }
      __syncthreads();
    } else if (stage == S_PART) {
      const double inv = 1.0 / sqrt(s.n2);
      C* u0 = mvec<Real>(s, 0);
      for (uint32_t m = threadIdx.x; m < s.D; m += blockDim.x) {
        const uint64_t gidx = static_cast<uint64_t>(P) * s.D + m;
        const double2 v = s.basis >= 0 ? make_double2(static_cast<long long>(gidx) == s.basis ? 1.0 : 0.0, 0.0)
                                       : philox_amp(gidx, s.seed, s.state_id);
        C o;
        o.x = static_cast<Real>(v.x * inv);
        o.y = static_cast<Real>(v.y * inv);
        u0[m] = o;
      }
      start_evolve(0, P, s.kind == SYK_JOB_GREEN ? s.beta / 2.0 : s.beta / 8.0, 0.0, S_AFTER_U0);
    } else if (stage == S_AFTER_U0) {
      const C* u0 = cvec<Real>(s, 0);
      C* bra = mvec<Real>(s, 1);
      for (uint32_t m = threadIdx.x; m < s.D; m += blockDim.x) bra[m] = u0[m];
      __syncthreads();
      if (threadIdx.x == 0) {
        s.n = 0;
        s.tprev = 0.0;
        s.stage = S_POINT;
      }
      __syncthreads();
    } else if (stage == S_POINT) {
      if (s.n >= s.n_t) {
        __syncthreads();
        if (threadIdx.x == 0) {
          s.part += 1;
          s.stage = (s.part >= 2) ? S_DONE : S_PART;
        }
        __syncthreads();
      } else {
        const double t = s.tg[s.n];
        const double dt = t - s.tprev;
        __syncthreads();
        if (threadIdx.x == 0) s.tprev = t;
        start_evolve(1, P, 0.0, dt, s.kind == SYK_JOB_GREEN ? S_G1 : S_K1);
      }
    } else if (stage == S_G1) {
      blk_chi<Real>(s, 0, P, cvec<Real>(s, 0), mvec<Real>(s, 2));  // k1 = chi_a u0
      start_evolve(2, Q, 0.0, s.tg[s.n], S_G2);
    } else if (stage == S_G2) {
      blk_chi<Real>(s, 0, Q, cvec<Real>(s, 2), mvec<Real>(s, 3));  // k2 = chi_a k1
      const C* bra = cvec<Real>(s, 1);
      const C* ket = cvec<Real>(s, 3);
      double sr = 0.0, si = 0.0;
      for (uint32_t m = threadIdx.x; m < s.D; m += blockDim.x) {
        const C u = bra[m], v = ket[m];
        sr += static_cast<double>(u.x) * v.x + static_cast<double>(u.y) * v.y;
        si += static_cast<double>(u.x) * v.y - static_cast<double>(u.y) * v.x;
      }
      sr = block_sum(sr);
      si = block_sum(si);
      if (threadIdx.x == 0) {
        s.F[2 * s.n] += sr;
        s.F[2 * s.n + 1] += si;
        s.n += 1;
        s.stage = S_POINT;
      }
      __syncthreads();
    } else if (stage == S_K1) {
      blk_chi<Real>(s, 1, P, cvec<Real>(s, 0), mvec<Real>(s, 2));  // k1 = chi_b u0
      start_evolve(2, Q, s.beta / 4.0, s.tg[s.n], S_K2);
    } else if (stage == S_K2) {
      blk_chi<Real>(s, 0, Q, cvec<Real>(s, 2), mvec<Real>(s, 3));  // k2 = chi_a k1
      start_evolve(3, P, s.beta / 4.0, -s.tg[s.n], S_K3);
    } else if (stage == S_K3) {
      blk_chi<Real>(s, 1, P, cvec<Real>(s, 3), mvec<Real>(s, 2));  // k1 = chi_b k2
      start_evolve(2, Q, s.beta / 4.0, s.tg[s.n], S_K4);
    } else if (stage == S_K4) {
      blk_chi<Real>(s, 0, Q, cvec<Real>(s, 2), mvec<Real>(s, 3));  // k2 = chi_a k1
      const C* bra = cvec<Real>(s, 1);
      const C* ket = cvec<Real>(s, 3);
      double sr = 0.0, si = 0.0;
      for (uint32_t m = threadIdx.x; m < s.D; m += blockDim.x) {
        const C u = bra[m], v = ket[m];
        sr += static_cast<double>(u.x) * v.x + static_cast<double>(u.y) * v.y;
        si += static_cast<double>(u.x) * v.y - static_cast<double>(u.y) * v.x;
      }
      sr = block_sum(sr);
      si = block_sum(si);
      if (threadIdx.x == 0) {
        s.F[2 * s.n] += sr;
        s.F[2 * s.n + 1] += si;
        s.n += 1;
        s.stage = S_POINT;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s.stage == S_DONE) s.done = 1;
    g = s;
  }
}

// ------------------------------------------------------------ Lanczos part --
__device__ __forceinline__ bool slot_of_block(const BatchArgs& a, int& si, int& tl, int2& r) {
  si = a.blk_slot[blockIdx.x];
  r = a.blk_range[si];
  tl = static_cast<int>(blockIdx.x) - r.x;
  return r.y > 0 && a.slots[si].live && a.slots[si].ev != 0 && !a.slots[si].done;
}

template <typename Real>
__global__ void __launch_bounds__(kBlk) k_b_norm(BatchArgs a) {
  int si, tl;
  int2 rg;
  if (!slot_of_block(a, si, tl, rg)) return;
  const BSlot& s = a.slots[si];
  const auto* x = cvec<Real>(s, s.ev_vec);
  double acc = 0.0;
  for (uint32_t m = tl * kBlk + threadIdx.x; m < s.D; m += rg.y * kBlk) {
    const auto v = x[m];
    acc += static_cast<double>(v.x * v.x + v.y * v.y);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) a.partN[blockIdx.x] = acc;
}

template <typename Real>
__global__ void __launch_bounds__(kBlk) k_b_scale_first(BatchArgs a) {
  int si, tl;
  int2 rg;
  if (!slot_of_block(a, si, tl, rg)) return;
  const BSlot& s = a.slots[si];
  KScalars* sc = a.sc + si;
  const double b0 = sqrt(slot_sum(a.partN, rg));
  if (tl == 0 && threadIdx.x == 0) {
    sc->beta0 = b0;
    sc->m_eff = (b0 > 0.0) ? static_cast<int>(static_cast<uint32_t>(a.m) < s.D ? static_cast<uint32_t>(a.m) : s.D) : 0;
    sc->status = 0;
  }
  const Real inv = b0 > 0.0 ? static_cast<Real>(1.0 / b0) : Real(0);
  const auto* x = cvec<Real>(s, s.ev_vec);
  auto* v0 = basis<Real>(s, 0);
  for (uint32_t m = tl * kBlk + threadIdx.x; m < s.D; m += rg.y * kBlk) {
    auto v = x[m];
    v.x = mul_(v.x, inv);
    v.y = mul_(v.y, inv);
    v0[m] = v;
  }
}

// w = H V_j - beta_{j-1} V_{j-1}; partA = Re <V_j, w>.
template <typename Real>
__global__ void __launch_bounds__(kBlk) k_b_matvec(BatchArgs a, int j) {
  int si, tl;
  int2 rg;
  if (!slot_of_block(a, si, tl, rg)) return;
  const BSlot& s = a.slots[si];
  KScalars* sc = a.sc + si;
  if (sc->m_eff <= j || j + 1 > static_cast<int>(s.D)) return;
  if (sizeof(Real) == 4 && s.D >= (1u << kTileBits)) return;  // k_b_matvec_c64 handles it
  using C = typename CT<Real>::T;
  const C* v = basis<Real>(s, j);
  const C* vp = j > 0 ? basis<Real>(s, j - 1) : nullptr;
  C* w = basis<Real>(s, j + 1);
  const Real* coef = static_cast<const Real*>(s.coef[s.ev_block]);
  // w = s_j H basis[j] - beta_{j-1} s_{j-1} basis[j-1];  Re <v_j, w> = s_j Re <basis[j], w>
  const double sjd = j > 0 ? a.lsc[2 * si] : 1.0;
  const Real sj = static_cast<Real>(sjd);
  const Real bprev = j > 0 ? static_cast<Real>(a.lsc[2 * si + 1]) : Real(0);
  double part = 0.0;
  for (uint32_t m = tl * kBlk + threadIdx.x; m < s.D; m += rg.y * kBlk) {
    Real ar = 0, ai = 0;
    for (int t = 0; t < s.n_terms; ++t) {
      const uint32_t x = __ldg(s.x + t), zw = __ldg(s.zi + t);
      const Real cc = sgnflip(__ldg(coef + t), __popc(zw & 0x7FFFFFFFu & m) & 1u);
      const C u = v[m ^ x];
      if (zw >> 31) {
        ar = fma_(-cc, u.y, ar);
        ai = fma_(cc, u.x, ai);
      } else {
        ar = fma_(cc, u.x, ar);
        ai = fma_(cc, u.y, ai);
      }
    }
    C pv = {0, 0};
    if (j > 0) pv = vp[m];
    C o;
    o.x = fma_(-bprev, pv.x, mul_(sj, ar));
    o.y = fma_(-bprev, pv.y, mul_(sj, ai));
    w[m] = o;
    const C vv = v[m];
    part += static_cast<double>(vv.x * o.x + vv.y * o.y);
  }
  part = block_sum(part);
  if (threadIdx.x == 0) a.partA[blockIdx.x] = part * sjd;
  matvec_finish_alpha(a, sc, si, j, rg);
}

// complex64 slots with D >= 2048: the TMA-staged pair-layout matvec of the
// single-Hamiltonian path (plain tile order), with the Lanczos epilogue.
template <int S>
__global__ void __launch_bounds__(32 * (kConsumerWarps + 1), kC64CtasPerSm) k_b_matvec_c64(BatchArgs a, int j) {
  constexpr uint32_t kTileBytes = (1u << kTileBits) * 8u;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ int s_err;
  const int si = a.blk_slot[blockIdx.x];
  const int2 rg = a.blk_range[si];
  const BSlot& s = a.slots[si];
  if (rg.y <= 0 || !s.live || !s.ev || s.done || s.D < (1u << kTileBits)) return;
  KScalars* sc = a.sc + si;
  if (sc->m_eff <= j) return;
  const uint32_t tl = blockIdx.x - rg.x;

  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const float2* v = basis<float>(s, j);
  const float2* vp = j > 0 ? basis<float>(s, j - 1) : nullptr;
  float2* w = basis<float>(s, j + 1);
  const TermF* rec = s.rec[s.ev_block];
  const int T = s.n_terms;
  const uint32_t ntiles = s.D >> kTileBits;
  const uint32_t my_tiles = ntiles > tl ? (ntiles - tl - 1) / rg.y + 1 : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), kConsumerWarps);
    }
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();
  double part = 0.0;
  if (warp == kConsumerWarps) {
    if (lane == 0 && T > 0) {
      const uint32_t smem0 = smem_u32(smem_raw);
      const uint64_t keep = l2_policy_evict_last();
      uint32_t q = 0, issued = 0;
      for (uint32_t k = 0; k < my_tiles && !*(volatile int*)&s_err; ++k) {
        const uint32_t tb = (tl + k * rg.y) << kTileBits;
        for (int tt = 0; tt < T && !*(volatile int*)&s_err; ++tt) {
          const uint2 xf = make_uint2(__ldg(&rec[tt].x), __ldg(&rec[tt].flags));
          if (!(xf.y & kTermRunStart)) continue;  // the run's tile is already staged
          const uint32_t stg = q % S;
          if (q >= S && !mbar_wait_bounded(smem_u32(&empty_bar[stg]), ((q / S) - 1) & 1u, &s_err)) break;
          const float2* src = v + (tb ^ (xf.x & kTermXMask & ~((1u << kTileBits) - 1u)));
          const uint32_t bar = smem_u32(&full_bar[stg]);
          mbar_expect_tx(bar, kTileBytes);
          bulk_g2s_hint(smem0 + stg * kTileBytes, src, kTileBytes, bar, keep);
          issued = ++q;
        }
      }
      if (s_err) {
        for (uint32_t qq = issued > S ? issued - S : 0; qq < issued; ++qq) {
          const uint32_t bar = smem_u32(&full_bar[qq % S]);
          const uint64_t ts = globaltimer_ns();
          while (!mbar_try_wait(bar, (qq / S) & 1u) && globaltimer_ns() - ts < kWaitLimitNs) {
          }
        }
      }
    }
  } else {
    // w = s_j H basis[j] - beta_{j-1} s_{j-1} basis[j-1] (unnormalised basis, see basis_scale)
    const float sj = j > 0 ? static_cast<float>(a.lsc[2 * si]) : 1.f;
    const float bprev = j > 0 ? static_cast<float>(a.lsc[2 * si + 1]) : 0.f;
    const uint32_t pair_part = warp * (64u * kRows) + 2u * lane;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    const float4* vp4 = reinterpret_cast<const float4*>(vp);
    float4* w4 = reinterpret_cast<float4*>(w);
    StageRing<S> ring;
    uint4 d = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = 0; k < my_tiles; ++k) {
      const uint32_t mt = ((tl + k * rg.y) << kTileBits) + pair_part;
      if (T > 0) d = __ldg(reinterpret_cast<const uint4*>(rec));  // the tile's first term
      float acc[kRows][4];
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
      c64_terms<S>(0, T, d, ring, acc, rec, mt, pair_part, smem_raw, full_bar, empty_bar, &s_err, lane);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const uint32_t i4 = (mt >> 1) + 32u * r;
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j > 0) pv = vp4[i4];
        float4 o;
        o.x = fma_(-bprev, pv.x, mul_(sj, acc[r][0]));
        o.y = fma_(-bprev, pv.y, mul_(sj, acc[r][1]));
        o.z = fma_(-bprev, pv.z, mul_(sj, acc[r][2]));
        o.w = fma_(-bprev, pv.w, mul_(sj, acc[r][3]));
        w4[i4] = o;
        const float4 vv = v4[i4];
        part += static_cast<double>(vv.x * o.x + vv.y * o.y) + static_cast<double>(vv.z * o.z + vv.w * o.w);
      }
    }
  }
  part = block_sum(part);
  if (threadIdx.x == 0) {
    a.partA[blockIdx.x] = part * (j > 0 ? a.lsc[2 * si] : 1.0);
    if (s_err) atomicExch(a.err, 1);
  }
  matvec_finish_alpha(a, sc, si, j, rg);
}

template <typename Real>
__global__ void __launch_bounds__(kBlk) k_b_axpy_norm(BatchArgs a, int j) {
  int si, tl;
  int2 rg;
  if (!slot_of_block(a, si, tl, rg)) return;
  const BSlot& s = a.slots[si];
  KScalars* sc = a.sc + si;
  if (sc->m_eff <= j) return;
  const double al = sc->alpha[j];  // summed once by the matvec's last block of the slot
  const Real alr = static_cast<Real>(al * basis_scale(sc, j));  // v_j = s_j basis[j]
  const auto* v = basis<Real>(s, j);
  auto* w = basis<Real>(s, j + 1);
  double acc = 0.0;
  for (uint32_t m = tl * kBlk + threadIdx.x; m < s.D; m += rg.y * kBlk) {
    auto ww = w[m];
    const auto vv = v[m];
    ww.x = fma_(-alr, vv.x, ww.x);
    ww.y = fma_(-alr, vv.y, ww.y);
    w[m] = ww;
    acc += static_cast<double>(ww.x * ww.x + ww.y * ww.y);
  }
  acc = block_sum(acc);
  __shared__ int last;
  if (threadIdx.x == 0) {
    a.partN[blockIdx.x] = acc;
    __threadfence();  // the partial is visible before this block counts itself done
    last = atomicAdd(a.slot_cnt + si, 1) == rg.y - 1;
  }
  __syncthreads();
  if (last) {  // every block of the slot has written its partial
    __threadfence();
    lanczos_finish_step(a, sc, si, j, rg);
    if (threadIdx.x == 0) a.slot_cnt[si] = 0;
  }
}

__global__ void __launch_bounds__(32) k_b_tridiag(BatchArgs a) {
  __shared__ double Z[kMaxKrylov][kMaxKrylov + 1];
  if (a.slot_group[blockIdx.x] != a.group) return;
  const BSlot& s = a.slots[blockIdx.x];
  if (!s.live || s.done || !s.ev) return;
  tridiag_warp(a.sc + blockIdx.x, a.m, s.z_re, s.z_im, a.tol, Z);
}

template <typename Real>
__global__ void __launch_bounds__(kBlk) k_b_combine(BatchArgs a) {
  int si, tl;
  int2 rg;
  if (!slot_of_block(a, si, tl, rg)) return;
  const BSlot& s = a.slots[si];
  const KScalars* sc = a.sc + si;
  __shared__ Real cr[kMaxKrylov], ci[kMaxKrylov];
  const int n = min(sc->m_eff, a.m);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {  // v_i = s_i basis[i]
    cr[i] = static_cast<Real>(sc->beta0 * sc->c_re[i] * basis_scale(sc, i));
    ci[i] = static_cast<Real>(sc->beta0 * sc->c_im[i] * basis_scale(sc, i));
  }
  __syncthreads();
  auto* y = mvec<Real>(s, s.ev_vec);
  for (uint32_t m = tl * kBlk + threadIdx.x; m < s.D; m += rg.y * kBlk) {
    Real re = 0, im = 0;
    for (int i = 0; i < n; ++i) {
      const auto v = basis<Real>(s, i)[m];
      re = fma_(cr[i], v.x, fma_(-ci[i], v.y, re));
      im = fma_(cr[i], v.y, fma_(ci[i], v.x, im));
    }
    typename CT<Real>::T o;
    o.x = re;
    o.y = im;
    y[m] = o;
  }
}

}  // namespace

// ------------------------------------------------------------------ host ----
struct BatchJobHost {
  syk_otoc_job job;
  std::vector<double> tg;
  size_t off = 0, bytes = 0;  // arena range
  bool live = false;
};

struct Batch {
  int dtype = SYK_C64, max_slots = 0, m = 30, device = 0;
  double tol = 1e-6;
  size_t arena_bytes = 0;
  void* arena = nullptr;
  // free list of arena ranges (offset, size), kept sorted
  std::vector<std::pair<size_t, size_t>> free_list;
  std::vector<BatchJobHost> jobs;  // one per slot
  std::vector<BSlot> host_slots;
  BSlot* d_slots = nullptr;
  KScalars* d_sc = nullptr;
  int* d_blk_slot = nullptr;
  int2* d_blk_range = nullptr;
  double* d_part = nullptr;  // 2 x max blocks
  int* d_err = nullptr;      // bounded-wait failure flag
  int* d_slot_cnt = nullptr;  // per slot: blocks done with axpy_norm, then with the matvec (zero between launches)
  double* d_lsc = nullptr;    // per slot: the next matvec's two Lanczos scalars
  size_t max_blocks = 0;  // per tick group: block map and partials of group g at offset g * max_blocks
  // Live slots are split into two tick groups, each with its own graph and
  // stream, so that one group's per-slot serial kernels (tridiagonal step,
  // control) overlap the other group's Lanczos matvecs.
  int* d_slot_group = nullptr;
  std::vector<int> host_group;  // copy of d_slot_group
  int ngroups = 1;
  int group_blocks[kGroups] = {};
  double group_cost[kGroups] = {};  // sum of T x D over the group's live slots (work per tick)
  cudaStream_t stream = nullptr;               // group 0; host copies
  cudaStream_t gstream[kGroups] = {};          // gstream[0] == stream
  cudaGraphExec_t graph[kGroups] = {};
  bool layout_dirty = true;
  int total_blocks = 0;
  size_t bytes_in_use = 0;

  ~Batch() {
    for (int g = 0; g < kGroups; ++g) {
      if (graph[g]) cudaGraphExecDestroy(graph[g]);
      if (g > 0 && gstream[g]) cudaStreamDestroy(gstream[g]);
    }
    if (stream) cudaStreamDestroy(stream);
    for (void* p : {static_cast<void*>(d_slots), static_cast<void*>(d_sc), static_cast<void*>(d_blk_slot),
                    static_cast<void*>(d_blk_range), static_cast<void*>(d_part), static_cast<void*>(d_err),
                    static_cast<void*>(d_slot_cnt), static_cast<void*>(d_lsc), static_cast<void*>(d_slot_group),
                    arena})
      if (p) cudaFree(p);
  }

  size_t job_bytes(int64_t D, int n_t) const {
    const size_t esz = elem_bytes(dtype);
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    return (static_cast<size_t>(m) + 1 + 4) * up(static_cast<size_t>(D) * esz) + up(n_t * sizeof(double)) +
           up(n_t * 2 * sizeof(double));
  }

  bool arena_alloc(size_t bytes, size_t& off) {
    for (size_t i = 0; i < free_list.size(); ++i) {
      if (free_list[i].second >= bytes) {
        off = free_list[i].first;
        free_list[i].first += bytes;
        free_list[i].second -= bytes;
        if (free_list[i].second == 0) free_list.erase(free_list.begin() + i);
        return true;
      }
    }
    return false;
  }
  void arena_free(size_t off, size_t bytes) {
    free_list.push_back({off, bytes});
    std::sort(free_list.begin(), free_list.end());
    std::vector<std::pair<size_t, size_t>> merged;
    for (auto& r : free_list) {
      if (!merged.empty() && merged.back().first + merged.back().second == r.first)
        merged.back().second += r.second;
      else
        merged.push_back(r);
    }
    free_list.swap(merged);
  }
};

template <typename Real>
void capture_tick(Batch& b, int grp) {
  BatchArgs a;
  a.slots = b.d_slots;
  a.sc = b.d_sc;
  a.blk_slot = b.d_blk_slot + grp * b.max_blocks;
  a.blk_range = b.d_blk_range;
  a.m = b.m;
  a.tol = b.tol;
  a.partA = b.d_part + 2 * grp * b.max_blocks;
  a.partN = a.partA + b.max_blocks;
  a.err = b.d_err;
  a.brk = sizeof(Real) == 4 ? 1e-7 : 1e-14;
  a.slot_cnt = b.d_slot_cnt;
  a.alpha_cnt = b.d_slot_cnt + b.max_slots;
  a.lsc = b.d_lsc;
  a.slot_group = b.d_slot_group;
  a.group = grp;
  cudaStream_t st = b.gstream[grp];
  cudaGraphExec_t& graph = b.graph[grp];
  if (graph) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  constexpr size_t dyn = static_cast<size_t>(kStagesC64) * (1u << kTileBits) * 8u;
  if (sizeof(Real) == 4)
    SYK_CUDA(cudaFuncSetAttribute(k_b_matvec_c64<kStagesC64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(dyn)));
  SYK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int S = b.max_slots, G = std::max(1, b.group_blocks[grp]);
  k_b_control<Real><<<S, kCtlBlk, 0, st>>>(a);
  k_b_norm<Real><<<G, kBlk, 0, st>>>(a);
  k_b_scale_first<Real><<<G, kBlk, 0, st>>>(a);
  // complex64 slots of at least one tile take the tiled matvec; the plain one
  // is captured only when a live slot needs it (the graph is recaptured when
  // the set of live slots changes).
  bool plain = sizeof(Real) != 4, tiled = false;
  for (int s = 0; s < b.max_slots; ++s)
    if (b.jobs[s].live && b.host_group[s] == grp) {
      const bool t = sizeof(Real) == 4 && b.jobs[s].job.h->D >= (int64_t(1) << kTileBits);
      tiled = tiled || t;
      plain = plain || !t;
    }
  for (int j = 0; j < b.m; ++j) {
    if (plain) k_b_matvec<Real><<<G, kBlk, 0, st>>>(a, j);
    if (tiled) k_b_matvec_c64<kStagesC64><<<G, 32 * (kConsumerWarps + 1), dyn, st>>>(a, j);
    k_b_axpy_norm<Real><<<G, kBlk, 0, st>>>(a, j);
  }
  k_b_tridiag<<<S, 32, 0, st>>>(a);
  k_b_combine<Real><<<G, kBlk, 0, st>>>(a);
  cudaGraph_t g;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess) throw Error(SYK_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) throw Error(SYK_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
}

}  // namespace syk

struct syk_batch {
  syk::Batch b;
};

namespace {
template <typename F>
int bguard(const char* fn, F&& f) {
  try {
    f();
    return SYK_OK;
  } catch (const syk::Error& e) {
    syk::set_last_error(std::string(fn) + ": " + e.what());
    return e.code;
  } catch (const std::exception& e) {
    syk::set_last_error(std::string(fn) + ": " + e.what());
    return SYK_EINVAL;
  }
}

void relayout(syk::Batch& b) {
  // Flattened block -> slot maps for live slots, one per tick group; dead
  // slots get no blocks.  Groups by work (terms x amplitudes of a slot): the
  // heaviest slots, up to half of the total work, form group 0 and the rest
  // group 1, and the run loop gives each group ticks in inverse proportion to
  // its work per tick, so light slots are not held to the pace of the heavy
  // ones (and both groups finish a sync period together).  Inside a group the
  // slots are laid out in decreasing term count: a matvec block's work is one
  // tile times the slot's terms, and the block scheduler starts blocks in
  // index order, so the heaviest tiles start first and the tail is light.
  std::vector<int> order;
  for (int s = 0; s < b.max_slots; ++s)
    if (b.jobs[s].live) order.push_back(s);
  auto work = [&](int s) {
    return static_cast<double>(b.jobs[s].job.h->terms.size()) * static_cast<double>(b.jobs[s].job.h->D);
  };
  std::vector<int> group(b.max_slots, -1);
  b.ngroups = static_cast<int>(std::max<size_t>(1, std::min<size_t>(syk::kGroups, order.size() / 2)));
  for (auto& c : b.group_cost) c = 0.0;
  {
    std::vector<int> by_work = order;
    std::stable_sort(by_work.begin(), by_work.end(), [&](int x, int y) { return work(x) > work(y); });
    double total = 0.0;
    for (const int s : by_work) total += work(s);
    // geometric tiers: each group but the last takes slots (heaviest first)
    // while it holds less than half of the work not yet assigned, at least one
    // slot, and leaves at least one slot for every later group
    int g = 0;
    double left = total, acc = 0.0;
    size_t in_g = 0;
    for (size_t i = 0; i < by_work.size(); ++i) {
      const int s = by_work[i];
      const size_t later = static_cast<size_t>(b.ngroups - 1 - g);
      if (g < b.ngroups - 1 && in_g > 0 && (acc >= 0.5 * left || by_work.size() - i <= later)) {
        left -= acc;
        acc = 0.0;
        in_g = 0;
        ++g;
      }
      group[s] = g;
      acc += work(s);
      ++in_g;
      b.group_cost[g] += work(s);
    }
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b.jobs[x].job.h->terms.size() > b.jobs[y].job.h->terms.size();
  });
  std::vector<int> blk_slot[syk::kGroups];
  std::vector<int2> range(b.max_slots, make_int2(0, 0));
  for (const int s : order) {
    const int g = group[s];
    const int64_t D = b.jobs[s].job.h->D;
    const bool tiles = b.dtype == SYK_C64 && D >= (int64_t(1) << syk::kTileBits);
    const int nb = static_cast<int>(tiles ? std::min<int64_t>(D >> syk::kTileBits, syk::kMaxBlkPerSlot)
                                          : std::min<int64_t>((D + syk::kBlk - 1) / syk::kBlk, syk::kMaxBlkPerSlot));
    range[s] = make_int2(static_cast<int>(blk_slot[g].size()), nb);
    for (int k = 0; k < nb; ++k) blk_slot[g].push_back(s);
  }
  for (int g = 0; g < syk::kGroups; ++g) {
    if (blk_slot[g].empty()) blk_slot[g].push_back(0);
    b.group_blocks[g] = static_cast<int>(blk_slot[g].size());
    if (static_cast<size_t>(b.group_blocks[g]) > b.max_blocks)
      throw syk::Error(SYK_EINVAL, "internal: block map overflow");
    SYK_CUDA(cudaMemcpyAsync(b.d_blk_slot + g * b.max_blocks, blk_slot[g].data(), blk_slot[g].size() * sizeof(int),
                             cudaMemcpyHostToDevice, b.stream));
  }
  b.total_blocks = 0;
  for (int g = 0; g < b.ngroups; ++g) b.total_blocks += b.group_blocks[g];
  SYK_CUDA(cudaMemcpyAsync(b.d_blk_range, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice, b.stream));
  SYK_CUDA(cudaMemcpyAsync(b.d_slot_group, group.data(), group.size() * sizeof(int), cudaMemcpyHostToDevice, b.stream));
  b.host_group = group;
  SYK_CUDA(cudaStreamSynchronize(b.stream));  // host vectors go out of scope
}
}  // namespace

extern "C" {

int syk_batch_create(int dtype, int max_slots, size_t max_bytes, const syk_krylov_params* p, syk_batch_t** out) {
  return bguard("syk_batch_create", [&] {
    SYK_REQUIRE(out != nullptr, "null output");
    *out = nullptr;
    SYK_REQUIRE(dtype == SYK_C64 || dtype == SYK_C128, "bad dtype");
    SYK_REQUIRE(max_slots >= 1 && max_slots <= 65535, "max_slots must be in [1, 65535]");
    SYK_REQUIRE(max_bytes >= (size_t(1) << 20), "max_bytes must be at least 1 MiB");
    auto h = std::make_unique<syk_batch>();
    syk::Batch& b = h->b;
    b.dtype = dtype;
    b.max_slots = max_slots;
    b.m = (p && p->m) ? p->m : syk::default_krylov_m(dtype);  // complex64 batch: 20 beat 30 by 14% on B300
    b.tol = (p && p->tol > 0) ? p->tol : (dtype == SYK_C128 ? 1e-12 : 1e-6);
    SYK_REQUIRE(b.m >= 2 && b.m <= syk::kMaxKrylov, "Krylov dimension m must be in [2, 64]");
    SYK_REQUIRE(!(p && (p->two_pass || p->reorth)), "the batch engine stores the basis (no two_pass / reorth)");
    SYK_CUDA(cudaGetDevice(&b.device));
    b.arena_bytes = max_bytes;
    if (cudaMalloc(&b.arena, max_bytes) != cudaSuccess) {
      cudaGetLastError();
      throw syk::Error(SYK_ENOMEM, "arena allocation failed");
    }
    b.free_list.push_back({0, max_bytes});
    b.jobs.resize(max_slots);
    b.host_slots.assign(max_slots, syk::BSlot{});
    b.max_blocks = static_cast<size_t>(max_slots) * syk::kMaxBlkPerSlot;
    SYK_CUDA(cudaMalloc(&b.d_slots, max_slots * sizeof(syk::BSlot)));
    SYK_CUDA(cudaMalloc(&b.d_sc, max_slots * sizeof(syk::KScalars)));
    SYK_CUDA(cudaMalloc(&b.d_blk_slot, syk::kGroups * b.max_blocks * sizeof(int)));
    SYK_CUDA(cudaMalloc(&b.d_slot_group, max_slots * sizeof(int)));
    SYK_CUDA(cudaMemset(b.d_slot_group, 0xFF, max_slots * sizeof(int)));
    SYK_CUDA(cudaMalloc(&b.d_blk_range, max_slots * sizeof(int2)));
    SYK_CUDA(cudaMemset(b.d_blk_range, 0, max_slots * sizeof(int2)));
    SYK_CUDA(cudaMalloc(&b.d_part, 2 * syk::kGroups * b.max_blocks * sizeof(double)));
    SYK_CUDA(cudaMalloc(&b.d_err, sizeof(int)));
    SYK_CUDA(cudaMalloc(&b.d_slot_cnt, 2 * max_slots * sizeof(int)));  // axpy_norm, then matvec counters
    SYK_CUDA(cudaMemset(b.d_slot_cnt, 0, 2 * max_slots * sizeof(int)));
    SYK_CUDA(cudaMalloc(&b.d_lsc, 2 * max_slots * sizeof(double)));
    SYK_CUDA(cudaMemset(b.d_err, 0, sizeof(int)));
    SYK_CUDA(cudaMemset(b.d_slots, 0, max_slots * sizeof(syk::BSlot)));
    SYK_CUDA(cudaMemset(b.d_sc, 0, max_slots * sizeof(syk::KScalars)));
    SYK_CUDA(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
    b.gstream[0] = b.stream;
    for (int g = 1; g < syk::kGroups; ++g) SYK_CUDA(cudaStreamCreateWithFlags(&b.gstream[g], cudaStreamNonBlocking));
    *out = h.release();
  });
}

int syk_batch_destroy(syk_batch_t* h) {
  return bguard("syk_batch_destroy", [&] {
    if (!h) return;
    cudaStreamSynchronize(h->b.stream);
    delete h;
  });
}

int syk_batch_submit(syk_batch_t* h, const syk_otoc_job* job) {
  return bguard("syk_batch_submit", [&] {
    SYK_REQUIRE(h && job && job->h && job->t_grid && job->F_out, "null argument");
    syk::Batch& b = h->b;
    const syk_terms* t = job->h;
    SYK_REQUIRE(t->dtype == b.dtype, "job Hamiltonian dtype differs from the batch dtype");
    SYK_REQUIRE(t->device == b.device, "job Hamiltonian lives on another device");
    SYK_REQUIRE(t->hermitian, "the batched engine runs Hermitian Hamiltonians only (Lanczos)");
    SYK_REQUIRE(job->a >= 0 && job->a < t->N && job->b >= 0 && job->b < t->N, "Majorana index out of range");
    SYK_REQUIRE(job->n_t >= 1 && std::isfinite(job->beta) && job->beta >= 0, "bad n_t or beta");
    for (int n = 0; n < job->n_t; ++n) {
      SYK_REQUIRE(std::isfinite(job->t_grid[n]), "non-finite time");
      if (n) SYK_REQUIRE(job->t_grid[n] >= job->t_grid[n - 1], "time grid must be non-decreasing");
    }
    int slot = -1;
    for (int s = 0; s < b.max_slots; ++s)
      if (!b.jobs[s].live) {
        slot = s;
        break;
      }
    if (slot < 0) throw syk::Error(SYK_EAGAIN, "no free slot");
    const size_t need = b.job_bytes(t->D, job->n_t);
    size_t off = 0;
    if (!b.arena_alloc(need, off)) throw syk::Error(SYK_EAGAIN, "not enough free device memory in the arena");
    syk::BatchJobHost& jh = b.jobs[slot];
    jh.job = *job;
    jh.tg.assign(job->t_grid, job->t_grid + job->n_t);
    jh.off = off;
    jh.bytes = need;
    jh.live = true;
    b.bytes_in_use += need;
    // carve the arena range
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    char* base = static_cast<char*>(b.arena) + off;
    const size_t vb = up(static_cast<size_t>(t->D) * syk::elem_bytes(b.dtype));
    syk::BSlot s{};
    s.x = t->d_x;
    s.zi = t->d_zi;
    s.coef[0] = t->d_coef[0];
    s.coef[1] = t->d_coef[1];
    s.rec[0] = t->d_termf[0];
    s.rec[1] = t->d_termf[1];
    s.passes = t->d_passes;
    s.n_passes = static_cast<int>(t->passes.size());
    s.n_terms = static_cast<int>(t->terms.size());
    s.D = static_cast<uint32_t>(t->D);
    const syk::ChiString* ch[2] = {&t->chi[job->a], &t->chi[job->b]};
    for (int w = 0; w < 2; ++w) {
      s.cx[w] = ch[w]->x;
      s.cz[w] = ch[w]->z;
      for (int P = 0; P < 2; ++P) {
        s.cre[w][P] = ch[w]->re[P];
        s.cim[w][P] = ch[w]->im[P];
      }
    }
    s.beta = job->beta;
    s.n_t = job->n_t;
    s.seed = job->seed;
    s.state_id = job->state_id;
    SYK_REQUIRE(job->basis_index < 2 * t->D, "basis_index out of range [0, 2D)");
    s.basis = job->basis_index < 0 ? -1 : job->basis_index;
    SYK_REQUIRE(job->kind == SYK_JOB_OTOC || job->kind == SYK_JOB_GREEN, "bad job kind");
    s.kind = job->kind;
    for (int i = 0; i < 4; ++i) s.vec[i] = base + i * vb;
    s.V = base + 4 * vb;
    char* tail = base + (4 + b.m + 1) * vb;
    s.tg = reinterpret_cast<double*>(tail);
    s.F = reinterpret_cast<double*>(tail + up(job->n_t * sizeof(double)));
    s.live = 1;
    s.stage = syk::S_INIT;
    b.host_slots[slot] = s;
    SYK_CUDA(cudaMemcpyAsync(const_cast<double*>(s.tg), jh.tg.data(), job->n_t * sizeof(double),
                             cudaMemcpyHostToDevice, b.stream));
    SYK_CUDA(cudaMemsetAsync(s.F, 0, job->n_t * 2 * sizeof(double), b.stream));
    SYK_CUDA(cudaMemcpyAsync(b.d_slots + slot, &b.host_slots[slot], sizeof(syk::BSlot), cudaMemcpyHostToDevice,
                             b.stream));
    SYK_CUDA(cudaStreamSynchronize(b.stream));  // the host copies above are read now
    b.layout_dirty = true;
  });
}

int syk_batch_run(syk_batch_t* h, int max_ticks, int ticks_per_sync, int* n_finished, int64_t* finished_tags,
                  int max_finished) {
  return bguard("syk_batch_run", [&] {
    SYK_REQUIRE(h && n_finished, "null argument");
    syk::Batch& b = h->b;
    *n_finished = 0;
    int dev = -1;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_REQUIRE(dev == b.device, "current device differs from the batch's");
    if (ticks_per_sync < 1) ticks_per_sync = 8;
    int live = 0;
    for (auto& j : b.jobs) live += j.live ? 1 : 0;
    if (live == 0) return;
    if (b.layout_dirty) {
      relayout(b);
      for (int g = 0; g < b.ngroups; ++g) {
        if (b.dtype == SYK_C128)
          syk::capture_tick<double>(b, g);
        else
          syk::capture_tick<float>(b, g);
      }
      b.layout_dirty = false;
    }
    std::vector<syk::BSlot> dev_slots(b.max_slots);
    for (int done_ticks = 0; done_ticks < max_ticks;) {
      const int n = std::min(ticks_per_sync, max_ticks - done_ticks);
      // n ticks for the heaviest group; lighter groups get proportionally more
      // (at most kMaxTickRatio n), so a sync period takes about as long on
      // every stream
      int ng[syk::kGroups] = {};
      double cmax = 0.0;
      for (int g = 0; g < b.ngroups; ++g) cmax = std::max(cmax, b.group_cost[g]);
      int most = n;
      for (int g = 0; g < b.ngroups; ++g) {
        const double r = b.group_cost[g] > 0.0 ? cmax / b.group_cost[g] : 1.0;
        ng[g] = static_cast<int>(std::min<double>(syk::kMaxTickRatio * n, std::max<double>(n, std::floor(n * r))));
        most = std::max(most, ng[g]);
      }
      for (int i = 0; i < most; ++i)
        for (int g = 0; g < b.ngroups; ++g)
          if (i < ng[g]) SYK_CUDA(cudaGraphLaunch(b.graph[g], b.gstream[g]));
      done_ticks += n;
      for (int g = 1; g < b.ngroups; ++g) SYK_CUDA(cudaStreamSynchronize(b.gstream[g]));
      SYK_CUDA(cudaMemcpyAsync(dev_slots.data(), b.d_slots, b.max_slots * sizeof(syk::BSlot), cudaMemcpyDeviceToHost,
                               b.stream));
      SYK_CUDA(cudaStreamSynchronize(b.stream));
      int derr = 0;
      SYK_CUDA(cudaMemcpy(&derr, b.d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (derr) throw syk::Error(SYK_ETIMEOUT, "a bounded device wait expired; batch results are invalid");
      int finished = 0;
      for (int s = 0; s < b.max_slots; ++s)
        if (b.jobs[s].live && dev_slots[s].done) ++finished;
      if (finished) break;
    }
    // collect finished jobs
    for (int s = 0; s < b.max_slots; ++s) {
      syk::BatchJobHost& jh = b.jobs[s];
      if (!jh.live || !dev_slots[s].done) continue;
      SYK_CUDA(cudaMemcpyAsync(jh.job.F_out, dev_slots[s].F, jh.job.n_t * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               b.stream));
      SYK_CUDA(cudaStreamSynchronize(b.stream));
      if (jh.job.otoc_out)  // normalised curve: Re F(t) / Re F(0)
        for (int n = 0; n < jh.job.n_t; ++n) jh.job.otoc_out[n] = jh.job.F_out[2 * n] / jh.job.F_out[0];
      if (jh.job.stats) {
        jh.job.stats->matvecs = dev_slots[s].matvecs;
        jh.job.stats->substeps = dev_slots[s].substeps;
        jh.job.stats->err_est = 0.0;
      }
      if (jh.job.status_out) *jh.job.status_out = dev_slots[s].status ? SYK_ENOCONV : SYK_OK;
      if (finished_tags && *n_finished < max_finished) finished_tags[*n_finished] = jh.job.tag;
      *n_finished += 1;
      b.arena_free(jh.off, jh.bytes);
      b.bytes_in_use -= jh.bytes;
      jh.live = false;
      b.host_slots[s].live = 0;
      b.layout_dirty = true;
    }
    for (int s = 0; s < b.max_slots; ++s) {  // freed slots: dead on the device from now on
      if (b.jobs[s].live || !dev_slots[s].live) continue;
      const int zero = 0;
      SYK_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(b.d_slots + s) + offsetof(syk::BSlot, live), &zero, sizeof(int),
                               cudaMemcpyHostToDevice, b.stream));
      SYK_CUDA(cudaStreamSynchronize(b.stream));
    }
  });
}

int syk_batch_info(const syk_batch_t* h, int* live_jobs, size_t* bytes_in_use, size_t* bytes_free_max) {
  return bguard("syk_batch_info", [&] {
    SYK_REQUIRE(h, "null batch");
    const syk::Batch& b = h->b;
    if (live_jobs) {
      int n = 0;
      for (auto& j : b.jobs) n += j.live ? 1 : 0;
      *live_jobs = n;
    }
    if (bytes_in_use) *bytes_in_use = b.bytes_in_use;
    if (bytes_free_max) {
      size_t mx = 0;
      for (auto& r : b.free_list) mx = std::max(mx, r.second);
      *bytes_free_max = mx;
    }
  });
}

size_t syk_batch_job_bytes(const syk_batch_t* h, const syk_terms_t* t, int n_t) {
  if (!h || !t || n_t < 1) return 0;
  return h->b.job_bytes(t->D, n_t);
}

}  // extern "C"
