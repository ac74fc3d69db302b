// Device kernels of the sparse-SYK hot path.  H_P psi is the matrix-free
// Pauli-string action of Algorithm 1 (supplement Sec. I.A), with optional
// fused Lanczos epilogues, in four forms by vector size and type:
//  * k_matvec_c64  — complex64, >= 2048 amplitudes: warp-specialised TMA
//                    pipeline over L2-blocked passes (the benchmark kernel);
//  * k_matvec_tma  — complex128, >= 2048 amplitudes: TMA-staged tiles;
//  * k_matvec      — fewer than 2048 amplitudes: coalesced gathers (below);
//  * k_matvec_tiny — fewer than 32 amplitudes;
//  * k_sum_chunks  — the in-order sum of a split pass's chunks;
//  * k_chi         — one Majorana between parity blocks;
//  * k_random      — Philox4x32-10 + Box-Muller typical-state amplitudes;
//  * vector kernels for the Lanczos recurrence and the OTOC inner products.
//
// k_matvec layout.  A warp owns 32*R consecutive output amplitudes
// m = base + 32 r + lane (r < R).  For a term (x, z, c) the input of lane
// `lane` in row r is psi[(row ^ x_hi) | (lane ^ x_lo)] with x_lo = x & 31,
// so every load instruction of the warp reads one contiguous, aligned
// 32-amplitude segment (coalesced).  The sign (-1)^{popc(z & m)} splits into
// a per-lane part (popc(z & lane), once per term) and a per-row part
// (popc(z & row), warp-uniform), both folded into the coefficient's sign bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>

#include "device_common.cuh"
#include "tma_common.cuh"
#include "kernels.cuh"

namespace syk {
namespace {

enum { EPI_STORE = 0, EPI_LANCZOS = 1, EPI_RECUR = 2 };

template <typename Real>
struct MV {
  TermsView<Real> tv;
  const PassPlan* pass;  // device pointer to this launch's pass
  const TermF* rec;      // complex64: packed (x, z, c) records of the block being applied
  const typename CT<Real>::T* psi;
  typename CT<Real>::T* out;
  uint64_t D;
  const typename CT<Real>::T* vprev;  // Lanczos: v_{j-1} (null for j = 0)
  typename CT<Real>::T* y;            // second pass: accumulated result
  double* partial;                    // Lanczos: Re <v_j, w> per block
  const KScalars* sc;
  int j;
  unsigned long long* sched = nullptr;  // complex64 EPI_STORE: [0] next item, [1] CTAs finished
  uint32_t ny = 1;                      // complex64 EPI_STORE: states in this launch (chunks when split)
  const typename CT<Real>::T* prev = nullptr;  // complex64 split pass: the partial sum of earlier passes
  int chunk_terms = 0;                         // complex64 split pass: terms per chunk
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

// ACCUM: add the partial sum already in `out` (passes after the first).  The
// Lanczos epilogues run only in the last pass of a launch sequence.
template <typename Real, int R, int EPI, bool ACCUM>
__global__ void __launch_bounds__(256) k_matvec(MV<Real> p) {
  using C = typename CT<Real>::T;
  if (EPI == EPI_LANCZOS && p.sc->m_eff <= p.j) return;
  if (EPI == EPI_RECUR && p.j + 1 >= p.sc->m_eff) return;
  const int t0 = p.pass->t0, ti = p.pass->ti, t1 = p.pass->t1;
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
    // R == 8 tiles are 2^kTileBits amplitudes placed by the pass's deposit tables
    // (super-tile order); smaller vectors use the plain order.
    const uint32_t tb = (R == 8) ? (__ldg(&p.pass->dep[0][bt & 255u]) | __ldg(&p.pass->dep[1][(bt >> 8) & 255u]) |
                                    __ldg(&p.pass->dep[2][(bt >> 16) & 255u]))
                                 : bt * tile;
    const uint32_t base = tb + warp * 32u * R;
    Real ar[R], ai[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ar[r] = ai[r] = Real(0);
    for (int t = t0; t < ti; ++t) {
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
    for (int t = ti; t < t1; ++t) {  // coefficient i * c
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
      if (ACCUM) {
        const C prev = out[m];
        ar[r] += prev.x;
        ai[r] += prev.y;
      }
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

// ---------------------------------------------------------------------------
// TMA-staged matvec for vectors of at least one 2^kTileBits tile.
//
// A CTA (8 warps) owns a 2048-amplitude output tile at a time.  For a term
// with flip mask x the whole input tile T ^ (x & ~2047) is contiguous, so one
// elected thread moves it into shared memory with a single bulk copy
// (cp.async.bulk, completion counted on an mbarrier).  S stages keep S-1
// copies in flight ahead of the consumers, which read their permuted
// amplitudes from shared memory (x & 2047 permutes inside the tile; the XOR
// keeps each warp's 32 reads in 32 distinct 8-byte slots, conflict-free).
// One __syncthreads per term releases the stage that the next copy reuses.
// Every mbarrier wait is bounded (1 s of %globaltimer); a timeout records an
// error flag and the CTA drains and exits instead of spinning forever.
template <typename Real, int S>
struct TmaSmem {
  static constexpr uint32_t kTileAmps = 1u << kTileBits;
  static constexpr uint32_t kTileBytes = kTileAmps * 2 * sizeof(Real);
  static constexpr size_t kDynBytes = static_cast<size_t>(S) * kTileBytes;
};

template <typename Real, int EPI, bool ACCUM, int S>
__global__ void __launch_bounds__(256) k_matvec_tma(MV<Real> p, int* err_flag) {
  using C = typename CT<Real>::T;
  constexpr uint32_t kTileBytes = TmaSmem<Real, S>::kTileBytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ int s_err;
  if (EPI == EPI_LANCZOS && p.sc->m_eff <= p.j) return;
  if (EPI == EPI_RECUR && p.j + 1 >= p.sc->m_eff) return;
  const int t0 = p.pass->t0, ti = p.pass->ti, t1 = p.pass->t1;
  const int Tp = t1 - t0;
  const uint64_t soff = static_cast<uint64_t>(blockIdx.y) * p.D;
  const C* __restrict__ psi = p.psi + soff;
  C* __restrict__ out = p.out + soff;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t ntiles = static_cast<uint32_t>(p.D >> kTileBits);
  const uint32_t my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x - 1) / gridDim.x + 1 : 0;
  const uint64_t njobs = static_cast<uint64_t>(my_tiles) * static_cast<uint64_t>(Tp);
  const uint32_t smem0 = smem_u32(smem_raw);
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) mbar_init(smem_u32(&full_bar[i]), 1);
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();
  auto tile_base = [&](uint32_t k) -> uint32_t {
    const uint32_t bt = blockIdx.x + k * gridDim.x;
    return __ldg(&p.pass->dep[0][bt & 255u]) | __ldg(&p.pass->dep[1][(bt >> 8) & 255u]) |
           __ldg(&p.pass->dep[2][(bt >> 16) & 255u]);
  };
  // Job j = (tile k = j / Tp, term t0 + j % Tp) goes to stage j % S.
  auto issue = [&](uint64_t j) {
    const uint32_t k = static_cast<uint32_t>(j / Tp);
    const int tt = t0 + static_cast<int>(j % Tp);
    const uint32_t src = tile_base(k) ^ (__ldg(p.tv.x + tt) & ~((1u << kTileBits) - 1u));
    const uint32_t stg = static_cast<uint32_t>(j % S);
    const uint32_t bar = smem_u32(&full_bar[stg]);
    mbar_expect_tx(bar, kTileBytes);
    bulk_g2s(smem0 + stg * kTileBytes, psi + src, kTileBytes, bar);
  };
  uint64_t issued = 0;       // thread 0: jobs whose copy has been issued
  uint64_t first_fail = ~0ull;  // thread 0: first job it could not wait for
  if (threadIdx.x == 0)
    for (; issued + 1 < S && issued < njobs; ++issued) issue(issued);

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
  uint64_t j = 0;
  for (uint32_t k = 0; k < my_tiles; ++k) {
    const uint32_t base = tile_base(k) + warp * 256u;
    Real ar[8], ai[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) ar[r] = ai[r] = Real(0);
    for (int tt = t0; tt < t1; ++tt, ++j) {
      if (threadIdx.x == 0 && j + S - 1 < njobs && !s_err) {
        fence_proxy_async_smem();
        issue(j + S - 1);
        issued = j + S;
      }
      const uint32_t stg = static_cast<uint32_t>(j % S);
      const bool ok = mbar_wait_bounded(smem_u32(&full_bar[stg]), static_cast<uint32_t>((j / S) & 1), &s_err);
      if (!ok && threadIdx.x == 0 && first_fail == ~0ull) first_fail = j;
      if (ok) {
        const C* tile = reinterpret_cast<const C*>(smem_raw + stg * kTileBytes);
        const uint32_t x = __ldg(p.tv.x + tt), z = __ldg(p.tv.z + tt);
        const Real cl = sgnflip(__ldg(p.tv.coef + tt), __popc(z & lane) & 1u);
        const uint32_t off = lane ^ (x & 31u), xr = x & 0x7E0u;
        if (tt < ti) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const Real cc = sgnflip(cl, __popc(z & (base + 32u * r)) & 1u);
            const C v = tile[((warp * 256u + 32u * r) ^ xr) | off];
            ar[r] = fma_(cc, v.x, ar[r]);
            ai[r] = fma_(cc, v.y, ai[r]);
          }
        } else {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const Real cc = sgnflip(cl, __popc(z & (base + 32u * r)) & 1u);
            const C v = tile[((warp * 256u + 32u * r) ^ xr) | off];
            ar[r] = fma_(-cc, v.y, ar[r]);
            ai[r] = fma_(cc, v.x, ai[r]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t m = base + 32u * r + lane;
      if (ACCUM) {
        const C prev = out[m];
        ar[r] += prev.x;
        ai[r] += prev.y;
      }
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
  if (s_err && threadIdx.x == 0) {
    // Drain: wait (bounded) for every copy issued after the first job thread 0
    // could not wait for, so no bulk copy is still writing when the CTA exits.
    atomicExch(err_flag, 1);
    for (uint64_t q = first_fail; q < issued; ++q) {
      const uint32_t bar = smem_u32(&full_bar[q % S]);
      const uint64_t ts = globaltimer_ns();
      while (!mbar_try_wait(bar, static_cast<uint32_t>((q / S) & 1)) && globaltimer_ns() - ts < kWaitLimitNs) {
      }
    }
  }
}

// ---------------------------------------------------------------------------
// complex64 matvec, warp-specialised TMA pipeline (vectors of >= 2048 amplitudes).
//
// Warp kConsumerWarps is the producer: its lane 0 streams input tiles (one
// 16 KiB bulk copy per (tile, run) job) into S shared-memory stages, waiting
// on an "empty" mbarrier per stage before reusing it.  Warps 0..kConsumerWarps-1
// consume: each lane owns two neighbouring amplitudes in kRows rows of its
// warp's slice (m = tile + 64 kRows w + 64 r + 2 lane + {0, 1}), reads both
// inputs of a term with one 16-byte shared load, and signals the stage free
// with one arrive per warp.  Inside a pass the records are ordered by input
// tile (x >> 11), then class; consecutive terms with the same input tile (a
// run) share one staged copy.  A term's class (imag, x & 1, z & 1: the pair
// swap and the sign difference inside the pair) and its row permutation
// (x bits 6-8), precomputed in the record, select one of 64 compile-time
// bodies (c64_terms).
//
// Tile order.  The work items of a launch are (state, tile) pairs in the
// pass's super-tile order.  Passes that only store their sum (EPI_STORE) start
// each CTA at item blockIdx.x and then take items gridDim.x + p.sched[0]++
// from a device-wide counter, one claim prefetched per CTA (so a launch with
// no more items than CTAs does no extra work), so every CTA works within the
// same few super-tiles and the pass's inputs
// stay L2-resident for the whole launch; with a static round-robin split the
// CTAs drift apart by thousands of tiles over a long pass and evict each
// other's super-tiles.  The last CTA to finish returns the counter to zero
// (p.sched[1] counts finished CTAs), so launches that use one counter must
// not overlap on the GPU.  Passes with a Lanczos epilogue keep the static
// split: their per-CTA dot-product partials then cover a fixed set of tiles
// and the reduction is reproducible bit for bit.  The producer publishes each
// item in a small shared ring (s_item) before the stage barrier of the tile's
// first job completes, which orders it for the consumers; an item >= n_items
// ends the CTA's stream.  Every wait is bounded (1 s); on a timeout the CTA
// records the error, stops issuing, drains its copies and exits.
//
// SPLIT (EPI_STORE only; passes of a small block with many terms, one state):
// the items are (chunk, tile) pairs; item (c, tile) applies terms
// [t0 + c chunk_terms, ...) of the pass to the tile and writes its partial sum
// to p.out + c D (a workspace); chunk 0 also carries the earlier passes' sum
// (p.prev).  k_sum_chunks then adds the chunks in order, so the result does not
// depend on which CTA ran which chunk.
template <int EPI, bool ACCUM, int S, bool SPLIT = false, bool MERGE = false>
__global__ void __launch_bounds__(32 * (kConsumerWarps + 1), c64_ctas_for_stages(S))
    k_matvec_c64(MV<float> p, int* err_flag) {
  static_assert(!SPLIT || EPI == EPI_STORE, "split passes only store their sum");
  constexpr uint32_t kTileBytes = (1u << kTileBits) * 8u;
  constexpr bool kQueue = EPI == EPI_STORE;
  constexpr int kRing = 8;  // items in flight between producer and consumers: at most S + 1
  static_assert(kRing > S + 1, "item ring too small for the stage count");
  constexpr uint64_t kEnd = ~0ull;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ uint64_t s_item[kRing];
  __shared__ int s_err;
  if (EPI == EPI_LANCZOS && p.sc->m_eff <= p.j) return;
  if (EPI == EPI_RECUR && p.j + 1 >= p.sc->m_eff) return;
  int cls[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) cls[c] = p.pass->cls[c];
  const int t0 = cls[0], t1 = cls[8];
  const int Tp = t1 - t0;
  const bool feed = Tp > 0 || ACCUM;  // the producer has jobs (else the sum is zero)
  const bool queue = kQueue && feed;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t ntiles = static_cast<uint32_t>(p.D >> kTileBits);  // a power of two
  const uint32_t tshift = 31u - static_cast<uint32_t>(__clz(ntiles));
  // EPI_STORE launches are one-dimensional over p.ny states; the others use blockIdx.y.
  const uint64_t n_items = kQueue ? (static_cast<uint64_t>(p.ny) << tshift) : ntiles;
  const uint64_t ybase = kQueue ? 0ull : blockIdx.y;
  auto static_item = [&](uint64_t k) -> uint64_t {
    const uint64_t it = blockIdx.x + k * gridDim.x;
    return it < n_items ? it : kEnd;
  };
  auto tile_base = [&](uint64_t item) -> uint32_t {
    const uint32_t bt = static_cast<uint32_t>(item) & (ntiles - 1u);
    return __ldg(&p.pass->dep[0][bt & 255u]) | __ldg(&p.pass->dep[1][(bt >> 8) & 255u]) |
           __ldg(&p.pass->dep[2][(bt >> 16) & 255u]);
  };
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
    // ---------------- producer ----------------
    if (lane == 0 && feed) {
      const uint32_t smem0 = smem_u32(smem_raw);
      const uint64_t keep = l2_policy_evict_last();   // input tiles: re-read by the pass's other terms
      const uint64_t stream = l2_policy_evict_first();  // the output tile: read once per pass
      uint64_t q = 0, issued = 0;
      uint64_t next = static_item(0);  // the first item is blockIdx.x in both orders
      // Job stream per tile: [the tile of `out` (ACCUM only)] then one input tile per run.
      for (uint64_t k = 0; !*(volatile int*)&s_err; ++k) {
        const uint64_t item = next < n_items ? next : kEnd;
        if (item != kEnd) next = queue ? gridDim.x + atomicAdd(p.sched, 1ull) : static_item(k + 1);
        if (item == kEnd) {  // end marker: an arrive without bytes on the next stage
          const uint32_t stg = static_cast<uint32_t>(q % S);
          if (q >= S && !mbar_wait_bounded(smem_u32(&empty_bar[stg]), static_cast<uint32_t>(((q / S) - 1) & 1),
                                           &s_err))
            break;
          s_item[k % kRing] = kEnd;
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[stg])) : "memory");
          break;
        }
        const uint64_t hi = item >> tshift;  // state, or chunk when SPLIT
        const uint64_t soff = SPLIT ? 0ull : (ybase + hi) * p.D;
        const int ct0 = SPLIT ? t0 + static_cast<int>(hi) * p.chunk_terms : t0;
        const int ct1 = SPLIT ? min(t1, ct0 + p.chunk_terms) : t1;
        const bool acc_i = ACCUM && (!SPLIT || hi == 0);
        const uint32_t tb = tile_base(item);
        for (int tt = acc_i ? ct0 - 1 : ct0; tt < ct1 && !*(volatile int*)&s_err; ++tt) {
          const bool phi = acc_i && tt < ct0;
          const uint2 xf = phi ? make_uint2(0u, 0u) : make_uint2(__ldg(&p.rec[tt].x), __ldg(&p.rec[tt].flags));
          if (!phi && !(xf.y & kTermRunStart) && !(SPLIT && tt == ct0)) continue;  // the run's tile is staged
          const uint32_t stg = static_cast<uint32_t>(q % S);
          if (q >= S && !mbar_wait_bounded(smem_u32(&empty_bar[stg]), static_cast<uint32_t>(((q / S) - 1) & 1),
                                           &s_err))
            break;
          if (tt == (acc_i ? ct0 - 1 : ct0)) s_item[k % kRing] = item;
          const float2* src = phi ? (SPLIT ? p.prev : p.out) + soff + tb
                                  : p.psi + soff + (tb ^ (xf.x & kTermXMask & ~((1u << kTileBits) - 1u)));
          const uint32_t bar = smem_u32(&full_bar[stg]);
          mbar_expect_tx(bar, kTileBytes);
          bulk_g2s_hint(smem0 + stg * kTileBytes, src, kTileBytes, bar, (phi || (xf.y & kTermStraggler)) ? stream : keep);
          issued = ++q;
        }
      }
      if (s_err) {  // drain: the last copy issued into each stage must land before exit
        for (uint64_t qq = issued > S ? issued - S : 0; qq < issued; ++qq) {
          const uint32_t bar = smem_u32(&full_bar[qq % S]);
          const uint64_t ts = globaltimer_ns();
          while (!mbar_try_wait(bar, static_cast<uint32_t>((qq / S) & 1)) && globaltimer_ns() - ts < kWaitLimitNs) {
          }
        }
      }
      if (queue) {  // this CTA claims no more items; the last one to get here resets the counter
        __threadfence();
        if (atomicAdd(p.sched + 1, 1ull) == gridDim.x - 1ull) {
          __threadfence();
          atomicExch(p.sched, 0ull);
          atomicExch(p.sched + 1, 0ull);
        }
      }
    }
  } else {
    // ---------------- consumers ----------------
    float bprev = 0.f, alpha = 0.f, rbeta = 0.f;
    float2 cy = {0.f, 0.f};
    if (EPI != EPI_STORE && p.j > 0) bprev = static_cast<float>(p.sc->beta[p.j - 1]);
    if (EPI == EPI_RECUR) {
      alpha = static_cast<float>(p.sc->alpha[p.j]);
      rbeta = static_cast<float>(1.0 / p.sc->beta[p.j]);
      cy.x = static_cast<float>(p.sc->beta0 * p.sc->c_re[p.j + 1]);
      cy.y = static_cast<float>(p.sc->beta0 * p.sc->c_im[p.j + 1]);
    }
    const uint32_t pair_part = warp * (64u * kRows) + 2u * lane;
    const uint64_t out_pol = l2_policy_evict_first();  // output tiles are not re-read within the pass
    StageRing<S> ring;
    uint4 d = make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t k = 0;; ++k) {
      uint64_t item;
      if (feed) {  // the item rides with the tile's first job
        if (!mbar_wait_bounded(smem_u32(&full_bar[ring.stg]), ring.ph, &s_err)) break;
        item = *reinterpret_cast<volatile uint64_t*>(&s_item[k % kRing]);
      } else {
        item = static_item(k);
      }
      if (item >= n_items) break;
      const uint64_t hi = item >> tshift;  // state, or chunk when SPLIT
      const uint64_t soff = (ybase + hi) * p.D;
      const int ct0 = SPLIT ? t0 + static_cast<int>(hi) * p.chunk_terms : t0;
      const int ct1 = SPLIT ? min(t1, ct0 + p.chunk_terms) : t1;
      const bool acc_i = ACCUM && (!SPLIT || hi == 0);
      const float4* psi4 = reinterpret_cast<const float4*>(p.psi + (SPLIT ? 0ull : soff));
      float4* out4 = reinterpret_cast<float4*>(p.out + soff);
      const uint32_t mt = tile_base(item) + pair_part;  // amplitude of row 0, even
      if (Tp > 0) d = __ldg(reinterpret_cast<const uint4*>(p.rec + ct0));  // the tile's first term
      // The sum starts from the partial sum of the earlier passes (ACCUM: the
      // producer's first job of the tile is this tile of `out`), else from 0.
      float a[kRows][4];
      if (acc_i) {
        const uint32_t stg = ring.stg;
        const bool ok = mbar_wait_bounded(smem_u32(&full_bar[stg]), ring.ph, &s_err);
        const float4* t4 = reinterpret_cast<const float4*>(smem_raw + stg * kTileBytes);
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          const float4 pv = ok ? t4[(pair_part >> 1) + 32u * r] : make_float4(0.f, 0.f, 0.f, 0.f);
          a[r][0] = pv.x;
          a[r][1] = pv.y;
          a[r][2] = pv.z;
          a[r][3] = pv.w;
        }
        __syncwarp();
        if (lane == 0 && ok)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[stg])) : "memory");
        ring.next();
      } else {
#pragma unroll
        for (int r = 0; r < kRows; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = 0.f;
      }
      c64_terms<S, SPLIT, MERGE>(ct0, ct1, d, ring, a, p.rec, mt, pair_part, smem_raw, full_bar, empty_bar, &s_err,
                                 lane);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const uint32_t i4 = (mt >> 1) + 32u * r;
        if (EPI == EPI_STORE) {
          st_f4_hint(out4 + i4, make_float4(a[r][0], a[r][1], a[r][2], a[r][3]), out_pol);
        } else {
          float4 vp = make_float4(0.f, 0.f, 0.f, 0.f);
          if (p.j > 0) vp = reinterpret_cast<const float4*>(p.vprev + soff)[i4];
          const float2 w0 = lanczos_w1<float, float2>(a[r][0], a[r][1], bprev, make_float2(vp.x, vp.y));
          const float2 w1 = lanczos_w1<float, float2>(a[r][2], a[r][3], bprev, make_float2(vp.z, vp.w));
          const float4 v = psi4[i4];
          if (EPI == EPI_LANCZOS) {
            out4[i4] = make_float4(w0.x, w0.y, w1.x, w1.y);
            part += static_cast<double>(v.x * w0.x + v.y * w0.y) + static_cast<double>(v.z * w1.x + v.w * w1.y);
          } else {
            float4 vn;
            vn.x = mul_(fma_(-alpha, v.x, w0.x), rbeta);
            vn.y = mul_(fma_(-alpha, v.y, w0.y), rbeta);
            vn.z = mul_(fma_(-alpha, v.z, w1.x), rbeta);
            vn.w = mul_(fma_(-alpha, v.w, w1.y), rbeta);
            out4[i4] = vn;
            float4* y4 = reinterpret_cast<float4*>(p.y + soff);
            float4 yy = y4[i4];
            yy.x = fma_(cy.x, vn.x, fma_(-cy.y, vn.y, yy.x));
            yy.y = fma_(cy.x, vn.y, fma_(cy.y, vn.x, yy.y));
            yy.z = fma_(cy.x, vn.z, fma_(-cy.y, vn.w, yy.z));
            yy.w = fma_(cy.x, vn.w, fma_(cy.y, vn.z, yy.w));
            y4[i4] = yy;
          }
        }
      }
    }
  }
  if (EPI == EPI_LANCZOS) {
    part = block_sum(part);
    if (threadIdx.x == 0) p.partial[blockIdx.y * gridDim.x + blockIdx.x] = part;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_err) atomicExch(err_flag, 1);
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
  const int t0 = p.pass->t0, ti = p.pass->ti, t1 = p.pass->t1;
  if (m < p.D) {
    Real ar = 0, ai = 0;
    for (int t = t0; t < t1; ++t) {
      const uint32_t x = p.tv.x[t], z = p.tv.z[t];
      const Real cc = sgnflip(p.tv.coef[t], __popc(z & m) & 1u);
      const C v = psi[m ^ x];
      if (t < ti) {
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
  return v;
}

struct Shape {
  int R, warps, grid;  // R == 8: TMA-staged 2048-amplitude tiles
};

constexpr int kStagesD = 3;  // complex128 k_matvec_tma: 3 x 32 KiB in flight per CTA

// complex128 blocks of fewer tiles than this take the amplitude-parallel
// gather kernel: the TMA kernel runs one CTA per tile, so a small block would
// leave most SMs idle (B300, OTOC curves of the paper's benchmark rows: N=30,
// k=3 639 -> 260 ms; dense N=30 126 -> 15 s; N=40 1.41 -> 1.30 s).
constexpr uint64_t kC128GatherTiles = 512;

Shape shape_of(const syk_terms* h) {
  Shape s;
  const uint64_t D = static_cast<uint64_t>(h->D);
  if (D < 32) return {0, 1, 1};
  const uint64_t ntiles_cap = static_cast<uint64_t>(h->n_sm);
  const bool c128_gather = h->dtype == SYK_C128 && (D >> kTileBits) < kC128GatherTiles;
  if (D >= (1ull << kTileBits) && !c128_gather) {
    s.R = 8;
    s.warps = 8;
    // CTAs resident per SM given the stage buffers (complex64: the shape of the
    // passes with a Lanczos epilogue, the only ones launched on this grid)
    const uint64_t per_sm = h->dtype == SYK_C128 ? 2 : static_cast<uint64_t>(kC64EpiCtasPerSm);
    s.grid = static_cast<int>(std::min<uint64_t>(D >> kTileBits, ntiles_cap * per_sm));
    return s;
  }
  s.R = 1;
  s.warps = static_cast<int>(std::min<uint64_t>(8, D / 32));
  const uint64_t ntiles = D / (32ull * s.R * s.warps);
  s.grid = static_cast<int>(std::min<uint64_t>(ntiles, ntiles_cap * 8));
  return s;
}

// One complex64 pass on the TMA-staged kernel of the handle's shape.
template <int EPI, bool ACCUM, bool MERGE, int S>
void launch_c64_pass(const syk_terms* h, const Shape& s, const MV<float>& q, unsigned gy, cudaStream_t st) {
  constexpr size_t dyn = static_cast<size_t>(S) * (1u << kTileBits) * 8u;
  static std::atomic<uint64_t> configured{0};
  const uint64_t bit = 1ull << (h->device & 63);
  if (!(configured.load() & bit)) {
    SYK_CUDA(cudaFuncSetAttribute(k_matvec_c64<EPI, ACCUM, S, false, MERGE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn)));
    configured.fetch_or(bit);
  }
  if (EPI == EPI_STORE) {  // one-dimensional over (state, tile) items taken from the handle's counter
    MV<float> qq = q;
    qq.sched = h->d_sched;
    qq.ny = gy;
    const uint64_t items = (static_cast<uint64_t>(h->D) >> kTileBits) * gy;
    const uint64_t ctas = static_cast<uint64_t>(h->n_sm) * c64_ctas_for_stages(S);
    const unsigned grid = static_cast<unsigned>(std::min<uint64_t>(items, ctas));
    k_matvec_c64<EPI, ACCUM, S, false, MERGE><<<grid, 32 * (kConsumerWarps + 1), dyn, st>>>(qq, h->d_err);
  } else {
    k_matvec_c64<EPI, ACCUM, S, false, MERGE><<<dim3(s.grid, gy), 32 * (kConsumerWarps + 1), dyn, st>>>(q, h->d_err);
  }
}

template <typename Real, int EPI, bool ACCUM>
void launch_pass(const syk_terms* h, const Shape& s, const MV<Real>& q, unsigned gy, cudaStream_t st) {
  if constexpr (std::is_same<Real, float>::value) {
    if (s.R == 8) {
      // epilogue passes always take the 3-stage shape (at 72 registers their epilogues spill)
      if (h->c64_merge()) {
        launch_c64_pass<EPI, ACCUM, true, kStagesC64Epi>(h, s, q, gy, st);
      } else if constexpr (EPI != EPI_STORE) {
        launch_c64_pass<EPI, ACCUM, false, kStagesC64Epi>(h, s, q, gy, st);
      } else {
        if (h->c64_wide())
          launch_c64_pass<EPI, ACCUM, false, kStagesC64Epi>(h, s, q, gy, st);
        else
          launch_c64_pass<EPI, ACCUM, false, kStagesC64>(h, s, q, gy, st);
      }
      return;
    }
  }
  if (s.R == 8) {
    if constexpr (std::is_same<Real, double>::value) {  // complex64 took k_matvec_c64 above
      constexpr int S = kStagesD;
      constexpr size_t dyn = TmaSmem<Real, S>::kDynBytes;
      static std::atomic<uint64_t> configured{0};  // one bit per device ordinal (< 64)
      const uint64_t bit = 1ull << (h->device & 63);
      if (!(configured.load() & bit)) {
        SYK_CUDA(cudaFuncSetAttribute(k_matvec_tma<Real, EPI, ACCUM, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(dyn)));
        configured.fetch_or(bit);
      }
      k_matvec_tma<Real, EPI, ACCUM, S><<<dim3(s.grid, gy), 256, dyn, st>>>(q, h->d_err);
    }
  } else {
    k_matvec<Real, 1, EPI, ACCUM><<<dim3(s.grid, gy), 32 * s.warps, 0, st>>>(q);
  }
}

// out = sum over chunks c = 0..C-1 of ws[c] (in that order), float4 at a time.
__global__ void k_sum_chunks(const float4* __restrict__ ws, int C, uint64_t n4, float4* __restrict__ out) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    float4 a = ws[i];
    for (int c = 1; c < C; ++c) {
      const float4 v = ws[static_cast<uint64_t>(c) * n4 + i];
      a.x += v.x;
      a.y += v.y;
      a.z += v.z;
      a.w += v.w;
    }
    out[i] = a;
  }
}

// A split complex64 pass: chunks of terms on different CTAs into the
// workspace, then their sum into q.out (which, for passes after the first,
// chunk 0 started from).
template <bool ACCUM, bool MERGE, int S>
void launch_split_chunks(const syk_terms* h, int ip, const MV<float>& q, cudaStream_t st) {
  constexpr size_t dyn = static_cast<size_t>(S) * (1u << kTileBits) * 8u;
  static std::atomic<uint64_t> configured{0};
  const uint64_t bit = 1ull << (h->device & 63);
  if (!(configured.load() & bit)) {
    SYK_CUDA(cudaFuncSetAttribute(k_matvec_c64<EPI_STORE, ACCUM, S, true, MERGE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn)));
    configured.fetch_or(bit);
  }
  const int C = h->split_chunks[ip];
  MV<float> qs = q;
  qs.out = h->d_split_ws;
  qs.prev = q.out;
  qs.ny = static_cast<uint32_t>(C);
  qs.chunk_terms = h->split_terms[ip];
  qs.sched = h->d_sched;
  const uint64_t items = (static_cast<uint64_t>(h->D) >> kTileBits) * C;
  const uint64_t ctas = static_cast<uint64_t>(h->n_sm) * c64_ctas_for_stages(S);
  const unsigned grid = static_cast<unsigned>(std::min<uint64_t>(items, ctas));
  k_matvec_c64<EPI_STORE, ACCUM, S, true, MERGE><<<grid, 32 * (kConsumerWarps + 1), dyn, st>>>(qs, h->d_err);
}

template <bool ACCUM>
void launch_split_pass(const syk_terms* h, int ip, const MV<float>& q, cudaStream_t st) {
  if (h->c64_merge())
    launch_split_chunks<ACCUM, true, kStagesC64Epi>(h, ip, q, st);
  else if (h->c64_wide())
    launch_split_chunks<ACCUM, false, kStagesC64Epi>(h, ip, q, st);
  else
    launch_split_chunks<ACCUM, false, kStagesC64>(h, ip, q, st);
  const int C = h->split_chunks[ip];
  const uint64_t n4 = static_cast<uint64_t>(h->D) / 2;
  const unsigned g2 = static_cast<unsigned>(std::min<uint64_t>((n4 + 255) / 256, static_cast<uint64_t>(h->n_sm) * 8));
  k_sum_chunks<<<g2, 256, 0, st>>>(reinterpret_cast<const float4*>(h->d_split_ws), C, n4,
                                   reinterpret_cast<float4*>(q.out));
}

// One launch per pass: passes before the last write (first) or accumulate
// plain partial sums; the last pass applies the requested epilogue.  A split
// complex64 pass (plan_split) stores its sum like the others; when it is the
// last pass, the epilogue then runs as an accumulating pass with no terms.
template <typename Real, int EPI>
void run_matvec(const syk_terms* h, const MV<Real>& p, int64_t nstates, cudaStream_t st) {
  const Shape s = shape_of(h);
  const int np = static_cast<int>(h->passes.size());
  for (int64_t s0 = 0; s0 < nstates; s0 += 65535) {
    MV<Real> q = p;
    const uint64_t off = static_cast<uint64_t>(s0) * h->D;
    q.psi += off;
    q.out += off;
    const unsigned gy = static_cast<unsigned>(std::min<int64_t>(65535, nstates - s0));
    if (s.R == 0) {  // single pass
      q.pass = h->d_passes;
      k_matvec_tiny<Real, EPI><<<dim3(1, gy), 32, 0, st>>>(q);
      continue;
    }
    for (int ip = 0; ip < np; ++ip) {
      q.pass = h->d_passes + ip;
      const bool last = ip == np - 1, accum = ip > 0;
      if constexpr (std::is_same<Real, float>::value) {
        if (s.R == 8 && gy == 1 && h->split_chunks[ip] > 1) {
          accum ? launch_split_pass<true>(h, ip, q, st) : launch_split_pass<false>(h, ip, q, st);
          if (last && EPI != EPI_STORE) {
            q.pass = h->d_pass_tail;
            launch_pass<Real, EPI, true>(h, s, q, gy, st);
          }
          continue;
        }
      }
      if (!last)
        accum ? launch_pass<Real, EPI_STORE, true>(h, s, q, gy, st)
              : launch_pass<Real, EPI_STORE, false>(h, s, q, gy, st);
      else
        accum ? launch_pass<Real, EPI, true>(h, s, q, gy, st) : launch_pass<Real, EPI, false>(h, s, q, gy, st);
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

// Split a complex64 pass into chunks of terms when its block has too few tiles
// to fill the GPU and the pass has many terms (dense SYK, small N with large
// k): chunks x tiles ~ the resident CTAs, at least 32 terms a chunk.  The
// workspace holds one partial sum per chunk: at most (CTAs + tiles) tiles.
void plan_split(syk_terms* h) {
  const size_t np = h->passes.size();
  h->split_chunks.assign(np, 1);
  h->split_terms.assign(np, 0);
  h->split_ws_bytes = 0;
  if (h->dtype != SYK_C64 || h->D < (int64_t(1) << kTileBits)) return;
  const int64_t ntiles = h->D >> kTileBits;
  const int64_t cap = static_cast<int64_t>(h->n_sm) * (h->c64_wide() ? kC64EpiCtasPerSm : kC64CtasPerSm);
  if (2 * ntiles > cap) return;
  int64_t cmax = 1;
  for (size_t p = 0; p < np; ++p) {
    const int64_t Tp = h->passes[p].t1 - h->passes[p].t0;
    int64_t C = std::min<int64_t>((cap + ntiles - 1) / ntiles, Tp / 32);
    if (C < 2) continue;
    const int64_t Tc = (Tp + C - 1) / C;
    C = (Tp + Tc - 1) / Tc;  // every chunk non-empty
    h->split_chunks[p] = static_cast<int>(C);
    h->split_terms[p] = static_cast<int>(Tc);
    cmax = std::max(cmax, C);
  }
  if (cmax > 1) h->split_ws_bytes = static_cast<size_t>(cmax) * static_cast<size_t>(h->D) * 8u;
}

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
    p.rec = h->d_termf[block];
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
    p.rec = h->d_termf[block];
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
    p.rec = h->d_termf[block];
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
