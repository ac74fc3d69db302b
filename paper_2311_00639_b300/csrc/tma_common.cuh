// Bulk-copy (TMA) pipeline helpers and the complex64 pair-layout consumer,
// shared by the single-Hamiltonian matvec (apply.cu) and the batched engine
// (batch.cu).
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace syk {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the thread may sleep in hardware until
// the phase completes or about `ns` nanoseconds pass, instead of spinning.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// L2 eviction-priority policies (createpolicy) for bulk copies and stores.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void st_f4_hint(float4* ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per wait

// Bounded wait; returns false (and sets *s_err) on timeout or if another
// thread already recorded an error.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int* s_err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t_start = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;  // sleep up to 0.1 ms per try
    if (*s_err) return false;
    if (globaltimer_ns() - t_start > kWaitLimitNs) {
      *s_err = 1;
      return false;
    }
  }
}

// Consumer layout: each lane owns two neighbouring amplitudes in kRows rows of
// 64 amplitudes (m = tile + warp*64*kRows + 64 r + 2 lane + {0,1}); the warps of
// a CTA tile the 2048-amplitude tile.
#ifndef SYK_C64_ROWS
#define SYK_C64_ROWS 8
#endif
constexpr int kRows = SYK_C64_ROWS;
constexpr int kConsumerWarps = (1 << kTileBits) / (64 * kRows);
constexpr uint32_t kRowMask = static_cast<uint32_t>(kRows - 1) << 6;  // amplitude bits chosen by the row
constexpr uint32_t kPairXMask = 0x7FEu & ~kRowMask;                    // in-tile flip bits applied per lane
// Pipeline shape of the passes that only store their sum (the H psi passes
// and every pass but the last of a Lanczos matvec): 2 stages x 5 CTAs per SM
// (72 registers a thread).  The consumers, not the staging depth, bound these
// passes, so more consumer warps per SM beat deeper staging.  Measured on B300,
// N=64 H psi: 2 x 5 180.6 ms, 3 x 4 185.8, 2 x 4 192.8, 3 x 3 217.9;
// N=56: 8.85 / 9.25 ms for 2 x 5 / 3 x 4.
#ifndef SYK_C64_STAGES
#define SYK_C64_STAGES 2
#endif
constexpr int kStagesC64 = SYK_C64_STAGES;
#ifndef SYK_C64_MAX_CTAS
#define SYK_C64_MAX_CTAS 5
#endif
// CTAs per SM: shared memory holds S 16 KiB stages each (<= 227 KiB per SM),
// at most SYK_C64_MAX_CTAS (the register budget of __launch_bounds__).
constexpr int kC64CtasPerSm = (227 / (16 * kStagesC64 + 2)) < SYK_C64_MAX_CTAS ? (227 / (16 * kStagesC64 + 2))
                                                                               : SYK_C64_MAX_CTAS;
// Passes with a Lanczos epilogue (EPI_LANCZOS, EPI_RECUR) hold the epilogue's
// operands beside the row sums: 3 stages x 4 CTAs per SM, 96 registers a
// thread (at 72 their epilogues spill).
constexpr int kStagesC64Epi = 3;
constexpr int kC64EpiCtasPerSm = 4;
// The stage count of a complex64 matvec kernel fixes its shape: 2 stages run
// 5 CTAs per SM (72 registers a thread), 3 stages 4 CTAs (96 registers).
constexpr int c64_ctas_for_stages(int S) { return S == kStagesC64 ? kC64CtasPerSm : kC64EpiCtasPerSm; }

template <bool IMAG, bool XS, bool ZS, int XR>
__device__ __forceinline__ void c64_rows(const float4* __restrict__ t4, uint32_t pa2, const float (&c)[kRows],
                                         float (&a)[kRows][4]) {
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const float4 v = t4[pa2 + 32u * static_cast<uint32_t>(r ^ XR)];
    // inputs of amplitude m (even) and m + 1
    const float i0r = XS ? v.z : v.x, i0i = XS ? v.w : v.y;
    const float i1r = XS ? v.x : v.z, i1i = XS ? v.y : v.w;
    const float c0 = c[r];
    const float c1 = ZS ? -c[r] : c[r];
    if (!IMAG) {
      a[r][0] = fma_(c0, i0r, a[r][0]);
      a[r][1] = fma_(c0, i0i, a[r][1]);
      a[r][2] = fma_(c1, i1r, a[r][2]);
      a[r][3] = fma_(c1, i1i, a[r][3]);
    } else {  // (i c) * v = c * (-v.im, v.re)
      a[r][0] = fma_(-c0, i0i, a[r][0]);
      a[r][1] = fma_(c0, i0r, a[r][1]);
      a[r][2] = fma_(-c1, i1i, a[r][2]);
      a[r][3] = fma_(c1, i1r, a[r][3]);
    }
  }
}

// A consumer's position in the stage ring: the stage of its next job and the
// mbarrier phase parity that job completes.
template <int S>
struct StageRing {
  uint32_t stg = 0, ph = 0;
  __device__ __forceinline__ void next() {
    if (++stg == static_cast<uint32_t>(S)) {
      stg = 0;
      ph ^= 1u;
    }
  }
};

// Apply terms [tb0, tb1) of the current tile.  Consecutive terms with the
// same input tile (a run, see TermF) read one stage: the warp waits for the
// stage at the run's first term and releases it after the run's last.  `d`
// holds the record of term tb0 on entry; each iteration loads the next one
// (the record array has one spare entry past the last term) so that its
// latency overlaps the current term.  The term's body index (flags bits
// 8-13: class imag, x & 1, z & 1 and row permutation x bits 6-8) selects one
// of 64 compile-time bodies.  Consecutive terms with the same x and class (a
// merge group, kTermMerge) read the same staged inputs through the same body:
// their signed row coefficients are summed and the body runs once (8 adds per
// merged term instead of 8 loads and 32 FMAs).  A group's first record holds
// the group's length (flags bits 16-23): the consumer sums the rest of the
// group in a tight loop; a chunk of a split pass that starts inside a group
// keeps running sums record by record (dsum) up to the group's last record.
// MERGE = false ignores the flag and applies every term on its own (the same
// sum, in another rounding order): the kernels of Hamiltonians whose records
// merge nothing, where the running sums would only cost registers.
#define SYK_C64_BODY(k)                                                                                          \
  case k:                                                                                                        \
    c64_rows<((k) >> 5) & 1, ((k) >> 4) & 1, ((k) >> 3) & 1, ((k) & 7) % kRows>(t4, pa2, c, a);                 \
    break;
#define SYK_C64_BODY8(k) \
  SYK_C64_BODY(k) SYK_C64_BODY(k + 1) SYK_C64_BODY(k + 2) SYK_C64_BODY(k + 3) SYK_C64_BODY(k + 4) \
  SYK_C64_BODY(k + 5) SYK_C64_BODY(k + 6) SYK_C64_BODY(k + 7)
// FORCE: [tb0, tb1) is a chunk of a pass whose ends need not be run ends; the
// chunk's first term starts a run and its last ends one.
template <int S, bool FORCE = false, bool MERGE = false>
__device__ __forceinline__ void c64_terms(int tb0, int tb1, uint4& d, StageRing<S>& ring, float (&a)[kRows][4],
                                          const TermF* __restrict__ rec, uint32_t mt, uint32_t pair_part,
                                          const unsigned char* smem, uint64_t* full_bar, uint64_t* empty_bar,
                                          volatile int* s_err, uint32_t lane) {
  static_assert(kRows == 8, "the row permutation switch covers x bits 6-8");
  bool ok = false;
  bool pending = false;  // dsum holds the coefficients of earlier terms of a merge group
  float dsum[kRows] = {};
  const float4* t4 = reinterpret_cast<const float4*>(smem);
  for (int tt = tb0; tt < tb1; ++tt) {
    const uint4 cur = d;
    d = __ldg(reinterpret_cast<const uint4*>(rec + tt + 1));
    const uint32_t x = cur.x, z = cur.y, cb = cur.z;
    uint32_t fl = cur.w;
    if (FORCE) {
      fl |= (tt == tb0 ? kTermRunStart : 0u) | (tt == tb1 - 1 ? kTermRunEnd : 0u);
      if (tt == tb1 - 1) fl &= ~kTermMerge;  // a chunk's last term closes its group
    }
    if (fl & kTermRunStart) {
      ok = mbar_wait_bounded(smem_u32(&full_bar[ring.stg]), ring.ph, s_err);
      t4 = reinterpret_cast<const float4*>(smem + ring.stg * (1u << kTileBits) * 8u);
    }
    if (ok) {
      // sign (-1)^{popc(z & m)} of row r: the lane/warp/tile part popc(z & mt)
      // and the row part popc(z & 64 r) = parity of (z >> 6) & r, folded into
      // the coefficient's sign bit.  z's bits 6, 7, 8 sit in bit 31 of fl, x
      // and z (TermF); mt < 2^31, so bit 31 of z does not reach the popc.
      constexpr uint32_t M = 0x80000000u;
      const uint32_t s0 = (__popc(z & mt) << 31) ^ cb;
      float c[kRows];
      {
        const uint32_t c1 = s0 ^ (fl & M), c2 = s0 ^ (x & M), c3 = c1 ^ (x & M);
        c[0] = __uint_as_float(s0);
        c[1] = __uint_as_float(c1);
        c[2] = __uint_as_float(c2);
        c[3] = __uint_as_float(c3);
        c[4] = __uint_as_float(s0 ^ (z & M));
        c[5] = __uint_as_float(c1 ^ (z & M));
        c[6] = __uint_as_float(c2 ^ (z & M));
        c[7] = __uint_as_float(c3 ^ (z & M));
      }
      bool apply = true;
      if (MERGE) {
        const uint32_t glen = (fl >> kTermGroupShift) & kTermGroupMax;
        if (glen != 0) {
          // a merge group's first record: sum the coefficients of the rest
          // of the group (inside this chunk) in one loop, then run the body
          int n = static_cast<int>(glen);
          if (FORCE) n = min(n, tb1 - 1 - tt);
          // records two ahead: d holds record tt + j, e record tt + j + 1
          // (never past tb1 <= the pass end, which the record array covers)
          uint4 e = __ldg(reinterpret_cast<const uint4*>(rec + min(tt + 2, tb1)));
          for (int j = 1; j <= n; ++j) {
            const uint4 nx = d;
            d = e;
            e = __ldg(reinterpret_cast<const uint4*>(rec + min(tt + j + 2, tb1)));
            const uint32_t t0 = (__popc(nx.y & mt) << 31) ^ nx.z;
            const uint32_t t1 = t0 ^ (nx.w & M), t2 = t0 ^ (nx.x & M), t3 = t1 ^ (nx.x & M);
            c[0] += __uint_as_float(t0);
            c[1] += __uint_as_float(t1);
            c[2] += __uint_as_float(t2);
            c[3] += __uint_as_float(t3);
            c[4] += __uint_as_float(t0 ^ (nx.y & M));
            c[5] += __uint_as_float(t1 ^ (nx.y & M));
            c[6] += __uint_as_float(t2 ^ (nx.y & M));
            c[7] += __uint_as_float(t3 ^ (nx.y & M));
            fl = (fl & ~kTermRunEnd) | (nx.w & kTermRunEnd);  // the run may end at the group's last record
          }
          tt += n;
          if (FORCE && tt == tb1 - 1) fl |= kTermRunEnd;
        } else if (fl & kTermMerge) {
          // inside a group that began before this chunk: running sums
          if (pending) {
#pragma unroll
            for (int r = 0; r < kRows; ++r) dsum[r] += c[r];
          } else {
#pragma unroll
            for (int r = 0; r < kRows; ++r) dsum[r] = c[r];
            pending = true;
          }
          apply = false;
        } else if (pending) {  // that group's last record
#pragma unroll
          for (int r = 0; r < kRows; ++r) c[r] += dsum[r];
          pending = false;
        }
      }
      if (apply) {
        const uint32_t pa2 = (pair_part ^ (x & kPairXMask)) >> 1;  // float4 index of the row-0 input pair
        switch ((fl >> kTermBodyShift) & 63u) {
          SYK_C64_BODY8(0)
          SYK_C64_BODY8(8)
          SYK_C64_BODY8(16)
          SYK_C64_BODY8(24)
          SYK_C64_BODY8(32)
          SYK_C64_BODY8(40)
          SYK_C64_BODY8(48)
          SYK_C64_BODY8(56)
          default: break;
        }
      }
    }
    if (fl & kTermRunEnd) {
      __syncwarp();
      if (lane == 0 && ok) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[ring.stg])) : "memory");
      ring.next();
    }
  }
}
#undef SYK_C64_BODY8
#undef SYK_C64_BODY

}  // namespace
}  // namespace syk
