// Hardware probes for the roofline denominators the benchmark reports (the
// paper has no counterpart; nothing on the hot path calls them):
//   * syk_probe_staging — the rate at which 16 KiB bulk copies (cp.async.bulk
//     + mbarrier, one producer lane and 4 consumer warps per CTA, the stages
//     and CTAs per SM of the complex64 matvec's store passes) move an L2-resident
//     buffer into shared memory, with the consumers reading every staged tile
//     0, 1 or 2 times; or, for comparison, the rate of plain 16-byte global
//     loads of the same tiles (no shared memory);
//   * syk_probe_smem — the rate of 16-byte shared-memory loads of the whole GPU
//     in the complex64 matvec consumers' pattern (a warp reads 512 contiguous
//     bytes per load, no bank conflicts), with nothing else running;
//   * syk_probe_fp64 — the FP64 fused multiply-add rate of the whole GPU
//     (independent chains, all SMs).
// Every wait is bounded as in the matvec pipelines.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "tma_common.cuh"

namespace syk {
namespace {

constexpr uint32_t kProbeTileBytes = 16384;
constexpr int kProbeStages = kStagesC64;
constexpr int kProbeConsumers = 4;
constexpr int kProbeCtasPerSm = kC64CtasPerSm;

// One 16-byte shared-memory load that the compiler may not merge with another
// load of the same address (a probe reads the same tile more than once).
__device__ __forceinline__ float4 lds128_volatile(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}

// Tile visited by job q of CTA b: a scattered walk over the buffer's tiles.
__device__ __forceinline__ uint32_t probe_tile(uint32_t b, uint32_t q, uint32_t ntiles) {
  return (b * 977u + q * 61u) % ntiles;
}

template <int READS>
__global__ void __launch_bounds__(32 * (kProbeConsumers + 1), kProbeCtasPerSm) k_probe_stage(const float4* __restrict__ buf,
                                                                              uint32_t ntiles, uint32_t jobs,
                                                                              int* err, float* sink) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kProbeStages];
  __shared__ __align__(8) uint64_t empty_bar[kProbeStages];
  __shared__ int s_err;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kProbeStages; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), kProbeConsumers);
    }
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == kProbeConsumers) {
    if (lane == 0) {
      const uint32_t smem0 = smem_u32(smem_raw);
      uint64_t issued = 0;
      for (uint32_t q = 0; q < jobs; ++q) {
        const uint32_t stg = q % kProbeStages;
        if (q >= kProbeStages &&
            !mbar_wait_bounded(smem_u32(&empty_bar[stg]), ((q / kProbeStages) - 1u) & 1u, &s_err))
          break;
        const uint32_t bar = smem_u32(&full_bar[stg]);
        mbar_expect_tx(bar, kProbeTileBytes);
        bulk_g2s(smem0 + stg * kProbeTileBytes, buf + static_cast<size_t>(probe_tile(blockIdx.x, q, ntiles)) * 1024u,
                 kProbeTileBytes, bar);
        issued = q + 1;
      }
      if (s_err) {  // drain: the last copy issued into each stage must land before exit
        for (uint64_t qq = issued > kProbeStages ? issued - kProbeStages : 0; qq < issued; ++qq) {
          const uint32_t bar = smem_u32(&full_bar[qq % kProbeStages]);
          const uint64_t ts = globaltimer_ns();
          while (!mbar_try_wait(bar, static_cast<uint32_t>((qq / kProbeStages) & 1)) &&
                 globaltimer_ns() - ts < kWaitLimitNs) {
          }
        }
      }
    }
  } else {
    float acc = 0.f;
    for (uint32_t q = 0; q < jobs; ++q) {
      const uint32_t stg = q % kProbeStages;
      if (!mbar_wait_bounded(smem_u32(&full_bar[stg]), (q / kProbeStages) & 1u, &s_err)) break;
      const uint32_t t4 = smem_u32(smem_raw + stg * kProbeTileBytes);
#pragma unroll
      for (int r = 0; r < READS; ++r)
#pragma unroll
        for (int i = 0; i < 8; ++i) {  // 1024 float4 per tile: 8 per consumer thread
          const float4 v = lds128_volatile(t4 + 16u * ((warp * 32u + lane) + 128u * i));
          acc += (v.x + v.y) + (v.z + v.w);
        }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[stg])) : "memory");
    }
    if (acc == 1234.5f) *sink = acc;  // keeps the reads
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_err) atomicExch(err, 1);
}

// The same tiles read with 16-byte global loads that do not allocate in L1.
__global__ void __launch_bounds__(128) k_probe_ldg(const float4* __restrict__ buf, uint32_t ntiles, uint32_t jobs,
                                                   float* sink) {
  float acc = 0.f;
  for (uint32_t q = 0; q < jobs; ++q) {
    const float4* t4 = buf + static_cast<size_t>(probe_tile(blockIdx.x, q, ntiles)) * 1024u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4 v;
      asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "l"(t4 + threadIdx.x + 128u * i));
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == 1234.5f) *sink = acc;
}

// Shared-memory loads only: each thread of a 128-thread CTA reads 8 float4 of
// a 16 KiB tile per iteration (index (thread + 128 i + 32 it) mod 1024, so a
// warp's load covers 512 contiguous bytes), into four independent sums.
constexpr int kLdsThreads = 128;
constexpr int kLdsCtasPerSm = 8;
__global__ void __launch_bounds__(kLdsThreads) k_probe_lds(int iters, float* sink) {
  extern __shared__ __align__(16) float4 tile[];  // 1024 float4
  for (uint32_t i = threadIdx.x; i < 1024u; i += kLdsThreads) tile[i] = make_float4(1e-7f * i, 1.f, 2.f, 3.f);
  __syncthreads();
  const uint32_t base = smem_u32(tile);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (uint32_t it = 0; it < static_cast<uint32_t>(iters); ++it) {
#pragma unroll
    for (uint32_t i = 0; i < 8u; ++i) {
      const float4 v = lds128_volatile(base + 16u * ((threadIdx.x + 128u * i + 32u * it) & 1023u));
      s0 += v.x;
      s1 += v.y;
      s2 += v.z;
      s3 += v.w;
    }
  }
  if ((s0 + s1) + (s2 + s3) == 1234.5f) *sink = s0;  // keeps the loads
}

__global__ void __launch_bounds__(256) k_probe_dfma(double* sink, int iters) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  const double m = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __fma_rn(a[k], m, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 1234.5) *sink = s;
}

struct ProbeBuffers {
  int* err = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProbeBuffers() {
    if (cudaMalloc(&err, sizeof(int) + 256) != cudaSuccess) {
      cudaGetLastError();
      err = nullptr;
      throw Error(SYK_ENOMEM, "probe: device allocation failed");
    }
    sink = reinterpret_cast<float*>(reinterpret_cast<char*>(err) + 128);
    SYK_CUDA(cudaMemset(err, 0, sizeof(int)));
    SYK_CUDA(cudaEventCreate(&e0));
    SYK_CUDA(cudaEventCreate(&e1));
  }
  ~ProbeBuffers() {
    if (err) cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

template <typename F>
int probe_guard(const char* fn, F&& f) {
  try {
    f();
    return SYK_OK;
  } catch (const Error& e) {
    set_last_error(std::string(fn) + ": " + e.what());
    return e.code;
  }
}

}  // namespace
}  // namespace syk

extern "C" int syk_probe_staging(const void* buf, size_t bytes, int reads, int jobs_per_cta, double* bytes_per_s,
                                 syk_stream_t stream) {
  return syk::probe_guard("syk_probe_staging", [&] {
    SYK_REQUIRE(buf && bytes_per_s, "null argument");
    SYK_REQUIRE((reinterpret_cast<uintptr_t>(buf) & 15) == 0, "buffer must be 16-byte aligned");
    SYK_REQUIRE(bytes >= syk::kProbeTileBytes && bytes / syk::kProbeTileBytes <= (1u << 30), "bad buffer size");
    SYK_REQUIRE(reads >= -1 && reads <= 2, "reads must be -1 (plain loads), 0, 1 or 2");
    SYK_REQUIRE(jobs_per_cta >= 1 && jobs_per_cta <= (1 << 20), "jobs_per_cta out of range");
    auto st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t ntiles = static_cast<uint32_t>(bytes / syk::kProbeTileBytes);
    const int grid = nsm * syk::kProbeCtasPerSm;
    const size_t dyn = syk::kProbeStages * syk::kProbeTileBytes;
    const float4* b4 = static_cast<const float4*>(buf);
    syk::ProbeBuffers pb;
    auto launch = [&]() {
      switch (reads) {
        case -1:
          syk::k_probe_ldg<<<grid, 128, 0, st>>>(b4, ntiles, jobs_per_cta, pb.sink);
          break;
        case 0:
          syk::k_probe_stage<0><<<grid, 32 * (syk::kProbeConsumers + 1), dyn, st>>>(b4, ntiles, jobs_per_cta,
                                                                                     pb.err, pb.sink);
          break;
        case 1:
          syk::k_probe_stage<1><<<grid, 32 * (syk::kProbeConsumers + 1), dyn, st>>>(b4, ntiles, jobs_per_cta,
                                                                                     pb.err, pb.sink);
          break;
        default:
          syk::k_probe_stage<2><<<grid, 32 * (syk::kProbeConsumers + 1), dyn, st>>>(b4, ntiles, jobs_per_cta,
                                                                                     pb.err, pb.sink);
      }
      SYK_CUDA(cudaGetLastError());
    };
    SYK_CUDA(cudaFuncSetAttribute(syk::k_probe_stage<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(dyn)));
    SYK_CUDA(cudaFuncSetAttribute(syk::k_probe_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(dyn)));
    SYK_CUDA(cudaFuncSetAttribute(syk::k_probe_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(dyn)));
    launch();  // warm-up: the buffer becomes L2-resident
    SYK_CUDA(cudaEventRecord(pb.e0, st));
    launch();
    SYK_CUDA(cudaEventRecord(pb.e1, st));
    SYK_CUDA(cudaEventSynchronize(pb.e1));
    float ms = 0.f;
    SYK_CUDA(cudaEventElapsedTime(&ms, pb.e0, pb.e1));
    int e = 0;
    SYK_CUDA(cudaMemcpy(&e, pb.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) throw syk::Error(SYK_ETIMEOUT, "a bounded wait expired");
    *bytes_per_s = static_cast<double>(grid) * jobs_per_cta * syk::kProbeTileBytes / (ms * 1e-3);
  });
}

extern "C" int syk_probe_smem(double* bytes_per_s, syk_stream_t stream) {
  return syk::probe_guard("syk_probe_smem", [&] {
    SYK_REQUIRE(bytes_per_s, "null argument");
    auto st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    syk::ProbeBuffers pb;
    const int grid = nsm * syk::kLdsCtasPerSm, iters = 4096;
    const size_t dyn = 16384;
    syk::k_probe_lds<<<grid, syk::kLdsThreads, dyn, st>>>(64, pb.sink);  // warm-up
    SYK_CUDA(cudaGetLastError());
    SYK_CUDA(cudaEventRecord(pb.e0, st));
    syk::k_probe_lds<<<grid, syk::kLdsThreads, dyn, st>>>(iters, pb.sink);
    SYK_CUDA(cudaEventRecord(pb.e1, st));
    SYK_CUDA(cudaEventSynchronize(pb.e1));
    float ms = 0.f;
    SYK_CUDA(cudaEventElapsedTime(&ms, pb.e0, pb.e1));
    *bytes_per_s = static_cast<double>(grid) * syk::kLdsThreads * 8.0 * 16.0 * iters / (ms * 1e-3);
  });
}

extern "C" int syk_probe_fp64(double* dfma_per_s, syk_stream_t stream) {
  return syk::probe_guard("syk_probe_fp64", [&] {
    SYK_REQUIRE(dfma_per_s, "null argument");
    auto st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    SYK_CUDA(cudaGetDevice(&dev));
    SYK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    syk::ProbeBuffers pb;
    const int grid = nsm * 8, iters = 2048;
    double* sink = reinterpret_cast<double*>(pb.sink);
    syk::k_probe_dfma<<<grid, 256, 0, st>>>(sink, 64);  // warm-up
    SYK_CUDA(cudaGetLastError());
    SYK_CUDA(cudaEventRecord(pb.e0, st));
    syk::k_probe_dfma<<<grid, 256, 0, st>>>(sink, iters);
    SYK_CUDA(cudaEventRecord(pb.e1, st));
    SYK_CUDA(cudaEventSynchronize(pb.e1));
    float ms = 0.f;
    SYK_CUDA(cudaEventElapsedTime(&ms, pb.e0, pb.e1));
    *dfma_per_s = static_cast<double>(grid) * 256.0 * 8.0 * iters / (ms * 1e-3);
  });
}
