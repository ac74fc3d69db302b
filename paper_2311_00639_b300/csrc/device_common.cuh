// Device helpers shared by the libsyk translation units (internal linkage in
// each: everything lives in an anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

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

}  // namespace
}  // namespace syk
