// Failure-detection self-test: one CTA waits, through the same bounded wait
// the TMA pipelines use, on an mbarrier whose phase nothing ever completes.
// The wait gives up after its limit (1 s of %globaltimer), records the
// failure, and the call reports SYK_ETIMEOUT; nothing faults, traps or hangs,
// so the context stays usable.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "tma_common.cuh"

namespace syk {
namespace {

// flag: 1 when the bounded wait expired, 0 if the barrier completed.
__global__ void k_bounded_wait_selftest(int* flag) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);  // one arrival completes phase 0; none comes
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait_bounded(smem_u32(&bar), 0u, &s_err);
    *flag = ok ? 0 : (s_err ? 1 : 2);
  }
}

}  // namespace
}  // namespace syk

extern "C" int syk_bounded_wait_selftest(syk_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    syk::set_last_error("syk_bounded_wait_selftest: device allocation failed");
    return SYK_ENOMEM;
  }
  int flag = -1;
  syk::k_bounded_wait_selftest<<<1, 32, 0, st>>>(d);
  cudaError_t e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    syk::set_last_error(std::string("syk_bounded_wait_selftest: ") + cudaGetErrorString(e));
    return SYK_ECUDA;
  }
  if (flag == 1) {
    syk::set_last_error("syk_bounded_wait_selftest: the bounded wait expired (as intended)");
    return SYK_ETIMEOUT;
  }
  syk::set_last_error("syk_bounded_wait_selftest: the wait did not expire");
  return SYK_ECUDA;
}
