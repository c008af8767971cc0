// Self-test of the library's bounded device-side waits (failure detection without a
// GPU fault).  The step kernel and the tensor-core FNO kernels wait on mbarriers with an
// iteration limit: a wait that does not complete in time sets a status bit, the kernel
// returns, and the host reports LBM_ERR_TIMEOUT while the context stays usable.  This
// entry point runs the same form of wait on an mbarrier that nothing arrives on (or, for
// the positive case, one that has already completed) with a caller-chosen short limit,
// so that the reporting path can be exercised on a healthy GPU.
#include <stdint.h>

#include "common.cuh"
#include "sm100.cuh"

namespace lbmfno {
namespace {

constexpr unsigned kStatusCompleted = 2u;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_wait_selftest(unsigned* __restrict__ status, int arrive,
                                unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (arrive) mbar_arrive(&bar);
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(&bar, 0)) {
    if (global_ns() - t0 > limit_ns) {
      atomicOr(status, kStatusTimeout);
      return;
    }
  }
  atomicOr(status, kStatusCompleted);
}

inline cudaStream_t XS(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace lbmfno

using namespace lbmfno;

extern "C" int lbm_wait_selftest(unsigned* status_d, int arrive, double limit_ms, void* stream) {
  LBM_REQUIRE(status_d != nullptr, "lbm_wait_selftest: null status buffer");
  LBM_REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0,
              "lbm_wait_selftest: limit_ms must be in (0, 2000]");
  cudaStream_t s = XS(stream);
  LBM_CHECK_CUDA(cudaMemsetAsync(status_d, 0, sizeof(unsigned), s));
  k_wait_selftest<<<1, 32, 0, s>>>(status_d, arrive ? 1 : 0,
                                   (unsigned long long)(limit_ms * 1.0e6));
  LBM_CHECK_LAUNCH();
  unsigned st = 0;
  LBM_CHECK_CUDA(cudaMemcpyAsync(&st, status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  LBM_CHECK_CUDA(cudaStreamSynchronize(s));
  if (st & kStatusTimeout) {
    set_error("lbm_wait_selftest: the bounded wait expired after %.3f ms (status 0x%x)",
              limit_ms, st);
    return LBM_ERR_TIMEOUT;
  }
  if (!(st & kStatusCompleted)) {
    set_error("lbm_wait_selftest: the wait neither completed nor expired (status 0x%x)", st);
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
