// Self-test of the bounded device-side wait (library robustness; the paper
// has no counterpart).  One warp initialises an mbarrier, expects 16 bytes
// on it and then waits with the same bounded loop the construction kernel
// uses.  With `complete` set, a real 16-byte bulk copy delivers the bytes and
// the wait succeeds; without it nothing ever completes the phase, the wait
// gives up after `polls` polls and the kernel records kStatusTimeout.  No
// copy is left in flight either way, so the kernel ends cleanly.
#include "../../include/aco.h"
#include "aco_device.cuh"
#include "runtime.h"

namespace aco {

__global__ void selftest_wait_kernel(int polls, int complete, const int4* src, int* status) {
  __shared__ __align__(16) int4 dst;
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t bar_a = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x == 0) {
    if (complete) {
      bulk_load(smem_u32(&dst), src, 16u, bar_a);
    } else {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(16)
                   : "memory");
    }
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(bar_a, 0u, polls);
  if (threadIdx.x == 0) *status = ok ? 0 : kStatusTimeout;
}

}  // namespace aco

using namespace aco;

extern "C" int aco_selftest_bounded_wait(int32_t polls, int32_t complete) {
  if (polls < 1 || polls > kWaitPolls) return fail(ACO_EINVAL, "polls outside [1, %d]", kWaitPolls);
  if (complete != 0 && complete != 1) return fail(ACO_EINVAL, "complete must be 0 or 1");
  void* buf = nullptr;  // 16 source bytes and the status word
  cudaError_t e = cudaMalloc(&buf, 32);
  if (e != cudaSuccess) return cuda_fail(e, "selftest alloc");
  int status = -1;
  e = cudaMemset(buf, 0, 32);
  if (e == cudaSuccess) {
    selftest_wait_kernel<<<1, 32>>>(polls, complete, static_cast<const int4*>(buf),
                                    reinterpret_cast<int*>(static_cast<char*>(buf) + 16));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(&status, static_cast<char*>(buf) + 16, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "selftest");
  if (status == kStatusTimeout) return fail(ACO_ETIMEOUT, "the bounded wait gave up as expected");
  return status == 0 ? ACO_OK : fail(ACO_ECUDA, "selftest status %d", status);
}
