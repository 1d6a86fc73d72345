// Self-test of the bounded device-side wait (library robustness; the paper
// has no counterpart).  One warp initialises an mbarrier, expects 16 bytes
// on it and then waits with the same bounded loop the construction kernel
// uses.  With `complete` set, a real 16-byte bulk copy delivers the bytes and
// the wait succeeds; without it nothing ever completes the phase, the wait
// gives up after `polls` polls and the kernel records kStatusTimeout.  No
// copy is left in flight either way, so the kernel ends cleanly.
#include "../../include/aco.h"
#include "aco_device.cuh"
#include "construct.cuh"
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

namespace aco {

// The device Philox4x32-10 (the generator of every kernel) on given counters.
__global__ void philox_words_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                    uint4* __restrict__ out, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint4 c = ctr[i];
    const Philox4 x = philox4x32_10(c.x, c.y, c.z, c.w, k0, k1);
    out[i] = make_uint4(x.x0, x.x1, x.x2, x.x3);
  }
}

}  // namespace aco

extern "C" int aco_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                 int32_t count) {
  if (!ctr || !key || !out) return fail(ACO_EINVAL, "NULL argument");
  if (count < 1 || count > (1 << 24)) return fail(ACO_EINVAL, "count outside [1, 2^24]");
  const size_t bytes = (size_t)count * 16;
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * bytes);
  if (e != cudaSuccess) return cuda_fail(e, "philox alloc");
  uint4* dc = static_cast<uint4*>(d);
  uint4* dout = dc + count;
  e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    int blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    philox_words_kernel<<<blocks, 256>>>(dc, key[0], key[1], dout, count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "philox");
  return ACO_OK;
}

namespace aco {

// The exponential race's variate E(x) (the construction kernels' function).
__global__ void race_exponential_kernel(const uint32_t* __restrict__ x, float* __restrict__ out,
                                        int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = race_exponential(x[i]);
}

}  // namespace aco

extern "C" int aco_race_exponential(const uint32_t* x, float* out, int32_t count) {
  if (!x || !out) return fail(ACO_EINVAL, "NULL argument");
  if (count < 1 || count > (1 << 24)) return fail(ACO_EINVAL, "count outside [1, 2^24]");
  const size_t bytes = (size_t)count * 4;
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * bytes);
  if (e != cudaSuccess) return cuda_fail(e, "race alloc");
  uint32_t* dx = static_cast<uint32_t*>(d);
  float* dout = reinterpret_cast<float*>(dx + count);
  e = cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    int blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    race_exponential_kernel<<<blocks, 256>>>(dx, dout, count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "race exponential");
  return ACO_OK;
}
