// Read-bandwidth probes for the roofline denominators of the construction
// kernel (measurement infrastructure; the paper has no counterpart).
//
// The construction kernel's working set, the n x n choice_info matrix, stays
// in L2 (22.9 MB at n = 2392, well below the 129 MB L2), and the kernel only
// reads it.  Its ceiling is therefore the rate at which the SMs can read an
// L2-resident buffer, not an HBM copy rate.  Two probes measure that rate on
// a caller-owned device buffer:
//   mode 0: every thread streams 16-byte loads that bypass L1 (ld.global.cg),
//           four in flight per thread, 256 threads per CTA;
//   mode 1: one warp per CTA streams 16 KB chunks into shared memory with the
//           bulk-copy engine (cp.async.bulk + mbarrier, four stages), the
//           route the construction kernel's rows take.
// Each pass reads the whole buffer once; `reps` passes run in one launch so
// launch gaps do not count.  The caller times the launch with CUDA events on
// `stream` and divides reps * bytes by the time.
#include "../../include/aco.h"
#include "aco_device.cuh"
#include "runtime.h"

namespace aco {

constexpr int kReadThreads = 256;
constexpr int kBulkChunk = 16384;
constexpr int kBulkStages = 4;

__global__ void __launch_bounds__(kReadThreads)
    stream_read_float4_kernel(const float4* __restrict__ p, size_t n4, int reps,
                              float* __restrict__ sink) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  float acc = 0.0f;
  for (int r = 0; r < reps; ++r) {
    for (size_t i = tid; i < n4; i += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t j = i + (size_t)u * stride;
        v[u] = j < n4 ? __ldcg(p + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
    }
  }
  // The loads feed a store the compiler cannot drop; it never happens in
  // practice (a sum of exactly -1 from this thread's elements).
  if (acc == -1.0f) sink[0] = acc;
}

__global__ void __launch_bounds__(32)
    stream_read_bulk_kernel(const unsigned char* __restrict__ p, size_t nchunks, int reps,
                            float* __restrict__ sink, unsigned int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char sbuf[];
  const uint32_t base = smem_u32(sbuf);
  const uint32_t bars = base + kBulkStages * kBulkChunk;  // kBulkStages mbarriers
  const int lane = threadIdx.x;
  const size_t total = nchunks * (size_t)reps;
  // chunk items of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
  size_t count = 0;
  if ((size_t)blockIdx.x < total) count = (total - 1 - blockIdx.x) / gridDim.x + 1;
  if (lane == 0) {
    for (int s = 0; s < kBulkStages; ++s) mbar_init(bars + 8u * s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto src_of = [&](size_t t) {
    const size_t item = blockIdx.x + t * gridDim.x;
    return p + (item % nchunks) * (size_t)kBulkChunk;
  };
  if (lane == 0)
    for (size_t t = 0; t < count && t < (size_t)kBulkStages; ++t)
      bulk_load(base + (uint32_t)t * kBulkChunk, src_of(t), kBulkChunk, bars + 8u * (uint32_t)t);
  float acc = 0.0f;
  size_t issued = count < (size_t)kBulkStages ? count : (size_t)kBulkStages;
  size_t done = 0;
  bool ok = true;
  for (size_t t = 0; t < count; ++t) {
    const uint32_t s = (uint32_t)(t % kBulkStages);
    const uint32_t parity = (uint32_t)((t / kBulkStages) & 1);
    if (!mbar_wait_bounded(bars + 8u * s, parity)) {
      ok = false;
      break;
    }
    done = t + 1;
    // touch one word per lane of the chunk so the data is consumed
    acc += reinterpret_cast<const float*>(sbuf + s * kBulkChunk)[lane * 32];
    __syncwarp();
    if (lane == 0 && issued < count) {
      fence_proxy_async_smem();
      bulk_load(base + s * kBulkChunk, src_of(issued), kBulkChunk, bars + 8u * s);
      ++issued;
    }
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) atomicOr(status, (unsigned int)kStatusTimeout);
    // Wait (bounded again) for the copies still in flight before the CTA's
    // shared memory goes away.
    for (size_t t = done; t < issued; ++t)
      mbar_wait_bounded(bars + 8u * (uint32_t)(t % kBulkStages), (uint32_t)((t / kBulkStages) & 1));
  }
  if (acc == -1.0f) sink[0] = acc;
}

}  // namespace aco

using namespace aco;

extern "C" int aco_stream_read(const void* buf, uint64_t bytes, int32_t reps, int32_t mode,
                               int32_t blocks_per_sm, uint64_t stream, float* sink,
                               uint32_t* status) {
  if (!buf || !sink || !status) return fail(ACO_EINVAL, "NULL buffer, sink or status");
  if (((uintptr_t)buf & 15u) != 0) return fail(ACO_EINVAL, "buffer not 16-byte aligned");
  if (reps < 1 || reps > (1 << 20)) return fail(ACO_EINVAL, "reps outside [1, 2^20]");
  if (blocks_per_sm < 1 || blocks_per_sm > 32)
    return fail(ACO_EINVAL, "blocks_per_sm outside [1, 32]");
  const int sms = device_sms();
  if (sms <= 0) return fail(ACO_ECUDA, "no CUDA device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (mode == 0) {
    if (bytes == 0 || bytes % 16 != 0) return fail(ACO_EINVAL, "bytes must be a positive multiple of 16");
    stream_read_float4_kernel<<<sms * blocks_per_sm, kReadThreads, 0, st>>>(
        static_cast<const float4*>(buf), (size_t)(bytes / 16), reps, sink);
  } else if (mode == 1) {
    if (bytes == 0 || bytes % kBulkChunk != 0)
      return fail(ACO_EINVAL, "bytes must be a positive multiple of %d", kBulkChunk);
    const int smem = kBulkStages * kBulkChunk + 8 * kBulkStages;
    static std::atomic<unsigned long long> done{0};
    cudaError_t e = once_per_device(done, [smem] {
      return cudaFuncSetAttribute(stream_read_bulk_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (e != cudaSuccess) return cuda_fail(e, "bulk read attribute");
    stream_read_bulk_kernel<<<sms * blocks_per_sm, 32, smem, st>>>(
        static_cast<const unsigned char*>(buf), (size_t)(bytes / kBulkChunk), reps, sink, status);
  } else {
    return fail(ACO_EINVAL, "mode must be 0 (16-byte loads) or 1 (bulk copies)");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "stream read launch");
  return ACO_OK;
}
