// One persistent construction launch over every (instance, ant) item of a
// pool step (the batching pattern's single launch per phase), measured
// against one launch per tiling class.
//
// Each warp builds one ant at a time: it takes the next item from a global
// ticket (atomicAdd; no waiting on other warps), finds the item's class (the
// classes are listed largest chunk first, so the longest instances are taken
// first) and runs the Eq. 1 walk with that class's chunk width.  Every width
// is a separate code path of the one kernel, all under one register cap
// (64: the widest path spills a little, but the narrower ones, most of the
// work, keep 32 warps per SM; measured 24.36 ms per batched step against
// 24.49 at 72 and 25.01 at 80).
#include "construct.cuh"
#include "kernels.h"

namespace aco {

namespace {

constexpr int kSingleWarps = 4;
constexpr int kSingleBytes = StageLayout<36, 1, 32>::kBytes;  // the widest chunk handled

__global__ void __maxnreg__(64)
    construct_single_kernel(const Instance* __restrict__ insts, const int2* __restrict__ items,
                            SingleClasses cls, int total, int* ticket) {
  __shared__ GroupSmem gs[kSingleWarps];
  extern __shared__ __align__(16) unsigned char stage[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* srow = reinterpret_cast<float*>(stage + warp * kSingleBytes);
  const Seg<32> seg(lane);
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    if (t >= total) break;
    int k = 0, idx = t;
    while (k < cls.n - 1 && idx >= cls.count[k]) {
      idx -= cls.count[k];
      ++k;
    }
    const int2 it = items[cls.begin[k] + idx];
    const Instance& I = insts[it.x];
    const bool lc = cls.lane_copy[k] != 0;
    switch (cls.C[k]) {
      case 4:
        construct_ant<4, 1, 32, 0, true>(I, it.y, lane, seg, &gs[warp], 1 + warp, srow, lc);
        break;
      case 12:
        construct_ant<12, 1, 32, 0, true>(I, it.y, lane, seg, &gs[warp], 1 + warp, srow, lc);
        break;
      case 20:
        construct_ant_phased<20, 1, 32, true>(I, it.y, lane, seg, &gs[warp], 1 + warp, srow, lc);
        break;
      case 28:
        construct_ant_phased<28, 1, 32, true>(I, it.y, lane, seg, &gs[warp], 1 + warp, srow, lc);
        break;
      case 36:
        construct_ant_phased<36, 1, 32, true>(I, it.y, lane, seg, &gs[warp], 1 + warp, srow, lc);
        break;
      default:
        break;
    }
    __syncwarp();
  }
}

}  // namespace

bool single_launch_supports(int C) { return C == 4 || C == 12 || C == 20 || C == 28 || C == 36; }

cudaError_t launch_construct_single(const Instance* insts, const int2* items,
                                    const SingleClasses& cls, int total, int* ticket, int sms,
                                    cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  static std::atomic<unsigned long long> done{0};
  const int smem = kSingleWarps * kSingleBytes;
  cudaError_t e = once_per_device(done, [smem] {
    return cudaFuncSetAttribute(construct_single_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ticket, 0, sizeof(int), st)) != cudaSuccess) return e;
  // 64 registers: 32 resident warps per SM, eight CTAs of four warps.
  construct_single_kernel<<<sms * 8, 32 * kSingleWarps, smem, st>>>(insts, items, cls, total,
                                                                     ticket);
  return cudaGetLastError();
}

}  // namespace aco
