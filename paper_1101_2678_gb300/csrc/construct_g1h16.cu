// Construction kernel instantiations: 1 warp(s) per ant group, 16 lanes per ant.
#include "construct_dispatch.cuh"

namespace aco {

cudaError_t launch_construct_g1h16(const Instance& I, int C, int warps, cudaStream_t st) {
  return launch_construct_table<1, 16>(ChunksOneWarp{}, I, C, warps, st);
}

cudaError_t launch_construct_items_g1h16(const Instance* insts, const int2* items, int count,
                                          int C, int warps, int lane_copy, cudaStream_t st) {
  return launch_construct_items_table<1, 16>(ChunksOneWarp{}, insts, items, count, C, warps,
                                                lane_copy, st);
}

}  // namespace aco
