// Construction kernel instantiations: 2 warp(s) per ant group, 32 lanes per ant.
#include "construct_dispatch.cuh"

namespace aco {

cudaError_t launch_construct_g2h32(const Instance& I, int C, int warps, cudaStream_t st) {
  return launch_construct_table<2, 32>(ChunksTwoWarps{}, I, C, warps, st);
}

cudaError_t launch_construct_items_g2h32(const Instance* insts, const int2* items, int count,
                                          int C, int warps, int lane_copy, cudaStream_t st) {
  return launch_construct_items_table<2, 32>(ChunksTwoWarps{}, insts, items, count, C, warps,
                                                lane_copy, st);
}

}  // namespace aco
