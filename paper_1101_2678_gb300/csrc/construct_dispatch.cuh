// Launch tables of the construction kernels.  The chunk width C (cities per
// lane) is a compile-time parameter: a lane's chunk and its tabu bits live in
// registers.  A table instantiates the kernel for a list of widths and picks
// the one asked for at run time.  Each (G, H) tiling keeps its own
// translation unit (construct_g*.cu), so the instantiations compile in
// parallel.
#pragma once

#include "construct.cuh"
#include "construct_chunks.h"
#include "kernels.h"

namespace aco {

template <int C, int G, int H, int R>
inline bool launch_one(int c, const Instance& I, int grid, int warps, cudaStream_t st) {
  if (c != C) return false;
  const size_t smem = construct_smem_setup<C, G, H, false, R>(warps);
  if constexpr (R == 0 && Compaction<C, G>::kOn)
    construct_phased_kernel<C, G, H><<<grid, 32 * warps, smem, st>>>(I);
  else
    construct_kernel<C, G, H, R><<<grid, 32 * warps, smem, st>>>(I);
  return true;
}

template <int C, int G, int H>
inline bool launch_items_one(int c, const Instance* insts, const int2* items, int count, int grid,
                             int warps, int lane_copy, cudaStream_t st) {
  if (c != C) return false;
  const size_t smem = construct_smem_setup<C, G, H, true>(warps);
  if constexpr (Compaction<C, G>::kOn)
    construct_phased_items_kernel<C, G, H><<<grid, 32 * warps, smem, st>>>(insts, items, count,
                                                                        lane_copy);
  else
    construct_items_kernel<C, G, H><<<grid, 32 * warps, smem, st>>>(insts, items, count,
                                                                    lane_copy);
  return true;
}

// One instance: m ants, groups_per_cta<G, H>(warps) ants per CTA.
template <int G, int H, int R = 0, int... Cs>
inline cudaError_t launch_construct_table(ChunkList<Cs...>, const Instance& I, int C, int warps,
                                          cudaStream_t st) {
  const int per_cta = groups_per_cta<G, H>(warps);
  if (per_cta < 1) return cudaErrorInvalidValue;
  const int grid = (I.m + per_cta - 1) / per_cta;
  if (!(launch_one<Cs, G, H, R>(C, I, grid, warps, st) || ...)) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Many instances: `count` (instance, ant) items.
template <int G, int H, int... Cs>
inline cudaError_t launch_construct_items_table(ChunkList<Cs...>, const Instance* insts,
                                                const int2* items, int count, int C, int warps,
                                                int lane_copy, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int per_cta = groups_per_cta<G, H>(warps);
  if (per_cta < 1) return cudaErrorInvalidValue;
  const int grid = (count + per_cta - 1) / per_cta;
  if (!(launch_items_one<Cs, G, H>(C, insts, items, count, grid, warps, lane_copy, st) || ...))
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace aco
