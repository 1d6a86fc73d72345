// Construction kernel instantiations: 2 warp(s) per ant group, 32 lanes per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g2h32(const Instance& I, int C, int warps, cudaStream_t st) {
  const int per_cta = groups_per_cta<2, 32>(warps);
  const int grid = (I.m + per_cta - 1) / per_cta;
  const int threads = 32 * warps;
  switch (C) {
    case 12: {
      const size_t smem = construct_smem_setup<12, 2, 32, false>(warps);
      construct_kernel<12, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 2, 32, false>(warps);
      construct_kernel<20, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 2, 32, false>(warps);
      construct_kernel<28, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 2, 32, false>(warps);
      construct_kernel<36, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 2, 32, false>(warps);
      construct_kernel<44, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 2, 32, false>(warps);
      construct_kernel<52, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 2, 32, false>(warps);
      construct_kernel<60, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 2, 32, false>(warps);
      construct_kernel<68, 2, 32><<<grid, threads, smem, st>>>(I);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_construct_items_g2h32(const Instance* insts, const int2* items, int count,
                                          int C, int warps, int lane_copy, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int per_cta = groups_per_cta<2, 32>(warps);
  const int grid = (count + per_cta - 1) / per_cta;
  const int threads = 32 * warps;
  switch (C) {
    case 12: {
      const size_t smem = construct_smem_setup<12, 2, 32, true>(warps);
      construct_items_kernel<12, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 2, 32, true>(warps);
      construct_items_kernel<20, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 2, 32, true>(warps);
      construct_items_kernel<28, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 2, 32, true>(warps);
      construct_items_kernel<36, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 2, 32, true>(warps);
      construct_items_kernel<44, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 2, 32, true>(warps);
      construct_items_kernel<52, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 2, 32, true>(warps);
      construct_items_kernel<60, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 2, 32, true>(warps);
      construct_items_kernel<68, 2, 32><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
