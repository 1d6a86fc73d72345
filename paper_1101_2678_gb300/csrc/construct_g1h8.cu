// Construction kernel instantiations: 1 warp(s) per ant group, 8 lanes per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g1h8(const Instance& I, int C, int warps, cudaStream_t st) {
  const int per_cta = groups_per_cta<1, 8>(warps);
  const int grid = (I.m + per_cta - 1) / per_cta;
  const int threads = 32 * warps;
  switch (C) {
    case 4: {
      const size_t smem = construct_smem_setup<4, 1, 8, false>(warps);
      construct_kernel<4, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 12: {
      const size_t smem = construct_smem_setup<12, 1, 8, false>(warps);
      construct_kernel<12, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 1, 8, false>(warps);
      construct_kernel<20, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 1, 8, false>(warps);
      construct_kernel<28, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 1, 8, false>(warps);
      construct_kernel<36, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 1, 8, false>(warps);
      construct_kernel<44, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 1, 8, false>(warps);
      construct_kernel<52, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 1, 8, false>(warps);
      construct_kernel<60, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 1, 8, false>(warps);
      construct_kernel<68, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 76: {
      const size_t smem = construct_smem_setup<76, 1, 8, false>(warps);
      construct_kernel<76, 1, 8><<<grid, threads, smem, st>>>(I);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_construct_items_g1h8(const Instance* insts, const int2* items, int count,
                                          int C, int warps, int lane_copy, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int per_cta = groups_per_cta<1, 8>(warps);
  const int grid = (count + per_cta - 1) / per_cta;
  const int threads = 32 * warps;
  switch (C) {
    case 4: {
      const size_t smem = construct_smem_setup<4, 1, 8, true>(warps);
      construct_items_kernel<4, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 12: {
      const size_t smem = construct_smem_setup<12, 1, 8, true>(warps);
      construct_items_kernel<12, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 1, 8, true>(warps);
      construct_items_kernel<20, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 1, 8, true>(warps);
      construct_items_kernel<28, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 1, 8, true>(warps);
      construct_items_kernel<36, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 1, 8, true>(warps);
      construct_items_kernel<44, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 1, 8, true>(warps);
      construct_items_kernel<52, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 1, 8, true>(warps);
      construct_items_kernel<60, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 1, 8, true>(warps);
      construct_items_kernel<68, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    case 76: {
      const size_t smem = construct_smem_setup<76, 1, 8, true>(warps);
      construct_items_kernel<76, 1, 8><<<grid, threads, smem, st>>>(insts, items, count, lane_copy);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
