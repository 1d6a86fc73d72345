// Construction kernel instantiations with 4 warp(s) per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g4(const Instance& I, int C, int A, cudaStream_t st) {
  const int threads = 32 * 4 * A;
  const int grid = (I.m + A - 1) / A;
  switch (C) {
    case 4: {
      const size_t smem = construct_smem_setup<4, 4, false>(A);
      construct_kernel<4, 4><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 12: {
      const size_t smem = construct_smem_setup<12, 4, false>(A);
      construct_kernel<12, 4><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 4, false>(A);
      construct_kernel<20, 4><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 4, false>(A);
      construct_kernel<28, 4><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 4, false>(A);
      construct_kernel<36, 4><<<grid, threads, smem, st>>>(I);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_construct_items_g4(const Instance* insts, const int2* items, int count,
                                         int C, int A, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 32 * 4 * A;
  const int grid = (count + A - 1) / A;
  switch (C) {
    case 4: {
      const size_t smem = construct_smem_setup<4, 4, true>(A);
      construct_items_kernel<4, 4><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 12: {
      const size_t smem = construct_smem_setup<12, 4, true>(A);
      construct_items_kernel<12, 4><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 4, true>(A);
      construct_items_kernel<20, 4><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 4, true>(A);
      construct_items_kernel<28, 4><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 4, true>(A);
      construct_items_kernel<36, 4><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
