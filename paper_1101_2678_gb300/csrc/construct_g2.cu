// Construction kernel instantiations with 2 warp(s) per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g2(const Instance& I, int C, int A, cudaStream_t st) {
  const int threads = 32 * 2 * A;
  const int grid = (I.m + A - 1) / A;
  switch (C) {
    case 12: {
      const size_t smem = construct_smem_setup<12, 2, false>(A);
      construct_kernel<12, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 2, false>(A);
      construct_kernel<20, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 2, false>(A);
      construct_kernel<28, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 2, false>(A);
      construct_kernel<36, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 2, false>(A);
      construct_kernel<44, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 2, false>(A);
      construct_kernel<52, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 2, false>(A);
      construct_kernel<60, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 2, false>(A);
      construct_kernel<68, 2><<<grid, threads, smem, st>>>(I);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_construct_items_g2(const Instance* insts, const int2* items, int count,
                                         int C, int A, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 32 * 2 * A;
  const int grid = (count + A - 1) / A;
  switch (C) {
    case 12: {
      const size_t smem = construct_smem_setup<12, 2, true>(A);
      construct_items_kernel<12, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 2, true>(A);
      construct_items_kernel<20, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 2, true>(A);
      construct_items_kernel<28, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 2, true>(A);
      construct_items_kernel<36, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 2, true>(A);
      construct_items_kernel<44, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 2, true>(A);
      construct_items_kernel<52, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 2, true>(A);
      construct_items_kernel<60, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 2, true>(A);
      construct_items_kernel<68, 2><<<grid, threads, smem, st>>>(insts, items, count);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
