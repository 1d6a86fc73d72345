// Construction kernel instantiations with 4 warp(s) per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g4(const Instance& I, int C, int A, cudaStream_t st) {
  const int threads = 32 * 4 * A;
  const int grid = (I.m + A - 1) / A;
  switch (C) {
    case 4:
      construct_kernel<4, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 8:
      construct_kernel<8, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 12:
      construct_kernel<12, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 16:
      construct_kernel<16, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 20:
      construct_kernel<20, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 24:
      construct_kernel<24, 4><<<grid, threads, 0, st>>>(I);
      break;
    case 32:
      construct_kernel<32, 4><<<grid, threads, 0, st>>>(I);
      break;
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
    case 4:
      construct_items_kernel<4, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 8:
      construct_items_kernel<8, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 12:
      construct_items_kernel<12, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 16:
      construct_items_kernel<16, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 20:
      construct_items_kernel<20, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 24:
      construct_items_kernel<24, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 32:
      construct_items_kernel<32, 4><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
