// Construction kernel instantiations with 1 warp(s) per ant.
#include "construct.cuh"
#include "kernels.h"

namespace aco {

cudaError_t launch_construct_g1(const Instance& I, int C, int A, cudaStream_t st) {
  const int threads = 32 * 1 * A;
  const int grid = (I.m + A - 1) / A;
  switch (C) {
    case 4:
      construct_kernel<4, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 8:
      construct_kernel<8, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 12:
      construct_kernel<12, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 16:
      construct_kernel<16, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 20:
      construct_kernel<20, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 24:
      construct_kernel<24, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 32:
      construct_kernel<32, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 40:
      construct_kernel<40, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 48:
      construct_kernel<48, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 64:
      construct_kernel<64, 1><<<grid, threads, 0, st>>>(I);
      break;
    case 80:
      construct_kernel<80, 1><<<grid, threads, 0, st>>>(I);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_construct_items_g1(const Instance* insts, const int2* items, int count,
                                         int C, int A, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 32 * 1 * A;
  const int grid = (count + A - 1) / A;
  switch (C) {
    case 4:
      construct_items_kernel<4, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 8:
      construct_items_kernel<8, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 12:
      construct_items_kernel<12, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 16:
      construct_items_kernel<16, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 20:
      construct_items_kernel<20, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 24:
      construct_items_kernel<24, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 32:
      construct_items_kernel<32, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 40:
      construct_items_kernel<40, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 48:
      construct_items_kernel<48, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 64:
      construct_items_kernel<64, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    case 80:
      construct_items_kernel<80, 1><<<grid, threads, 0, st>>>(insts, items, count);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aco
