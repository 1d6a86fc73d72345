// Launcher of the construction kernels with a per-candidate random rule
// (R = 1: the paper's data-parallel rule; R = 2: the exponential race),
// whole warps per ant (G = 1 or 2); one translation unit per rule.
#pragma once

#include "construct.cuh"
#include "kernels.h"

namespace aco {

template <int R>
inline cudaError_t launch_construct_rule(const Instance& I, ConstructTiling t, cudaStream_t st) {
  if (t.H != 32 || (t.G != 1 && t.G != 2)) return cudaErrorInvalidValue;
  const int per_cta = t.W / t.G;
  if (per_cta < 1) return cudaErrorInvalidValue;
  const int grid = (I.m + per_cta - 1) / per_cta;
  const int threads = 32 * t.W;
  if (t.G == 1) {
    switch (t.C) {
      case 4: {
        const size_t smem = construct_smem_setup<4, 1, 32, false, R>(t.W);
        construct_kernel<4, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 12: {
        const size_t smem = construct_smem_setup<12, 1, 32, false, R>(t.W);
        construct_kernel<12, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 20: {
        const size_t smem = construct_smem_setup<20, 1, 32, false, R>(t.W);
        construct_kernel<20, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 28: {
        const size_t smem = construct_smem_setup<28, 1, 32, false, R>(t.W);
        construct_kernel<28, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 36: {
        const size_t smem = construct_smem_setup<36, 1, 32, false, R>(t.W);
        construct_kernel<36, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 44: {
        const size_t smem = construct_smem_setup<44, 1, 32, false, R>(t.W);
        construct_kernel<44, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 52: {
        const size_t smem = construct_smem_setup<52, 1, 32, false, R>(t.W);
        construct_kernel<52, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 60: {
        const size_t smem = construct_smem_setup<60, 1, 32, false, R>(t.W);
        construct_kernel<60, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 68: {
        const size_t smem = construct_smem_setup<68, 1, 32, false, R>(t.W);
        construct_kernel<68, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      case 76: {
        const size_t smem = construct_smem_setup<76, 1, 32, false, R>(t.W);
        construct_kernel<76, 1, 32, R><<<grid, threads, smem, st>>>(I);
        return cudaGetLastError();
      }
      default:
        return cudaErrorInvalidValue;
    }
  }
  switch (t.C) {
    case 12: {
      const size_t smem = construct_smem_setup<12, 2, 32, false, R>(t.W);
      construct_kernel<12, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 20: {
      const size_t smem = construct_smem_setup<20, 2, 32, false, R>(t.W);
      construct_kernel<20, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 28: {
      const size_t smem = construct_smem_setup<28, 2, 32, false, R>(t.W);
      construct_kernel<28, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 36: {
      const size_t smem = construct_smem_setup<36, 2, 32, false, R>(t.W);
      construct_kernel<36, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 44: {
      const size_t smem = construct_smem_setup<44, 2, 32, false, R>(t.W);
      construct_kernel<44, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 52: {
      const size_t smem = construct_smem_setup<52, 2, 32, false, R>(t.W);
      construct_kernel<52, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 60: {
      const size_t smem = construct_smem_setup<60, 2, 32, false, R>(t.W);
      construct_kernel<60, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    case 68: {
      const size_t smem = construct_smem_setup<68, 2, 32, false, R>(t.W);
      construct_kernel<68, 2, 32, R><<<grid, threads, smem, st>>>(I);
      return cudaGetLastError();
    }
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace aco
