// Launcher of the construction kernels with a per-candidate random rule
// (R = 1: the paper's data-parallel rule; R = 2: the exponential race),
// whole warps per ant (G = 1 or 2); one translation unit per rule.
#pragma once

#include "construct_dispatch.cuh"

namespace aco {

template <int R>
inline cudaError_t launch_construct_rule(const Instance& I, ConstructTiling t, cudaStream_t st) {
  if (t.H != 32 || (t.G != 1 && t.G != 2)) return cudaErrorInvalidValue;
  if (t.G == 1) return launch_construct_table<1, 32, R>(ChunksOneWarp{}, I, t.C, t.W, st);
  return launch_construct_table<2, 32, R>(ChunksTwoWarps{}, I, t.C, t.W, st);
}

}  // namespace aco
