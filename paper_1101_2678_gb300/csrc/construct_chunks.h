// Chunk widths (cities per lane) compiled for each construction tiling,
// shared by the launch tables (construct_dispatch.cuh) and the tiling choice
// on the host (colony.cu).
#pragma once

namespace aco {

template <int... Cs>
struct ChunkList {};

// Widths compiled per tiling: C = 4 + 8k (C/4 odd, conflict-free chunk reads).
using ChunksOneWarp = ChunkList<4, 12, 20, 28, 36, 44, 52, 60, 68, 76>;  // G = 1, any H
using ChunksTwoWarps = ChunkList<12, 20, 28, 36, 44, 52, 60, 68>;        // G = 2
using ChunksFourWarps = ChunkList<4, 12, 20, 28, 36>;                     // G = 4

template <int... Cs>
constexpr int chunk_count(ChunkList<Cs...>) {
  return sizeof...(Cs);
}

template <int... Cs>
inline const int* chunk_values(ChunkList<Cs...>) {
  static constexpr int v[] = {Cs...};
  return v;
}

}  // namespace aco
