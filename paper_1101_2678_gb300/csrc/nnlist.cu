// Nearest-neighbour-list construction (the construction of the paper's
// Table 2 versions 4-6, Section II): an ant at city i samples Eq. 1 among the
// unvisited cities of list(i), the nn nearest cities of i; if all of them are
// visited it moves to the unvisited city with the largest choice_info value.
#include <algorithm>
#include <climits>

#include "aco_device.cuh"
#include "construct.cuh"
#include "kernels.h"

namespace aco {

// list(i) = the nn cities j != i with the smallest (d_ij, j), in that order:
// one warp per row, nn rounds of a lexicographic minimum above the previous
// pick.
__global__ void nn_list_kernel(Instance I, int nn) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * warps + (threadIdx.x >> 5);
  if (i >= I.n) return;
  const int n = I.n;
  const int32_t* row = I.dist + (size_t)i * I.ld;
  long long last_d = -1;
  int last_j = -1;
  for (int l = 0; l < nn; ++l) {
    long long bd = LLONG_MAX;
    int bj = INT_MAX;
    for (int j = lane; j < n; j += 32) {
      if (j == i) continue;
      const long long dj = row[j];
      const bool after = dj > last_d || (dj == last_d && j > last_j);
      if (after && (dj < bd || (dj == bd && j < bj))) {
        bd = dj;
        bj = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long od = __shfl_xor_sync(FULL, bd, o);
      const int oj = __shfl_xor_sync(FULL, bj, o);
      if (od < bd || (od == bd && oj < bj)) {
        bd = od;
        bj = oj;
      }
    }
    if (lane == 0) I.nnlist[(size_t)i * kNnStride + l] = bj;
    last_d = bd;
    last_j = bj;
  }
}

// nnchoice[i][l] = choice[i][list(i)[l]].
__global__ void nn_choice_kernel(Instance I) {
  const size_t total = (size_t)I.n * kNnStride;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kNnStride), l = (int)(e % kNnStride);
    if (l < I.nn) I.nnchoice[e] = I.choice[(size_t)i * I.ld + I.nnlist[e]];
  }
}

// One warp per ant; lane l holds list entry l of the current city.  The
// tabu list is a bitmap of n bits in shared memory (one per warp).
__device__ __forceinline__ void nn_construct_ant(const Instance& I, const int ant, const int lane,
                                                 uint32_t* bits) {
  const int n = I.n, nn = I.nn, ld = I.ld, words = (n + 31) >> 5;
  const uint32_t iter = (uint32_t)I.st->iteration;
  const unsigned long long seed = I.seed;
  for (int i = lane; i < words; i += 32) bits[i] = 0u;
  __syncwarp();
  const Philox4 x0 = step_draw(seed, 0u, (uint32_t)ant, iter);
  const int start = (int)__umulhi(x0.x0, (uint32_t)n);
  int32_t* tour = I.tours + (size_t)ant * I.ldt;
  if (lane == 0) {
    bits[start >> 5] |= 1u << (start & 31);
    tour[0] = start;
  }
  __syncwarp();
  int cur = start;
  unsigned long long rwin = 0;
  for (int s = 1; s < n; ++s) {
    const int off = (s - 1) & 31;
    if (off == 0) {
      const Philox4 x = step_draw(seed, (uint32_t)(s + lane), (uint32_t)ant, iter);
      rwin = ((unsigned long long)x.x1 << 32) | x.x0;
    }
    const unsigned long long r = shfl_u64(rwin, off);
    int j = 0;
    uint32_t wb = 0u;
    bool unv = false;
    if (lane < nn) {
      j = I.nnlist[(size_t)cur * kNnStride + lane];
      wb = __float_as_uint(I.nnchoice[(size_t)cur * kNnStride + lane]);
      unv = !((bits[j >> 5] >> (j & 31)) & 1u);
    }
    const uint32_t any = __ballot_sync(FULL, unv);
    int next;
    if (any) {
      const uint32_t wm = unv ? wb : 0u;
      const uint32_t mx = __reduce_max_sync(FULL, wm);
      if (mx == 0u) {
        next = __shfl_sync(FULL, j, __ffs(any) - 1);  // first unvisited entry
      } else {
        float f1, f1s, f2;
        quant_factors(kRouletteBits - 1 - exponent_of_bits(mx), f1, f1s, f2);
        const unsigned long long q = quant_value(wm, f1, f1s, f2);
        unsigned long long incl = q;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long t = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += t;
        }
        const unsigned long long T = __umul64hi(r, shfl_u64(incl, 31));
        const int L = max(__ffs(__ballot_sync(FULL, incl > T)) - 1, 0);
        next = __shfl_sync(FULL, j, L);
      }
    } else {
      // Every list entry is visited: the heaviest unvisited city, ties to
      // the lower index ((weight bits << 32) | ~j, maximised).
      const float* row = I.choice + (size_t)cur * ld;
      unsigned long long key = 0;
      for (int jj = lane; jj < n; jj += 32) {
        if ((bits[jj >> 5] >> (jj & 31)) & 1u) continue;
        const unsigned long long k =
            ((unsigned long long)__float_as_uint(row[jj]) << 32) | (0xffffffffu - (uint32_t)jj);
        key = k > key ? k : key;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(FULL, key, o);
        key = other > key ? other : key;
      }
      next = (int)(0xffffffffu - (uint32_t)key);
    }
    if ((unsigned)next >= (unsigned)n) {
      if (lane == 0) atomicOr(&I.st->status, kStatusBadTour);
      next = start;
    }
    if (lane == 0) {
      bits[next >> 5] |= 1u << (next & 31);
      tour[s] = next;
    }
    __syncwarp();
    cur = next;
  }
  if (lane == 0) tour[n] = start;
  __syncwarp();
  long long len = 0;
  for (int s = lane; s < n; s += 32) {
    const int a = tour[s], b = tour[s + 1];
    const int p = tour[s == 0 ? n - 1 : s - 1];
    len += I.dist[(size_t)a * ld + b];
    I.nbr[(size_t)a * I.ldm + ant] = ((uint32_t)p << 16) | (uint32_t)b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(FULL, len, o);
  if (lane == 0) I.lens[ant] = len;
}

__global__ void __launch_bounds__(128) construct_nn_kernel(Instance I) {
  extern __shared__ uint32_t nn_bits[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ant = blockIdx.x * (blockDim.x >> 5) + warp;
  if (ant >= I.m) return;
  nn_construct_ant(I, ant, lane, nn_bits + (size_t)warp * ((I.n + 31) / 32));
}

// Many instances: warp w builds ant items[w].y of instance insts[items[w].x];
// the bitmaps are sized for the largest n among them.
__global__ void __launch_bounds__(128) construct_nn_items_kernel(
    const Instance* __restrict__ insts, const int2* __restrict__ items, int count, int words) {
  extern __shared__ uint32_t nn_bits[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  if (idx >= count) return;
  const int2 it = items[idx];
  nn_construct_ant(insts[it.x], it.y, lane, nn_bits + (size_t)warp * words);
}

// nnchoice refresh for many instances: block row y serves insts[slots[y]].
__global__ void nn_choice_slots_kernel(const Instance* __restrict__ insts,
                                       const int* __restrict__ slots) {
  const Instance& I = insts[slots[blockIdx.y]];
  const size_t total = (size_t)I.n * kNnStride;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kNnStride), l = (int)(e % kNnStride);
    if (l < I.nn) I.nnchoice[e] = I.choice[(size_t)i * I.ld + I.nnlist[e]];
  }
}

cudaError_t launch_nn_lists(const Instance& I, int nn, cudaStream_t st) {
  nn_list_kernel<<<(I.n + 3) / 4, 128, 0, st>>>(I, nn);
  return cudaGetLastError();
}

cudaError_t launch_nn_choice(const Instance& I, cudaStream_t st) {
  const size_t total = (size_t)I.n * kNnStride;
  size_t blocks = (total + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  nn_choice_kernel<<<(int)blocks, 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_construct_nn(const Instance& I, cudaStream_t st) {
  const int warps = 4;
  const size_t smem = (size_t)warps * ((I.n + 31) / 32) * sizeof(uint32_t);
  construct_nn_kernel<<<(I.m + warps - 1) / warps, 32 * warps, smem, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_construct_nn_items(const Instance* insts, const int2* items, int count,
                                      int max_n, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int warps = 4, words = (max_n + 31) / 32;
  const size_t smem = (size_t)warps * words * sizeof(uint32_t);
  construct_nn_items_kernel<<<(count + warps - 1) / warps, 32 * warps, smem, st>>>(insts, items,
                                                                                  count, words);
  return cudaGetLastError();
}

cudaError_t launch_nn_choice_slots(const Instance* insts, const int* slots, int count,
                                   int max_n, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t total = (size_t)max_n * kNnStride;
  const unsigned bx = (unsigned)std::min<size_t>((total + 255) / 256, 64);
  nn_choice_slots_kernel<<<dim3(bx, (unsigned)count), 256, 0, st>>>(insts, slots);
  return cudaGetLastError();
}

}  // namespace aco
