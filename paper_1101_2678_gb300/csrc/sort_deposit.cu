// Atomic-free deposit by sorting (Eqs. 3-4; Section III-B, the paper's
// scatter-to-gather idea done with a sort instead of an n^2-thread scan):
//  1. every tour edge (k, s) becomes the key min(a,b) * n + max(a,b) with
//     the ant index k as its value;
//  2. a stable LSD radix sort (8-bit digits, as many passes as the keys'
//     bits need) groups equal edges;
//  3. one thread per run of equal keys sums q_k over the run (exact 64-bit
//     integers, so the order inside the run does not matter) and stores it in
//     the upper-triangle accumulator cell of the edge;
//  4. the symmetric apply pass (update.cu) evaporates, adds and writes both
//     halves of tau and choice_info.
// No atomics anywhere: each sort pass counts digits per tile of kSortTile
// keys with warp match/ballot ranks and shared-memory counters, scans each
// digit's per-tile counts (one CTA per digit), and scatters every key to its
// stable position (digit start + earlier tiles' count + rank in the tile).
#include "aco_device.cuh"
#include "kernels.h"

namespace aco {

constexpr int kSortTile = 1024;  // keys per tile = threads per CTA
constexpr int kRadix = 256;

__global__ void sort_keys_kernel(Instance I, uint32_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
  const int n = I.n;
  const size_t total = (size_t)I.m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n), s = (int)(e % n);
    const int32_t* t = I.tours + (size_t)k * I.ldt;
    const uint32_t a = (uint32_t)t[s], b = (uint32_t)t[s + 1];
    keys[e] = (a < b ? a : b) * (uint32_t)n + (a < b ? b : a);
    vals[e] = (uint32_t)k;
  }
}

// Stable rank of this thread's digit among the tile's earlier keys: within
// the warp by match/popc, across warps by the exclusive per-digit prefix of
// the warps' counts (cnt[w][d], shared).  Returns the rank; cnt holds, after
// the call, the exclusive prefix over warps and tile_total[d] the count.
__device__ __forceinline__ int tile_rank(uint32_t d, bool valid, int (*cnt)[kRadix],
                                         int* tile_total) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < (kSortTile / 32) * kRadix; i += blockDim.x)
    (&cnt[0][0])[i] = 0;
  __syncthreads();
  const unsigned act = __ballot_sync(FULL, valid);
  unsigned peers = __match_any_sync(FULL, valid ? d : 0xffffffffu) & act;
  int r = 0;
  if (valid) {
    r = __popc(peers & ((1u << lane) - 1u));
    if (r == 0) cnt[warp][d] = __popc(peers);
  }
  __syncthreads();
  if (threadIdx.x < kRadix) {
    int run = 0;
    for (int w = 0; w < kSortTile / 32; ++w) {
      const int c = cnt[w][threadIdx.x];
      cnt[w][threadIdx.x] = run;
      run += c;
    }
    tile_total[threadIdx.x] = run;
  }
  __syncthreads();
  return valid ? r + cnt[warp][d] : 0;
}

// Per-tile digit counts, digit-major: hist[d * tiles + tile].
__global__ void __launch_bounds__(kSortTile) sort_hist_kernel(const uint32_t* __restrict__ keys,
                                                              size_t total, int shift,
                                                              uint32_t* __restrict__ hist,
                                                              int tiles) {
  __shared__ int cnt[kSortTile / 32][kRadix];
  __shared__ int tile_total[kRadix];
  const size_t e = (size_t)blockIdx.x * kSortTile + threadIdx.x;
  const bool valid = e < total;
  const uint32_t d = valid ? (keys[e] >> shift) & (kRadix - 1) : 0u;
  tile_rank(d, valid, cnt, tile_total);
  if (threadIdx.x < kRadix) hist[(size_t)threadIdx.x * tiles + blockIdx.x] = tile_total[threadIdx.x];
}

// Block-wide exclusive scan of one value per thread (blockDim.x = 1024);
// returns the exclusive prefix and sets *total.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                                   unsigned long long* warp_tot,
                                                                   unsigned long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long w = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += w;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    unsigned long long ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long w = __shfl_up_sync(FULL, ti, o);
      if (lane >= o) ti += w;
    }
    warp_tot[lane] = ti - t;  // exclusive prefix of the warp totals
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  const unsigned long long ex = warp_tot[warp] + incl - v;
  *total = warp_tot[32];
  __syncthreads();
  return ex;
}

// One CTA per digit d: exclusive scan, in place, of the tiles' counts of d
// (row d of the digit-major table), and the digit's total in totals[d].
__global__ void __launch_bounds__(1024) sort_rowscan_kernel(uint32_t* __restrict__ hist,
                                                            int tiles,
                                                            uint32_t* __restrict__ totals) {
  __shared__ unsigned long long warp_tot[33];
  uint32_t* row = hist + (size_t)blockIdx.x * tiles;
  const int per = (tiles + (int)blockDim.x - 1) / (int)blockDim.x;
  const int lo = (int)threadIdx.x * per;
  const int hi = lo + per < tiles ? lo + per : tiles;
  unsigned long long sum = 0;
  for (int i = lo; i < hi; ++i) sum += row[i];
  unsigned long long total;
  unsigned long long run = block_exclusive_scan(sum, warp_tot, &total);
  for (int i = lo; i < hi; ++i) {
    const uint32_t c = row[i];
    row[i] = (uint32_t)run;
    run += c;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = (uint32_t)total;
}

__global__ void __launch_bounds__(kSortTile) sort_scatter_kernel(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, size_t total, int shift,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ totals, int tiles,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
  __shared__ int cnt[kSortTile / 32][kRadix];
  __shared__ int tile_total[kRadix];
  __shared__ unsigned long long warp_tot[33];
  __shared__ uint32_t base[kRadix];
  // Start of each digit's range in the output: exclusive scan of the totals.
  {
    unsigned long long all;
    const unsigned long long ex = block_exclusive_scan(
        threadIdx.x < kRadix ? (unsigned long long)totals[threadIdx.x] : 0ull, warp_tot, &all);
    if (threadIdx.x < kRadix) base[threadIdx.x] = (uint32_t)ex;
  }
  const size_t e = (size_t)blockIdx.x * kSortTile + threadIdx.x;
  const bool valid = e < total;
  const uint32_t key = valid ? keys[e] : 0u;
  const uint32_t d = (key >> shift) & (kRadix - 1);
  const int r = tile_rank(d, valid, cnt, tile_total);
  if (valid) {
    const size_t pos = (size_t)base[d] + offs[(size_t)d * tiles + blockIdx.x] + (size_t)r;
    keys_out[pos] = key;
    vals_out[pos] = vals[e];
  }
}

// One thread per run of equal keys: the sum of q_k over the run into the
// upper-triangle accumulator cell (lo, hi) of the edge.
__global__ void sort_segment_sum_kernel(Instance I, const uint32_t* __restrict__ keys,
                                        const uint32_t* __restrict__ vals, size_t total) {
  const uint32_t n = (uint32_t)I.n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const uint32_t key = keys[e];
    if (e > 0 && keys[e - 1] == key) continue;
    unsigned long long sum = 0;
    for (size_t j = e; j < total && keys[j] == key; ++j) sum += I.q[vals[j]];
    I.acc[(size_t)(key / n) * I.ld + key % n] = sum;
  }
}

size_t sort_deposit_bytes(int n, int m) {
  const size_t total = (size_t)n * m;
  const int tiles = (int)((total + kSortTile - 1) / kSortTile);
  return 4 * total * sizeof(uint32_t) + (size_t)kRadix * (tiles + 1) * sizeof(uint32_t);
}

cudaError_t launch_sort_deposit(const Instance& I, void* scratch, int sms, cudaStream_t st) {
  const size_t total = (size_t)I.n * I.m;
  const int tiles = (int)((total + kSortTile - 1) / kSortTile);
  uint32_t* k0 = static_cast<uint32_t*>(scratch);
  uint32_t* v0 = k0 + total;
  uint32_t* k1 = v0 + total;
  uint32_t* v1 = k1 + total;
  uint32_t* hist = v1 + total;
  uint32_t* totals = hist + (size_t)kRadix * tiles;
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)sms * 8) blocks = (size_t)sms * 8;
  sort_keys_kernel<<<(int)blocks, 256, 0, st>>>(I, k0, v0);
  cudaError_t e = cudaGetLastError();
  // key < n^2: bits of the largest key, in 8-bit digits
  const unsigned long long kmax = (unsigned long long)I.n * I.n - 1;
  int bits = 1;
  while (bits < 32 && (kmax >> bits) != 0) ++bits;
  for (int shift = 0; shift < bits && e == cudaSuccess; shift += 8) {
    sort_hist_kernel<<<tiles, kSortTile, 0, st>>>(k0, total, shift, hist, tiles);
    sort_rowscan_kernel<<<kRadix, 1024, 0, st>>>(hist, tiles, totals);
    sort_scatter_kernel<<<tiles, kSortTile, 0, st>>>(k0, v0, total, shift, hist, totals, tiles,
                                                      k1, v1);
    e = cudaGetLastError();
    uint32_t* t = k0;
    k0 = k1;
    k1 = t;
    t = v0;
    v0 = v1;
    v1 = t;
  }
  if (e != cudaSuccess) return e;
  sort_segment_sum_kernel<<<(int)blocks, 256, 0, st>>>(I, k0, v0, total);
  return cudaGetLastError();
}

int sort_deposit_launches(int n) {
  const unsigned long long kmax = (unsigned long long)n * n - 1;
  int bits = 1;
  while (bits < 32 && (kmax >> bits) != 0) ++bits;
  return 2 + 3 * ((bits + 7) / 8);  // keys, passes x (hist, row scan, scatter), segment sums
}

}  // namespace aco
