// Ant Colony System (Dorigo and Gambardella, IEEE Trans. Evol. Comp. 1(1),
// 1997), the ACO variant the paper names as its next target (Section V), on
// the same data layout as the Ant System:
//  - the pseudo-random proportional rule: at step s ant k draws Philox
//    (s, k, iteration, 0); it exploits when word x2 < floor(q0 2^32), taking
//    the unvisited city of largest choice_info (ties to the lower index), and
//    otherwise samples Eq. 1 by the exact integer roulette;
//  - the local update: the ants move in lockstep, all choosing their s-th
//    city from the same state; then every edge crossed at that step gets
//    tau <- fl(fl((1-xi) tau) + fl(xi tau0)) once per ant that crossed it,
//    in both directions, with its choice_info; the closing edge is the n-th
//    such step;
//  - the global update: only the best-so-far tour's edges get
//    tau <- fl(fl((1-rho) tau) + fl(rho dtau)), dtau = 1/C_bs.
// The colony (m <= 32 ants, the variant's usual m = 10) runs in one CTA, one
// warp per ant, so the per-step lockstep is a CTA barrier; many colonies (a
// pool's Ant Colony System slots) run as one launch of one CTA per colony.
#include "aco_device.cuh"
#include "construct.cuh"
#include "kernels.h"

namespace aco {

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long w = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += w;
  }
  return v;
}

// One local update of one cell.
__device__ __forceinline__ float acs_local(float tau, float keep, float add) {
  return __fadd_rn(__fmul_rn(keep, tau), add);
}

// One colony in one CTA.  Warp k < m builds ant k's tour; further warps (a
// launch over colonies with different m sizes the CTA for the largest) take
// part in the lockstep barriers only.  kNN: with the instance's
// nearest-neighbour lists (I.nn entries): lane l holds entry l of the
// current city's list and its current choice_info value.
template <bool kNN>
__device__ __forceinline__ void acs_construct_body(const Instance& I, uint32_t* acs_seen,
                                                   uint32_t* s_edge) {
  const int n = I.n, ld = I.ld, m = I.m;
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool active = k < m;
  const int words = (n + 31) >> 5;
  uint32_t* seen = acs_seen + (size_t)k * words;
  const uint32_t it = (uint32_t)I.st->iteration;
  const float tau0 = I.st->acs_tau0;
  const float keep = __fsub_rn(1.0f, I.acs_xi), add = __fmul_rn(I.acs_xi, tau0);
  int32_t* tour = I.tours + (size_t)k * I.ldt;

  int start = 0;
  if (active) {
    for (int w = lane; w < words; w += 32) seen[w] = 0u;
    __syncwarp();
    const Philox4 x0 = step_draw(I.seed, 0u, (uint32_t)k, it);
    start = (int)__umulhi(x0.x0, (uint32_t)n);
    if (lane == 0) {
      seen[start >> 5] |= 1u << (start & 31);
      tour[0] = start;
    }
    __syncwarp();
  }
  int cur = start;
  for (int s = 1; s <= n; ++s) {
    int next = start;
    bool listed = false;  // chosen among the list entries
    if constexpr (kNN) {
      if (active && s < n) {
        const Philox4 x = step_draw(I.seed, (uint32_t)s, (uint32_t)k, it);
        const float* row = I.choice + (size_t)cur * ld;
        int j = 0;
        uint32_t wb = 0u;
        bool unv = false;
        if (lane < I.nn) {
          j = I.nnlist[(size_t)cur * kNnStride + lane];
          wb = __float_as_uint(row[j]);  // after this colony's local updates
          unv = !((seen[j >> 5] >> (j & 31)) & 1u);
        }
        const unsigned any = __ballot_sync(FULL, unv);
        if (any) {
          listed = true;
          if ((unsigned long long)x.x2 < I.acs_threshold) {
            // the heaviest unvisited entry, ties to the earlier entry
            const uint32_t key = unv ? wb + 1u : 0u;
            const uint32_t top = __reduce_max_sync(FULL, key);
            next = __shfl_sync(FULL, j, __ffs(__ballot_sync(FULL, key == top)) - 1);
          } else {
            // Eq. 1 over the unvisited entries, in list order
            const uint32_t wm = unv ? wb : 0u;
            const uint32_t mx = __reduce_max_sync(FULL, wm);
            if (mx == 0u) {
              next = __shfl_sync(FULL, j, __ffs(any) - 1);
            } else {
              float f1, f1s, f2;
              quant_factors(kRouletteBits - 1 - exponent_of_bits(mx), f1, f1s, f2);
              const unsigned long long incl =
                  warp_incl_scan_u64(quant_value(wm, f1, f1s, f2), lane);
              const unsigned long long r = ((unsigned long long)x.x1 << 32) | x.x0;
              const unsigned long long T = __umul64hi(r, __shfl_sync(FULL, incl, 31));
              next = __shfl_sync(FULL, j, max(__ffs(__ballot_sync(FULL, incl > T)) - 1, 0));
            }
          }
        }
      }
    }
    if (active && s < n && !listed) {
      const Philox4 x = step_draw(I.seed, (uint32_t)s, (uint32_t)k, it);
      const float* row = I.choice + (size_t)cur * ld;
      // Lane l reads cities 4l..4l+3 of every 128 with one 16-byte load (ld
      // is a multiple of 4, so the load stays inside the row); the three
      // passes read the same lines, the later two from L1.  Loads after the
      // CTA barrier see the local updates of the previous step.
      // Pass 1: the largest unvisited weight, ties to the lower index.  The
      // bits of non-negative floats order like their values; an unvisited
      // city's key is bits(w) + 1 and a visited one's 0, so a zero weight
      // still beats every visited city.  Each lane visits its cities in
      // ascending order and keeps the first of its largest keys; the warp
      // reduction breaks ties by index.
      uint32_t bkey = 0u;
      int bj = 0;
#pragma unroll 4
      for (int j0 = 4 * lane; j0 < n; j0 += 128) {
        const uint4 w4 = *reinterpret_cast<const uint4*>(row + j0);
        const uint32_t fr = ~seen[j0 >> 5] >> (j0 & 31);  // 4 free bits (j0 % 4 == 0)
        const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t kk = ((fr >> e) & 1u) && j0 + e < n ? wv[e] + 1u : 0u;
          if (kk > bkey) {
            bkey = kk;
            bj = j0 + e;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint32_t ok = __shfl_xor_sync(FULL, bkey, o);
        const int oj = __shfl_xor_sync(FULL, bj, o);
        if (ok > bkey || (ok == bkey && oj < bj)) {
          bkey = ok;
          bj = oj;
        }
      }
      const uint32_t mbits = bkey - 1u;  // bkey >= 1: a city is unvisited
      next = bj;
      // with lists, every entry is visited here: the heaviest city, always
      const bool exploit = kNN || (unsigned long long)x.x2 < I.acs_threshold;
      if (!exploit && mbits != 0u) {
        // Eq. 1 by the integer roulette: q_j = floor(w_j 2^(45 - ilogb M)),
        // T = floor(r Q / 2^64), the first j whose prefix sum exceeds T.
        // (the three-FMA quantiser of the construction kernel: exact, branch-free)
        float f1, f1s, f2;
        quant_factors(kRouletteBits - 1 - exponent_of_bits(mbits), f1, f1s, f2);
        unsigned long long part = 0ull;
#pragma unroll 4
        for (int j0 = 4 * lane; j0 < n; j0 += 128) {
          const uint4 w4 = *reinterpret_cast<const uint4*>(row + j0);
          const uint32_t fr = ~seen[j0 >> 5] >> (j0 & 31);
          const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            part += quant_value(((fr >> e) & 1u) && j0 + e < n ? wv[e] : 0u, f1, f1s, f2);
        }
        const unsigned long long Q = warp_sum_u64(part);
        const unsigned long long r = ((unsigned long long)x.x1 << 32) | x.x0;
        const unsigned long long T = __umul64hi(r, Q);
        // Pass 3: 256 cities at a time in ascending order, lane l holding
        // cities 8l..8l+7 of the chunk; a warp scan of the lanes' eight-city
        // sums finds the lane, the lane its city.
        unsigned long long running = 0ull;
        for (int c0 = 0; c0 < n; c0 += 256) {
          const int j0 = c0 + 8 * lane;
          unsigned long long q[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) q[e] = 0ull;
          if (j0 < n) {
            const uint32_t fr = ~seen[j0 >> 5] >> (j0 & 31);  // 8 free bits (j0 % 8 == 0)
            const uint4 wa = *reinterpret_cast<const uint4*>(row + j0);
            // the second half only if it starts inside the row (ld % 4 == 0)
            const uint4 wb = j0 + 4 < n ? *reinterpret_cast<const uint4*>(row + j0 + 4)
                                        : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
              q[e] = quant_value(((fr >> e) & 1u) && j0 + e < n ? wv[e] : 0u, f1, f1s, f2);
          }
          unsigned long long mine = 0ull;
#pragma unroll
          for (int e = 0; e < 8; ++e) mine += q[e];
          const unsigned long long incl = warp_incl_scan_u64(mine, lane);
          const unsigned long long total = __shfl_sync(FULL, incl, 31);
          if (running + total > T) {
            const unsigned hit = __ballot_sync(FULL, running + incl > T);
            const int L = __ffs(hit) - 1;
            int pick = 0;
            if (lane == L) {
              // the first e whose inclusive prefix exceeds T: count the
              // prefixes that do not
              unsigned long long c = running + incl - mine;
#pragma unroll
              for (int e = 0; e < 7; ++e) {
                c += q[e];
                pick += c <= T ? 1 : 0;
              }
            }
            next = c0 + 8 * L + __shfl_sync(FULL, pick, L);
            break;
          }
          running += total;
        }
      }
      if ((unsigned)next >= (unsigned)n) {  // cannot happen while a city is unvisited
        if (lane == 0) atomicOr(&I.st->status, kStatusBadTour);
        next = start;
      }
      // The next step reads row `next`: start bringing it into L1 now (one
      // 128-byte line per lane and round), while this ant waits at the
      // barrier for the others.  Only this CTA writes the colony's matrices,
      // through the same L1, so the lines the local updates change stay
      // current; the prefetch is a hint and changes no result.
      if (s + 1 < n) {
        const float* nrow = I.choice + (size_t)next * ld;
        for (int f = 32 * lane; f < n; f += 32 * 32)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(nrow + f));
      }
    }
    if constexpr (kNN) {
      if (active && s < n && (unsigned)next >= (unsigned)n) {  // cannot happen
        if (lane == 0) atomicOr(&I.st->status, kStatusBadTour);
        next = start;
      }
    }
    // lockstep: every ant has chosen from the same state; then the local
    // updates of this step, one writer per distinct edge applying it once
    // per ant that crossed the edge
    const uint32_t lo = (uint32_t)min(cur, next), hi = (uint32_t)max(cur, next);
    const size_t ab = (size_t)lo * ld + hi, ba = (size_t)hi * ld + lo;
    // The crossed cell's tau and eta^beta, read before the barrier: only this
    // step's writer of the edge stores to it, after the barrier, so the
    // values read here are the current ones and the load latency overlaps
    // the other ants' selection.
    float t = 0.0f, h = 0.0f;
    if (active && lane == 0) {
      s_edge[k] = (lo << 16) | hi;
      t = __ldcg(I.tau + ab);
      h = I.heta[ab];
    }
    __syncthreads();
    if (active) {
      const uint32_t e = s_edge[k];
      const unsigned same = __ballot_sync(FULL, lane < m && s_edge[lane < m ? lane : 0] == e);
      if (lane == 0 && __ffs(same) - 1 == k) {
        for (int c = __popc(same); c > 0; --c) t = acs_local(t, keep, add);
        const float ch = choice_of(t, h, I.alpha);
        I.tau[ab] = t;
        I.tau[ba] = t;
        I.choice[ab] = ch;
        I.choice[ba] = ch;
      }
      if (lane == 0 && s < n) {
        seen[next >> 5] |= 1u << (next & 31);
        tour[s] = next;
      }
    }
    __syncthreads();
    cur = next;
  }
  if (!active) return;
  if (lane == 0) tour[n] = start;
  __syncwarp();
  long long len = 0;
  for (int s = lane; s < n; s += 32) len += I.dist[(size_t)tour[s] * ld + tour[s + 1]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(FULL, len, o);
  if (lane == 0) I.lens[k] = len;
}

template <bool kNN>
__global__ void __launch_bounds__(1024, 1) acs_construct_kernel(Instance I) {
  extern __shared__ uint32_t acs_seen[];  // m tabu bitmaps of (n + 31) / 32 words
  __shared__ uint32_t s_edge[32];         // (min << 16 | max) crossed by ant k
  acs_construct_body<kNN>(I, acs_seen, s_edge);
}

// Many colonies per launch: CTA b runs the colony of slot slots[b] (all of
// them with lists, or all without).
template <bool kNN>
__global__ void __launch_bounds__(1024, 1)
    acs_construct_slots_kernel(const Instance* __restrict__ insts, const int* __restrict__ slots) {
  extern __shared__ uint32_t acs_seen[];
  __shared__ uint32_t s_edge[32];
  acs_construct_body<kNN>(insts[slots[blockIdx.x]], acs_seen, s_edge);
}

// Global update on the best-so-far tour: edge s of the tour per thread from
// `first` in steps of `stride` (each edge of a closed tour of n >= 3 cities
// occurs once).
__device__ __forceinline__ void acs_global_body(const Instance& I, int first, int stride,
                                                bool bump_iteration) {
  const int n = I.n, ld = I.ld;
  const float keep = __fsub_rn(1.0f, I.rho);
  const float dep = __fmul_rn(I.rho, (float)(1.0 / (double)I.st->best_len));
  for (int s = first; s < n; s += stride) {
    const int a = I.best_tour[s], b = I.best_tour[s + 1];
    const size_t ab = (size_t)a * ld + b, ba = (size_t)b * ld + a;
    const float t = __fadd_rn(__fmul_rn(keep, I.tau[ab]), dep);
    const float ch = choice_of(t, I.heta[ab], I.alpha);
    I.tau[ab] = t;
    I.tau[ba] = t;
    I.choice[ab] = ch;
    I.choice[ba] = ch;
  }
  if (bump_iteration) I.st->iteration += 1;
}

__global__ void acs_global_kernel(Instance I) {
  acs_global_body(I, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                  blockIdx.x == 0 && threadIdx.x == 0);
}

__global__ void acs_global_slots_kernel(const Instance* __restrict__ insts,
                                        const int* __restrict__ slots) {
  acs_global_body(insts[slots[blockIdx.x]], threadIdx.x, blockDim.x, threadIdx.x == 0);
}

// Start: tau = tau0 = (float)(1 / (n C_nn)) off the diagonal, choice_info.
__global__ void acs_init_kernel(Instance I) {
  const float tau0 = (float)(1.0 / ((double)I.n * (double)I.st->nn_len));
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)n * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    const float t = (j != i && j < n) ? tau0 : 0.0f;
    I.tau[e] = t;
    I.choice[e] = choice_of(t, I.heta[e], I.alpha);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) I.st->acs_tau0 = tau0;
}

cudaError_t launch_acs_init(const Instance& I, int sms, cudaStream_t st) {
  size_t blocks = ((size_t)I.n * I.ld + 255) / 256;
  if (blocks > (size_t)sms * 8) blocks = (size_t)sms * 8;
  acs_init_kernel<<<(int)blocks, 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_acs_construct(const Instance& I, cudaStream_t st) {
  if (I.m < 1 || I.m > kAcsMaxAnts) return cudaErrorInvalidValue;
  const size_t smem = (size_t)I.m * ((I.n + 31) / 32) * sizeof(uint32_t);
  if (I.nn > 0)
    acs_construct_kernel<true><<<1, 32 * I.m, smem, st>>>(I);
  else
    acs_construct_kernel<false><<<1, 32 * I.m, smem, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_acs_global(const Instance& I, cudaStream_t st) {
  acs_global_kernel<<<(I.n + 255) / 256, 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_acs_construct_slots(const Instance* insts, const int* slots, int count,
                                       int max_m, int max_n, bool lists, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (max_m < 1 || max_m > kAcsMaxAnts) return cudaErrorInvalidValue;
  const size_t smem = (size_t)max_m * ((max_n + 31) / 32) * sizeof(uint32_t);
  if (lists)
    acs_construct_slots_kernel<true><<<count, 32 * max_m, smem, st>>>(insts, slots);
  else
    acs_construct_slots_kernel<false><<<count, 32 * max_m, smem, st>>>(insts, slots);
  return cudaGetLastError();
}

cudaError_t launch_acs_global_slots(const Instance* insts, const int* slots, int count,
                                    cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  acs_global_slots_kernel<<<count, 256, 0, st>>>(insts, slots);
  return cudaGetLastError();
}

}  // namespace aco
