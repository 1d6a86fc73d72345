// Tour construction (Section II, Eq. 1; data-parallel design of Section III-A).
//
// One group of threads builds one ant's tour: G whole warps (H = 32), or an
// H-lane segment of a warp (H = 8 or 16, G = 1), so that 32/H ants share
// every warp instruction.  Thread t of the group owns the contiguous cities
// [t*C, t*C + C) of every row: it reads them from the row staged in shared
// memory into registers, keeps their tabu bits (the paper's "1 = unvisited"
// integer per city, here one bit per city in registers) and takes part in the
// selection.  Each step:
//   1. one thread copies row choice[cur] into shared memory with the
//      bulk-copy engine; the group waits on an mbarrier and reads its chunks
//      (C floats per thread, conflict-free 16-byte loads); visited cities
//      are zeroed;
//   2. M = max over unvisited (max on the float bit patterns, which order
//      like the values for w >= 0), across warps through shared memory;
//   3. q_j = floor(w_j * 2^(45-ilogb M)) split exactly into two 23-bit halves
//      by three round-toward-zero FP32 FMAs (FP32 pipe; no float-to-int
//      conversion), per-thread u64 sums, warp inclusive scan, group totals
//      -> Q;
//   4. T = floor(r Q / 2^64) with r from Philox (one Philox call per lane per
//      H steps, broadcast by shuffle);
//   5. the thread whose prefix range holds T is found by ballot; it finds
//      the part of its chunk (up to four parts of whole 4-city groups, from
//      per-part sums kept in step 3) that holds the target, which is
//      rescanned by all lanes of its warp segment (about one city each); a
//      second scan and ballot give the city.
// Every operation is an exact max or an exact integer sum, so the chosen city
// is the same for every (C, G, H) tiling and equals the CPU oracle's choice.
// Every warp-level intrinsic names only the segment's lanes, so segments of
// one warp never wait on each other even when their control flow differs.
// After the last step the group computes C^k = sum of d over the tour and
// writes, for every city of the tour, its predecessor and successor into
// nbr[city][ant] (the bucketing used by the gather deposit).
#pragma once

#include "aco_device.cuh"

namespace aco {

struct GroupSmem {
  uint32_t wmax[4];
  unsigned long long wsum[4];
  long long wlen[4];
  int wmin[4];
  int next;
};

constexpr int kMaxGroupsPerCta = 8;

__device__ __forceinline__ void group_sync(int bar_id, int nthreads) {
  if (nthreads == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
  }
}

// Roulette weight bits: q_j = floor(w_j * 2^(kRouletteBits-1-ilogb M)).
constexpr int kRouletteBits = 46;
constexpr float kTwo23 = 8388608.0f;
constexpr uint32_t kTwo23Bits = 0x4b000000u;

// q = floor(w * 2^sc) < 2^46 as hi * 2^23 + lo, in three FP32 FMAs.
// With t = w * f1 (f1 = 2^(sc-23), so t < 2^23):
//   zh = fma.rz(w, f1, 2^23)           = 2^23 + floor(t)          (one rounding of w*f1 + 2^23)
//   c  = fma(zh, -2^23, 2^46 + 2^23)   = 2^23 - floor(t) * 2^23   (exact: representable)
//   zl = fma.rz(w, f1 * 2^23, c)       = 2^23 + floor(frac(t) * 2^23)
// zh and zl are floats in [2^23, 2^24) whose bit patterns are 0x4b000000 +
// hi and 0x4b000000 + lo.  Each rounding is of an exactly known value, so
// both floors are exact for every w >= 0 (subnormal products included: the
// fused multiply-add never rounds w * f1 on its own).
struct QuantParts {
  uint32_t hi_bits, lo_bits;
};

constexpr float kTwo46p23 = 70368752566272.0f;  // 2^46 + 2^23

__device__ __forceinline__ QuantParts quant_parts(uint32_t b, float f1, float f1s) {
  const float w = __uint_as_float(b);
  const float zh = __fmaf_rz(w, f1, kTwo23);
  const float c = __fmaf_rn(zh, -kTwo23, kTwo46p23);
  const float zl = __fmaf_rz(w, f1s, c);
  return QuantParts{__float_as_uint(zh), __float_as_uint(zl)};
}

// q of a weight that still needs the pre-scaling by f2 (see quant_factors).
__device__ __forceinline__ unsigned long long quant_value(uint32_t b, float f1, float f1s,
                                                          float f2) {
  if (f2 != 1.0f) b = __float_as_uint(__fmul_rn(__uint_as_float(b), f2));
  const QuantParts q = quant_parts(b, f1, f1s);
  return ((unsigned long long)(q.hi_bits - kTwo23Bits) << 23) + (q.lo_bits - kTwo23Bits);
}

// Factors for the step: f1 = 2^(sc-23) and f1s = f1 * 2^23 must both be
// normal floats, i.e. sc - 23 <= 104.  Beyond that (largest unvisited
// weight below 2^-82) the weights are first scaled up exactly by f2.
__device__ __forceinline__ void quant_factors(int sc, float& f1, float& f1s, float& f2) {
  const int e = sc - 23;
  if (e <= 104) {
    f1 = pow2f(e);
    f1s = pow2f(e + 23);
    f2 = 1.0f;
  } else {
    f1 = pow2f(104);
    f1s = pow2f(127);
    f2 = pow2f(e - 104);
  }
}

// Sum of q over the thread's C weights (already scaled by f2, see the
// caller).  The float bit patterns are summed modulo 2^32 (two per IADD3)
// and the C offsets of 0x4b000000 removed once; the true part sums are below
// C * 2^23 <= 2^30, so the wrap-around is exact.
template <int C>
__device__ __forceinline__ unsigned long long chunk_sum(const uint32_t (&v)[C], float f1,
                                                        float f1s) {
  uint32_t hi0 = 0, lo0 = 0, hi1 = 0, lo1 = 0;
#pragma unroll
  for (int i = 0; i < C; i += 4) {
    const QuantParts a = quant_parts(v[i], f1, f1s), b = quant_parts(v[i + 1], f1, f1s);
    const QuantParts c = quant_parts(v[i + 2], f1, f1s), d = quant_parts(v[i + 3], f1, f1s);
    hi0 += a.hi_bits + b.hi_bits;
    lo0 += a.lo_bits + b.lo_bits;
    hi1 += c.hi_bits + d.hi_bits;
    lo1 += c.lo_bits + d.lo_bits;
  }
  const uint32_t off = (uint32_t)C * kTwo23Bits;
  const uint32_t hi = hi0 + hi1 - off, lo = lo0 + lo1 - off;
  return ((unsigned long long)hi << 23) + lo;
}

// A lane's chunk split into K parts of whole 4-city groups: part k holds the
// groups [k*NG/K, (k+1)*NG/K), NG = C/4.  After the warp has found the lane
// whose range holds the target, that lane finds the part from these sums,
// and only the part's cities are searched city by city.
template <int C, int K>
struct ChunkParts {
  static constexpr int NG = C / 4;
  static_assert(K >= 1 && K <= NG, "1 <= K <= C/4 parts");
  __host__ __device__ static constexpr int first_group(int k) { return k * NG / K; }
  __host__ __device__ static constexpr int cities(int k) {
    return 4 * (first_group(k + 1) - first_group(k));
  }
  static constexpr int max_cities() { return 4 * ((NG + K - 1) / K); }
};

// Per-part sums of q over the thread's C weights (already scaled by f2),
// as hi/lo bit-pattern sums with their offsets still in (removed by
// part_value).  Parts accumulate independently; a single part uses two
// chains so that the adds still overlap.
template <int C, int K>
__device__ __forceinline__ void chunk_sum_parts(const uint32_t (&v)[C], float f1, float f1s,
                                                uint32_t (&phi)[K], uint32_t (&plo)[K]) {
  using Pt = ChunkParts<C, K>;
  uint32_t hi2 = 0, lo2 = 0;  // second chain of a single part
#pragma unroll
  for (int k = 0; k < K; ++k) {
    phi[k] = 0;
    plo[k] = 0;
  }
#pragma unroll
  for (int g = 0; g < C / 4; ++g) {
    int k = 0;
#pragma unroll
    for (int j = 1; j < K; ++j)
      if (g >= Pt::first_group(j)) k = j;
    const QuantParts a = quant_parts(v[4 * g], f1, f1s), b = quant_parts(v[4 * g + 1], f1, f1s);
    const QuantParts c = quant_parts(v[4 * g + 2], f1, f1s),
                     d = quant_parts(v[4 * g + 3], f1, f1s);
    if (K == 1 && (g & 1)) {
      hi2 += a.hi_bits + b.hi_bits;
      lo2 += a.lo_bits + b.lo_bits;
      hi2 += c.hi_bits + d.hi_bits;
      lo2 += c.lo_bits + d.lo_bits;
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j == k) {
          phi[j] += a.hi_bits + b.hi_bits;
          plo[j] += a.lo_bits + b.lo_bits;
          phi[j] += c.hi_bits + d.hi_bits;
          plo[j] += c.lo_bits + d.lo_bits;
        }
    }
  }
  if (K == 1) {
    phi[0] += hi2;
    plo[0] += lo2;
  }
}

// The value of part k's sum: its bit-pattern sums minus the offsets of its
// cities; the true sums are below C * 2^23 <= 2^30, so the modular sums are
// exact.  k must be a compile-time constant (an unrolled loop index).
template <int C, int K>
__device__ __forceinline__ unsigned long long part_value(const uint32_t (&phi)[K],
                                                         const uint32_t (&plo)[K], int k) {
  const uint32_t off = (uint32_t)ChunkParts<C, K>::cities(k) * kTwo23Bits;
  return ((unsigned long long)(phi[k] - off) << 23) + (plo[k] - off);
}

// Same sum, also keeping each group of four weights' hi/lo part sums (with
// their 4 * 0x4b000000 offsets) for the in-lane search of the selected city.
template <int C>
__device__ __forceinline__ unsigned long long chunk_sum_groups(const uint32_t (&v)[C], float f1,
                                                               float f1s, uint32_t (&ghi)[C / 4],
                                                               uint32_t (&glo)[C / 4]) {
  uint32_t hi = 0, lo = 0;
#pragma unroll
  for (int g = 0; g < C / 4; ++g) {
    const QuantParts a = quant_parts(v[4 * g], f1, f1s), b = quant_parts(v[4 * g + 1], f1, f1s);
    const QuantParts c = quant_parts(v[4 * g + 2], f1, f1s),
                     d = quant_parts(v[4 * g + 3], f1, f1s);
    ghi[g] = a.hi_bits + b.hi_bits + c.hi_bits + d.hi_bits;
    glo[g] = a.lo_bits + b.lo_bits + c.lo_bits + d.lo_bits;
    hi += ghi[g];
    lo += glo[g];
  }
  const uint32_t off = (uint32_t)C * kTwo23Bits;
  return ((unsigned long long)(hi - off) << 23) + (lo - off);
}

// The lanes of one warp segment (H = 32: the whole warp).
template <int H>
struct Seg {
  unsigned mask;
  int sub;  // segment index within the warp
  int hl;   // lane within the segment
  __device__ __forceinline__ explicit Seg(int lane)
      : mask(H == 32 ? FULL : (((1u << H) - 1u) << ((lane / H) * H))), sub(lane / H),
        hl(lane % H) {}
  template <typename T>
  __device__ __forceinline__ T shfl(T v, int src) const {
    return __shfl_sync(mask, v, src, H);
  }
  template <typename T>
  __device__ __forceinline__ T shfl_up(T v, int d) const {
    return __shfl_up_sync(mask, v, d, H);
  }
  template <typename T>
  __device__ __forceinline__ T shfl_xor(T v, int d) const {
    return __shfl_xor_sync(mask, v, d, H);
  }
  __device__ __forceinline__ uint32_t ballot(bool p) const {
    const uint32_t b = __ballot_sync(mask, p);
    return H == 32 ? b : (b >> (sub * H)) & ((1u << H) - 1u);
  }
  __device__ __forceinline__ uint32_t max_u32(uint32_t v) const {
    if constexpr (H == 32) {
      return __reduce_max_sync(FULL, v);
    } else {
#pragma unroll
      for (int o = H / 2; o > 0; o >>= 1) v = max(v, shfl_xor(v, o));
      return v;
    }
  }
  __device__ __forceinline__ uint32_t min_u32(uint32_t v) const {
    if constexpr (H == 32) {
      return __reduce_min_sync(FULL, v);
    } else {
#pragma unroll
      for (int o = H / 2; o > 0; o >>= 1) v = min(v, shfl_xor(v, o));
      return v;
    }
  }
  __device__ __forceinline__ unsigned long long inclusive_scan(unsigned long long x) const {
#pragma unroll
    for (int o = 1; o < H; o <<= 1) {
      const unsigned long long t = shfl_up(x, o);
      if (hl >= o) x += t;
    }
    return x;
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

// Cities per thread before and after the compactions of the Eq. 1 walk (see
// construct_phased.cuh): C, then 4*ceil(C/8), 4*ceil(C/16) and 4*ceil(C/32)
// (about C/2, C/4 and C/8 in whole 4-city groups), repeats dropped.  Adding
// 4*ceil(3C/16), or that and 4*ceil(3C/32), measured slower at every size:
// 0.2-2 % for one instance, 10 % for the batched step.  One warp (or
// segment) or two warps per ant with C >= kCompactMinC compact; four warps
// per ant never do.
constexpr int kCompactMinC = 20;
template <int C, int G>
struct Compaction {
  static constexpr bool kOn = (G == 1 || G == 2) && C >= kCompactMinC;
  // candidate count i: C * kSixteenths[i] / 16 rounded up to a multiple of 4
  __host__ __device__ static constexpr int raw(int i) {
    constexpr int kSixteenths[4] = {16, 8, 4, 2};
    return kSixteenths[i] == 16 ? C : 4 * ((kSixteenths[i] * C + 63) / 64);
  }
  // Slot count of phase j (0 = the direct phase, C), or 0 past the last.
  __host__ __device__ static constexpr int slots(int j) {
    int prev = 1 << 30, k = -1;
    for (int i = 0; i < 4; ++i) {
      const int v = raw(i);
      if (v > 0 && v < prev) {
        if (++k == j) return v;
        prev = v;
      }
    }
    return 0;
  }
};

// Shared memory of one ant group: the staged row (H*G*C floats, 16-byte
// aligned), its mbarrier, and (when the walk compacts) the list of unvisited
// cities, up to H * 4*ceil(C/8) 16-bit entries.
template <int C, int G, int H>
struct StageLayout {
  static constexpr int kRowFloats = H * G * C;
  static constexpr int kListOffset = kRowFloats * 4 + 16;
  // A float index beside the row (after the mbarrier, before the list) that
  // holds 0: the list entry of a visited slot of the walk with compaction.
  static constexpr int kZeroSlot = kRowFloats + 2;
  static constexpr int kListEntries = Compaction<C, G>::kOn ? H * G * Compaction<C, G>::slots(1) : 0;
  static constexpr int kBytes = ((kListOffset + 2 * kListEntries) + 15) / 16 * 16;
};

// Ant groups per CTA of `warps` warps.
template <int G, int H>
__host__ __device__ constexpr int groups_per_cta(int warps) {
  return H == 32 ? warps / G : warps * (32 / H);
}

// E = -ln(v 2^-24) for the candidate word x, v = floor(x / 2^8) + 1 in
// [1, 2^24], in single precision by the range-reduced inverse-hyperbolic-
// tangent series of the logarithm: v = 2^e f with f in [1, 2), halved when
// f > sqrt 2; s = (f - 1) / (f + 1); ln f = 2 s (1 + z/3 + z^2/5 + z^3/7 +
// z^4/9), z = s^2; E = (24 - e) ln 2 - ln f.  Every operation is rounded on
// its own (no contraction), so any IEEE implementation of the same sequence
// gives the same bits.  The constants are the floats nearest sqrt 2, ln 2,
// 1/3, 1/5, 1/7 and 1/9.
__device__ __forceinline__ float race_exponential(uint32_t x) {
  const uint32_t v = (x >> 8) + 1u;
  int e = 31 - __clz((int)v);
  // v 2^-e, exact: v < 2^25 is a float and 2^-e a normal power of two
  float f = __fmul_rn(__uint2float_rn(v), __uint_as_float((uint32_t)(127 - e) << 23));
  if (f > 0x1.6a09e6p+0f) {
    f = __fmul_rn(f, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float z = __fmul_rn(s, s);
  float p = 0x1.c71c72p-4f;
  p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);
  p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);
  p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);
  p = __fadd_rn(__fmul_rn(p, z), 1.0f);
  const float ln_f = __fmul_rn(__fadd_rn(s, s), p);
  return __fsub_rn(__fmul_rn(__int2float_rn(24 - e), 0x1.62e430p-1f), ln_f);
}

// R = 0: Eq. 1 by the integer roulette.  R = 1: the paper's data-parallel
// rule: every unvisited city scores u_j * w_j with its own uniform u_j, the
// highest score wins (ties to the lower index; all scores 0: the lowest
// unvisited city).  R = 2: the exponential race, which samples Eq. 1: every
// unvisited city gets the key E_j / w_j from its own exponential variate
// E_j, the smallest key wins (ties to the lower index; zero weights and
// overflowing keys are +inf, so with every weight 0 the lowest unvisited
// city wins).
// kPool: the ant belongs to a many-instance launch, where the GPU is full and
// issue-bound (fewer instructions per step pay even at a longer chain).
template <int C, int G, int H, int R = 0, bool kPool = false>
__device__ __forceinline__ void construct_ant(const Instance& I, const int ant, const int tg,
                                              const Seg<H> seg, GroupSmem* gs, const int bar_id,
                                              float* srow, const bool lane_copy) {
  static_assert(C % 4 == 0 && C >= 4 && C <= 128, "C must be a multiple of 4 in [4,128]");
  static_assert((C / 4) % 2 == 1, "C/4 must be odd: lanes then read their chunks from shared "
                                  "memory without bank conflicts");
  static_assert(G == 1 || G == 2 || G == 4, "G must be 1, 2 or 4");
  static_assert(H == 8 || H == 16 || H == 32, "H must be 8, 16 or 32");
  static_assert(H == 32 || G == 1, "segments smaller than a warp serve one ant each");
  constexpr int NW = (C + 31) / 32;  // tabu words per thread
  // The smallest chunk (4 cities) keeps its sums in registers and the
  // selected lane finds the city alone; larger chunks are rescanned by the
  // whole segment, which measured faster than a serial in-lane search.
  constexpr bool kGroupPick = C <= 4;
  constexpr int NG = kGroupPick ? C / 4 : 1;
  // Larger chunks keep per-part sums (K parts of whole 4-city groups) so the
  // rescan covers one part: at most about one city per lane.  This cuts the
  // instructions of a step but lengthens its dependent chain (the selected
  // lane picks the part first), so a single instance, whose ants may not
  // fill the GPU, splits only chunks of more than two cities per lane in the
  // rescan (measured: 2.8 % faster at C = 76, 2.4 % slower at C = 36).
  constexpr int KW = (C + H - 1) / H;  // cities per lane in an unsplit rescan
  constexpr int KP = (kGroupPick || (!kPool && KW <= 2)) ? 1 : (KW < 4 ? KW : 4);
  using Parts = ChunkParts<C, (KP < C / 4 ? KP : C / 4)>;
  constexpr int K = KP < C / 4 ? KP : C / 4;
  constexpr int PP = (Parts::max_cities() + H - 1) / H;  // cities per lane in the rescan
  constexpr int NT = H == 32 ? 32 * G : H;  // threads per ant
  const int n = I.n, ld = I.ld;
  const int hl = seg.hl;          // lane within the segment
  const int wg = H == 32 ? tg >> 5 : 0;  // warp within the group (G > 1)
  const int base = tg * C;
  const uint32_t iter = (uint32_t)I.st->iteration;
  const unsigned long long seed = I.seed;
  auto group_wait = [&]() {
    if (H == 32)
      group_sync(bar_id, NT);
    else
      seg.sync();
  };

  // Tabu bits: 1 = visited.  Padding cities (index >= n) and bits beyond C
  // start out visited.
  uint32_t vis[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int real = n - (base + 32 * w);  // local cities of word w below n
    uint32_t word = real <= 0 ? FULL : (real >= 32 ? 0u : (FULL << real));
    const int inchunk = C - 32 * w;
    if (inchunk < 32) word |= FULL << inchunk;
    vis[w] = word;
  }

  const Philox4 x0 = step_draw(seed, 0u, (uint32_t)ant, iter);
  const int start = (int)__umulhi(x0.x0, (uint32_t)n);
  {
    const int li = start - base;
    if (li >= 0 && li < C) {
#pragma unroll
      for (int w = 0; w < NW; ++w)
        if (w == (li >> 5)) vis[w] |= 1u << (li & 31);
    }
  }
  int32_t* tour = I.tours + (size_t)ant * I.ldt;
  const float* const choice = I.choice;
  if (tg == 0) tour[0] = start;
  int cur = start;
  unsigned long long rwin = 0;

  const uint32_t srow_a = smem_u32(srow);
  const uint32_t bar = srow_a + (uint32_t)StageLayout<C, G, H>::kRowFloats * 4u;
  const uint32_t row_bytes = (uint32_t)ld * 4u;
  uint32_t phase = 0;
  bool waits_ok = true;
  if (tg == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  group_wait();

  for (int s = 1; s < n; ++s) {
    // Everyone is done with the previous row (the group agreed on `cur`).
    if (lane_copy) {
      // The group copies the row with coalesced 16-byte loads (through L1,
      // so a row another group of this SM read recently may hit there).
      const float4* src = reinterpret_cast<const float4*>(choice + (size_t)cur * ld);
      float4* dst = reinterpret_cast<float4*>(srow);
      for (int i = tg; i < (ld >> 2); i += NT) dst[i] = src[i];
    } else if (tg == 0) {
      fence_proxy_async_smem();
      bulk_load(srow_a, choice + (size_t)cur * ld, row_bytes, bar);
    }
    const int off = (s - 1) % H;
    if (off == 0) {
      const Philox4 x = step_draw(seed, (uint32_t)(s + hl), (uint32_t)ant, iter);
      rwin = ((unsigned long long)x.x1 << 32) | x.x0;
    }
    const unsigned long long r = seg.shfl(rwin, off);
    if (lane_copy) {
      group_wait();
    } else {
      if (waits_ok && !mbar_wait_bounded(bar, phase)) {
        waits_ok = false;  // stale data from here on; the status word says so
        if (tg == 0) atomicOr(&I.st->status, kStatusTimeout);
      }
      phase ^= 1u;
    }
    const float* row = srow;

    // The race over long chunks reads its weights from the staged row as it
    // goes (a register copy of 60 or more weights beside its per-candidate
    // arithmetic measured slower); everything else works on a register copy.
    constexpr bool kRowRace = R == 2 && C >= 60;
    uint32_t v[C];  // weight bits; w >= 0 orders like its bit pattern
    uint32_t mx = 0u;
    if constexpr (!kRowRace) {
#pragma unroll
      for (int i = 0; i < C; i += 4) {
        // Chunk entries at or beyond ld hold stale data; their tabu bits are set.
        const uint4 t = *reinterpret_cast<const uint4*>(row + base + i);
        v[i] = t.x;
        v[i + 1] = t.y;
        v[i + 2] = t.z;
        v[i + 3] = t.w;
      }
    }
    if constexpr (R != 2) {
      uint32_t m4[4] = {0u, 0u, 0u, 0u};  // four independent max chains
#pragma unroll
      for (int i = 0; i < C; ++i) {
        if ((vis[i >> 5] >> (i & 31)) & 1u) v[i] = 0u;
        m4[i & 3] = max(m4[i & 3], v[i]);
      }
      mx = seg.max_u32(max(max(m4[0], m4[1]), max(m4[2], m4[3])));
      if (G > 1) {
        if (hl == 0) gs->wmax[wg] = mx;
        group_sync(bar_id, NT);
#pragma unroll
        for (int w = 0; w < G; ++w) mx = max(mx, gs->wmax[w]);
      }
    }

    int next;
    if constexpr (R == 1) {
      // Scores u_j * w_j; a thread's four consecutive cities share one
      // Philox call (C and base are multiples of 4).
      // Each thread walks its cities in ascending order and keeps the first
      // of its highest scores (bits of a non-negative float order like its
      // value; 0 = no positive score); the segment reduction breaks ties by
      // index.
      uint32_t bs = 0u, bj = 0xffffffffu;
#pragma unroll
      for (int i = 0; i < C; i += 4) {
        const Philox4 x = philox4x32_10((uint32_t)s, (uint32_t)ant, iter,
                                        1u + (uint32_t)((base + i) >> 2), (uint32_t)seed,
                                        (uint32_t)(seed >> 32));
        const uint32_t xs[4] = {x.x0, x.x1, x.x2, x.x3};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t sb = __float_as_uint(
              __fmul_rn(candidate_uniform_of(xs[e]), __uint_as_float(v[i + e])));
          if (sb > bs) {
            bs = sb;
            bj = (uint32_t)(base + i + e);
          }
        }
      }
#pragma unroll
      for (int o = H / 2; o > 0; o >>= 1) {
        const uint32_t os = seg.shfl_xor(bs, o), oj = seg.shfl_xor(bj, o);
        if (os > bs || (os == bs && oj < bj)) {
          bs = os;
          bj = oj;
        }
      }
      // (score bits << 32) | ~index: max = best score, lowest index
      uint64_t key = bs ? ((uint64_t)bs << 32) | (uint32_t)(0xffffffffu - bj) : 0ull;
      if (G > 1) {
        if (hl == 0) gs->wsum[wg] = key;
        group_sync(bar_id, NT);
#pragma unroll
        for (int w = 0; w < G; ++w) key = gs->wsum[w] > key ? gs->wsum[w] : key;
      }
      if (key != 0) mx = 1u;  // a positive score exists
      else mx = 0u;           // every score is 0: the rule below takes the lowest unvisited
      next = (int)(0xffffffffu - (uint32_t)key);
    }
    if constexpr (R == 2) {
      // Keys are non-negative floats (their bits order like their values);
      // a visited city keeps the sentinel above every key.  A thread's four
      // consecutive cities share one Philox call, and each thread walks its
      // cities in ascending order keeping the first smallest key.
      uint32_t bkey = 0xffffffffu, bj = 0xffffffffu;
#pragma unroll
      for (int i = 0; i < C; i += 4) {
        const Philox4 x = philox4x32_10((uint32_t)s, (uint32_t)ant, iter,
                                        1u + (uint32_t)((base + i) >> 2), (uint32_t)seed,
                                        (uint32_t)(seed >> 32));
        const uint32_t xs[4] = {x.x0, x.x1, x.x2, x.x3};
        uint32_t wv[4];
        if constexpr (kRowRace) {
          const uint4 t = *reinterpret_cast<const uint4*>(row + base + i);
          wv[0] = t.x;
          wv[1] = t.y;
          wv[2] = t.z;
          wv[3] = t.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) wv[e] = v[i + e];
        }
        // the four tabu bits of these cities (i % 4 == 0: one word)
        const uint32_t vis4 = vis[i >> 5] >> (i & 31);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int li = i + e;
          const float w = __uint_as_float(wv[e]);
          const bool open = !((vis4 >> e) & 1u);
          // visited cities skip the logarithm and the division
          const float key = open && w > 0.0f ? __fdiv_rn(race_exponential(xs[e]), w)
                                             : __uint_as_float(0x7f800000u);
          const uint32_t kb = __float_as_uint(key);
          if (open && kb < bkey) {
            bkey = kb;
            bj = (uint32_t)(base + li);
          }
        }
      }
      uint64_t key = ((uint64_t)bkey << 32) | bj;
#pragma unroll
      for (int o = H / 2; o > 0; o >>= 1) {
        const uint64_t other = seg.shfl_xor(key, o);
        key = other < key ? other : key;
      }
      if (G > 1) {
        if (hl == 0) gs->wsum[wg] = key;
        group_sync(bar_id, NT);
#pragma unroll
        for (int w = 0; w < G; ++w) key = gs->wsum[w] < key ? gs->wsum[w] : key;
      }
      next = (int)(uint32_t)key;
    }
    if ((R == 1 && mx != 0u) || R == 2) {
      // chosen above
    } else if (mx == 0u) {
      // Every unvisited weight is zero: the lowest-index unvisited city.
      uint32_t cand = 0xffffffffu;
#pragma unroll
      for (int w = NW - 1; w >= 0; --w) {
        const uint32_t fr = ~vis[w];
        if (fr) cand = (uint32_t)(base + 32 * w + __ffs(fr) - 1);
      }
      cand = seg.min_u32(cand);
      if (G > 1) {
        if (hl == 0) gs->wmin[wg] = (int)cand;
        group_sync(bar_id, NT);
#pragma unroll
        for (int w = 0; w < G; ++w) cand = min(cand, (uint32_t)gs->wmin[w]);
      }
      next = (int)cand;
    } else if constexpr (R == 0) {
      const int sc = kRouletteBits - 1 - exponent_of_bits(mx);
      float f1, f1s, f2;
      quant_factors(sc, f1, f1s, f2);
      if (f2 != 1.0f) {
        // Largest unvisited weight below 2^-82 (rare): scale the chunk up
        // first, exactly (quant_value() does the same for reloaded weights).
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = __float_as_uint(__fmul_rn(__uint_as_float(v[i]), f2));
      }
      uint32_t ghi[NG], glo[NG];
      uint32_t phi[K], plo[K];
      unsigned long long mine;
      if constexpr (kGroupPick) {
        mine = chunk_sum_groups<C>(v, f1, f1s, ghi, glo);
      } else {
        chunk_sum_parts<C, K>(v, f1, f1s, phi, plo);
        uint32_t hs = phi[0], ls = plo[0];
#pragma unroll
        for (int k = 1; k < K; ++k) {
          hs += phi[k];
          ls += plo[k];
        }
        const uint32_t off = (uint32_t)C * kTwo23Bits;
        mine = ((unsigned long long)(hs - off) << 23) + (ls - off);
      }
      const unsigned long long incl = seg.inclusive_scan(mine);
      const unsigned long long wtot = seg.shfl(incl, H - 1);
      unsigned long long woff = 0, Q = wtot;
      if (G > 1) {
        if (hl == 0) gs->wsum[wg] = wtot;
        group_sync(bar_id, NT);
        Q = 0;
#pragma unroll
        for (int w = 0; w < G; ++w) {
          const unsigned long long u = gs->wsum[w];
          if (w < wg) woff += u;
          Q += u;
        }
      }
      const unsigned long long T = __umul64hi(r, Q);
      next = 0;
      if (G == 1 || (T >= woff && T - woff < wtot)) {
        const unsigned long long t1 = T - woff;
        const int L = max(__ffs(seg.ballot(incl > t1)) - 1, 0);
        const unsigned long long t2 = t1 - seg.shfl(incl - mine, L);
        const int baseL = (wg * H + L) * C;  // within the staged row
        if constexpr (kGroupPick) {
          // Lane L walks its group sums, then the four cities of the group
          // holding the target (all from registers).
          int pick = 0;
          if (hl == L) {
            unsigned long long cum = 0;
            bool found = false;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              const unsigned long long gv =
                  ((unsigned long long)(ghi[g] - 4u * kTwo23Bits) << 23) + (glo[g] - 4u * kTwo23Bits);
              if (!found && cum + gv > t2) {
                found = true;
                unsigned long long c = cum + quant_value(v[4 * g], f1, f1s, 1.0f);
                int e = 0;
                if (c <= t2) {
                  c += quant_value(v[4 * g + 1], f1, f1s, 1.0f);
                  e = 1;
                  if (c <= t2) {
                    c += quant_value(v[4 * g + 2], f1, f1s, 1.0f);
                    e = c <= t2 ? 3 : 2;
                  }
                }
                pick = 4 * g + e;
              }
              cum += gv;
            }
          }
          next = baseL + seg.shfl(pick, L);
        } else {
          // Lane L finds the part of its chunk that holds the target.
          int part = 0;
          unsigned long long t3 = t2;
          if constexpr (K > 1) {
            if (hl == L) {
              unsigned long long cum = 0;
              bool found = false;
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const unsigned long long pv = part_value<C, K>(phi, plo, k);
                if (!found && (k == K - 1 || cum + pv > t2)) {
                  found = true;
                  part = k;
                  t3 = t2 - cum;
                }
                cum += pv;
              }
            }
            part = seg.shfl(part, L);
            t3 = seg.shfl(t3, L);
          }
          // The segment rescans that part, PP cities per lane.
          const int pstart = 4 * (part * Parts::NG / K);
          const int psz = 4 * ((part + 1) * Parts::NG / K) - pstart;
          uint32_t visL[NW];
#pragma unroll
          for (int w = 0; w < NW; ++w) visL[w] = seg.shfl(vis[w], L);
          unsigned long long qv[PP];
          unsigned long long ps = 0;
#pragma unroll
          for (int p = 0; p < PP; ++p) {
            const int pi = hl * PP + p;  // position within the part
            const int li = pstart + pi;  // position within lane L's chunk
            uint32_t word = FULL;
#pragma unroll
            for (int w = 0; w < NW; ++w)
              if (w == (li >> 5)) word = visL[w];
            uint32_t w8 = 0u;
            if (pi < psz && baseL + li < ld && !((word >> (li & 31)) & 1u))
              w8 = __float_as_uint(row[baseL + li]);
            qv[p] = quant_value(w8, f1, f1s, f2);
            ps += qv[p];
          }
          const unsigned long long incl2 = seg.inclusive_scan(ps);
          const int L2 = max(__ffs(seg.ballot(incl2 > t3)) - 1, 0);
          int pick = 0;
          if constexpr (PP > 1) {
            if (hl == L2) {
              unsigned long long c = incl2 - ps;
              pick = -1;
#pragma unroll
              for (int p = 0; p < PP; ++p) {
                c += qv[p];
                if (pick < 0 && c > t3) pick = p;
              }
            }
            pick = max(seg.shfl(pick, L2), 0);
          }
          next = baseL + pstart + L2 * PP + pick;
        }
        if (G > 1 && hl == 0) gs->next = next;
      }
      if (G > 1) {
        group_sync(bar_id, NT);
        next = gs->next;
      }
    }

    // A city outside [0, n) can only come from a defect; record it and stay
    // in bounds instead of reading past the matrix.
    if ((unsigned)next >= (unsigned)n) {
      if (tg == 0) atomicOr(&I.st->status, kStatusBadTour);
      next = start;
    }
    const int li = next - base;
    if (li >= 0 && li < C) {
#pragma unroll
      for (int w = 0; w < NW; ++w)
        if (w == (li >> 5)) vis[w] |= 1u << (li & 31);
    }
    if (tg == 0) tour[s] = next;
    cur = next;
    group_wait();
  }
  if (tg == 0) tour[n] = start;
  group_wait();

  // C^k (Section II) and the per-city neighbour buckets.
  long long len = 0;
  for (int s = tg; s < n; s += NT) {
    const int a = tour[s], b = tour[s + 1];
    const int p = tour[s == 0 ? n - 1 : s - 1];
    len += I.dist[(size_t)a * ld + b];
    I.nbr[(size_t)a * I.ldm + ant] = ((uint32_t)p << 16) | (uint32_t)b;
  }
#pragma unroll
  for (int o = H / 2; o > 0; o >>= 1) len += seg.shfl_xor(len, o);
  if (G > 1) {
    if (hl == 0) gs->wlen[wg] = len;
    group_sync(bar_id, NT);
    len = 0;
#pragma unroll
    for (int w = 0; w < G; ++w) len += gs->wlen[w];
  }
  if (tg == 0) I.lens[ant] = len;
}

}  // namespace aco

#include "construct_phased.cuh"

namespace aco {

// Placement of one thread: its ant group within the CTA and its index tg
// within the group.
template <int G, int H>
__device__ __forceinline__ void group_of_thread(int& grp, int& tg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (H == 32) {
    grp = threadIdx.x / (32 * G);
    tg = threadIdx.x % (32 * G);
  } else {
    grp = warp * (32 / H) + lane / H;
    tg = lane % H;
  }
}

// One CTA holds groups_per_cta<G, H>(blockDim.x / 32) ant groups; dynamic
// shared memory holds one StageLayout<C, G, H> per group.
template <int C, int G, int H, int R = 0>
__global__ void __launch_bounds__(256) construct_kernel(Instance I) {
  __shared__ GroupSmem gs[kMaxGroupsPerCta];
  extern __shared__ __align__(16) unsigned char stage[];
  int grp, tg;
  group_of_thread<G, H>(grp, tg);
  const int ant = blockIdx.x * groups_per_cta<G, H>(blockDim.x >> 5) + grp;
  if (ant >= I.m) return;
  float* srow = reinterpret_cast<float*>(stage + grp * StageLayout<C, G, H>::kBytes);
  construct_ant<C, G, H, R>(I, ant, tg, Seg<H>(threadIdx.x & 31), &gs[H == 32 ? grp : 0], 1 + grp,
                            srow, I.stage != 0);
}

// Batched form: group g of block b builds ant items[b*A + g].y of instance
// insts[items[b*A + g].x].  Items are listed longest instance first.  The
// row staging is chosen per launch (`lane_copy`), not per instance.
template <int C, int G, int H>
__global__ void __launch_bounds__(256) construct_items_kernel(const Instance* __restrict__ insts,
                                                              const int2* __restrict__ items,
                                                              int count, int lane_copy) {
  __shared__ GroupSmem gs[kMaxGroupsPerCta];
  extern __shared__ __align__(16) unsigned char stage[];
  int grp, tg;
  group_of_thread<G, H>(grp, tg);
  const int idx = blockIdx.x * groups_per_cta<G, H>(blockDim.x >> 5) + grp;
  if (idx >= count) return;
  const int2 it = items[idx];
  // A reference into the descriptor table (read-only, L1-cached) rather than
  // a register copy of the whole descriptor, which cost ~40 registers.
  const Instance& I = insts[it.x];
  float* srow = reinterpret_cast<float*>(stage + grp * StageLayout<C, G, H>::kBytes);
  construct_ant<C, G, H, 0, true>(I, it.y, tg, Seg<H>(threadIdx.x & 31), &gs[H == 32 ? grp : 0],
                                  1 + grp, srow, lane_copy != 0);
}

// The Eq. 1 walk with compaction (construct_phased.cuh), one group of H lanes
// (or two warps) per ant.  Its phases are inlined into one body; without a
// ceiling the register allocator adds their needs up instead of sharing them
// (233 registers at C = 76, where phase 0 alone needs 128).  The ceilings were
// chosen by measurement on the GB300: 128 from C = 44 (no spills); 72 at
// C = 36 (no spills; the batched step 0.9 % faster than at 80, one instance
// of n = 1002 the same); 64 up to C = 28 (the batched step 22.38 ms against
// 22.91 ms at 80; 56 spills and was 2.5 % slower).
template <int C>
struct PhasedRegs {
  static constexpr int v = C <= 28 ? 64 : (C <= 36 ? 72 : 128);
};

template <int C, int G, int H>
__global__ void __maxnreg__((PhasedRegs<C>::v)) construct_phased_kernel(Instance I) {
  __shared__ GroupSmem gs[kMaxGroupsPerCta];
  extern __shared__ __align__(16) unsigned char stage[];
  int grp, tg;
  group_of_thread<G, H>(grp, tg);
  const int ant = blockIdx.x * groups_per_cta<G, H>(blockDim.x >> 5) + grp;
  if (ant >= I.m) return;
  construct_ant_phased<C, G, H, false>(
      I, ant, tg, Seg<H>(threadIdx.x & 31), &gs[H == 32 ? grp : 0], 1 + grp,
      reinterpret_cast<float*>(stage + grp * StageLayout<C, G, H>::kBytes), I.stage != 0);
}

template <int C, int G, int H>
__global__ void __maxnreg__((PhasedRegs<C>::v))
    construct_phased_items_kernel(const Instance* __restrict__ insts,
                                  const int2* __restrict__ items, int count, int lane_copy) {
  __shared__ GroupSmem gs[kMaxGroupsPerCta];
  extern __shared__ __align__(16) unsigned char stage[];
  int grp, tg;
  group_of_thread<G, H>(grp, tg);
  const int idx = blockIdx.x * groups_per_cta<G, H>(blockDim.x >> 5) + grp;
  if (idx >= count) return;
  const int2 it = items[idx];
  construct_ant_phased<C, G, H, true>(
      insts[it.x], it.y, tg, Seg<H>(threadIdx.x & 31), &gs[H == 32 ? grp : 0], 1 + grp,
      reinterpret_cast<float*>(stage + grp * StageLayout<C, G, H>::kBytes), lane_copy != 0);
}

// Dynamic shared memory for a CTA of `warps` warps, with the opt-in above
// 48 KB set once per kernel and device.
template <int C, int G, int H, bool kItems, int R = 0>
inline size_t construct_smem_setup(int warps) {
  const size_t bytes = (size_t)groups_per_cta<G, H>(warps) * StageLayout<C, G, H>::kBytes;
  static std::atomic<unsigned long long> done{0};
  once_per_device(done, [] {
    const int most = groups_per_cta<G, H>(8) * StageLayout<C, G, H>::kBytes;
    constexpr bool kPhased = R == 0 && Compaction<C, G>::kOn;
    if constexpr (kItems && kPhased)
      return cudaFuncSetAttribute(construct_phased_items_kernel<C, G, H>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    else if constexpr (kItems)
      return cudaFuncSetAttribute(construct_items_kernel<C, G, H>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    else if constexpr (kPhased)
      return cudaFuncSetAttribute(construct_phased_kernel<C, G, H>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    else
      return cudaFuncSetAttribute(construct_kernel<C, G, H, R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  });
  return bytes;
}

}  // namespace aco
