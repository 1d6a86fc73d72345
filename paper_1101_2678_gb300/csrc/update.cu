// Setup, iteration-best and pheromone-update kernels (Section II, Eqs. 2-4;
// Section III-B for the atomic and scatter-to-gather designs).
#include <climits>

#include "../../include/aco.h"

#include "aco_device.cuh"
#include "kernels.h"
#include "update.cuh"

namespace aco {

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------

// Nearest-neighbour tour from city 0 (ties to the lower index), C_nn and
// tau0 = m / C_nn.  One CTA of kNnTourThreads threads; thread t owns the
// cities 4t + 4*kNnTourThreads*r + e (e < 4), reads them with one 16-byte
// load per r and keeps their visited bits in a register.  Each step takes
// the minimum of the key (d << 32 | j) (lexicographic (d, j): ties to the
// lower index) over the unvisited cities: a warp butterfly, then the warps'
// minima through double-buffered shared memory, one barrier per step.
constexpr int kNnTourThreads = 256;
constexpr int kNnTourRounds = (ACO_MAX_N + 4 * kNnTourThreads - 1) / (4 * kNnTourThreads);

__global__ void __launch_bounds__(kNnTourThreads) nn_tour_kernel(Instance I) {
  __shared__ unsigned long long wmin[2][kNnTourThreads / 32];
  const int n = I.n, ld = I.ld;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int kWarps = kNnTourThreads / 32;
  uint32_t visited = 0;  // bit 4r + e: city 4t + 4*kNnTourThreads*r + e
#pragma unroll
  for (int r = 0; r < kNnTourRounds; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * t + 4 * kNnTourThreads * r + e;
      if (j >= n || j == 0) visited |= 1u << (4 * r + e);
    }
  int cur = 0;
  long long len = 0;
  for (int s = 1; s < n; ++s) {
    const int32_t* row = I.dist + (size_t)cur * ld;
    int4 d4[kNnTourRounds];
#pragma unroll
    for (int r = 0; r < kNnTourRounds; ++r) {
      const int j0 = 4 * t + 4 * kNnTourThreads * r;
      // ld is a multiple of 4, so a 16-byte load that starts below n ends below ld
      d4[r] = j0 < n ? *reinterpret_cast<const int4*>(row + j0) : make_int4(0, 0, 0, 0);
    }
    unsigned long long key = ~0ull;
#pragma unroll
    for (int r = 0; r < kNnTourRounds; ++r) {
      const int j0 = 4 * t + 4 * kNnTourThreads * r;
      const int dv[4] = {d4[r].x, d4[r].y, d4[r].z, d4[r].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const unsigned long long k =
            ((unsigned long long)(uint32_t)dv[e] << 32) | (uint32_t)(j0 + e);
        if (!((visited >> (4 * r + e)) & 1u) && k < key) key = k;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(FULL, key, o);
      key = other < key ? other : key;
    }
    if (lane == 0) wmin[s & 1][warp] = key;
    __syncthreads();
    key = wmin[s & 1][0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) {
      const unsigned long long other = wmin[s & 1][w];
      key = other < key ? other : key;
    }
    int next = (int)(uint32_t)key;
    if (key == ~0ull || next >= n) {  // cannot happen while a city is unvisited
      if (t == 0) atomicOr(&I.st->status, kStatusBadTour);
      next = 0;
    }
    const int rel = next - 4 * t;
    if (rel >= 0 && (rel % (4 * kNnTourThreads)) < 4)
      visited |= 1u << (4 * (rel / (4 * kNnTourThreads)) + (rel % (4 * kNnTourThreads)));
    len += (long long)(key >> 32);
    cur = next;
  }
  if (t == 0) {
    len += I.dist[(size_t)cur * ld];
    I.st->nn_len = len;
    I.st->tau0 = (float)((double)I.m / (double)len);
  }
}

// eta^beta (double, rounded once to float), tau = tau0 off the diagonal, and
// the first choice_info.  Padding columns stay zero.
__global__ void init_matrices_kernel(Instance I) {
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)n * ld;
  const float tau0 = I.st->tau0;
  const double beta = (double)I.beta;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    float h = 0.0f, t = 0.0f;
    if (j < n && j != i) {
      const double d = (double)I.dist[e];
      double v;
      if (beta == 0.0) v = 1.0;
      else if (beta == 1.0) v = 1.0 / d;
      else if (beta == 2.0) v = 1.0 / (d * d);
      else if (beta == 3.0) v = 1.0 / (d * d * d);
      else v = pow(d, -beta);
      h = (float)v;
      t = tau0;
    }
    I.heta[e] = h;
    I.tau[e] = t;
    I.choice[e] = (j < n && j != i) ? choice_of(t, h, I.alpha) : 0.0f;
  }
}

// choice_info from the current tau (no state change).
__global__ void choice_kernel(Instance I, int bump_iteration) {
  const size_t total = (size_t)I.n * I.ld;
  const float alpha = I.alpha;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    I.choice[e] = choice_of(I.tau[e], I.heta[e], alpha);
  if (bump_iteration && blockIdx.x == 0 && threadIdx.x == 0) I.st->iteration += 1;
}

// Iteration best, best-so-far and per-ant deposits: best_body() in update.cuh.
__global__ void best_kernel(Instance I) { best_body(I); }

// ---------------------------------------------------------------------------
// Pheromone update
// ---------------------------------------------------------------------------

// Gather deposit fused with evaporation and choice_info (gather_row() in
// update.cuh): one warp per row.
__global__ void update_gather_kernel(Instance I, int bump_iteration) {
  extern __shared__ unsigned long long acc_rows[];
  const int warps = blockDim.x >> 5;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * warps + wi;
  if (bump_iteration && blockIdx.x == 0 && threadIdx.x == 0) I.st->iteration += 1;
  if (i >= I.n) return;
  gather_row(I, i, acc_rows + (size_t)wi * I.ld, lane);
}

// Atomic deposit in 64-bit fixed point: one thread per tour edge (k, s) adds
// q_k to acc[a][b] and acc[b][a] with red.global.add.u64 (Fig. 2's design;
// integer addition commutes, so the result is deterministic).
__global__ void deposit_atomic_u64_kernel(Instance I) {
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)I.m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n), s = (int)(e % n);
    const int32_t* t = I.tours + (size_t)k * I.ldt;
    const int a = t[s], b = t[s + 1];
    const unsigned long long qk = I.q[k];
    atomicAdd(I.acc + (size_t)a * ld + b, qk);
    atomicAdd(I.acc + (size_t)b * ld + a, qk);
  }
}

// Evaporation + fixed-point deposit + choice_info, elementwise; clears acc.
__global__ void apply_acc_kernel(Instance I, int bump_iteration) {
  const size_t total4 = (size_t)I.n * I.ld / 4;
  const float keep = __fsub_rn(1.0f, I.rho);
  const float inv = inv_scale_of(I.st->deposit_shift);
  const float alpha = I.alpha;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total4;
       e += (size_t)gridDim.x * blockDim.x) {
    float4 t4 = reinterpret_cast<const float4*>(I.tau)[e];
    const float4 h4 = reinterpret_cast<const float4*>(I.heta)[e];
    ulonglong2* a2 = reinterpret_cast<ulonglong2*>(I.acc) + 2 * e;
    const ulonglong2 a01 = a2[0], a23 = a2[1];
    float4 c;
    t4.x = apply_deposit(t4.x, a01.x, keep, inv);
    t4.y = apply_deposit(t4.y, a01.y, keep, inv);
    t4.z = apply_deposit(t4.z, a23.x, keep, inv);
    t4.w = apply_deposit(t4.w, a23.y, keep, inv);
    c.x = choice_of(t4.x, h4.x, alpha);
    c.y = choice_of(t4.y, h4.y, alpha);
    c.z = choice_of(t4.z, h4.z, alpha);
    c.w = choice_of(t4.w, h4.w, alpha);
    reinterpret_cast<float4*>(I.tau)[e] = t4;
    reinterpret_cast<float4*>(I.choice)[e] = c;
    a2[0] = make_ulonglong2(0ull, 0ull);
    a2[1] = make_ulonglong2(0ull, 0ull);
  }
  if (bump_iteration && blockIdx.x == 0 && threadIdx.x == 0) I.st->iteration += 1;
}

// Symmetric form of the two kernels above (the paper's "Reduction" version,
// Section III-B: the symmetric TSP needs only half of the pheromone cells).
// The tour edge (a, b) adds q_k once, to acc[min(a,b)][max(a,b)]: half the
// atomics of the full form.  The apply pass then reads tau, eta^beta and acc
// only in the upper triangle and writes both halves of tau and choice_info.
// tau and eta^beta are symmetric bit for bit (the same arithmetic on the same
// operands in both halves), so the result equals the full form's exactly.
__global__ void deposit_symmetric_kernel(Instance I) {
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)I.m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n), s = (int)(e % n);
    const int32_t* t = I.tours + (size_t)k * I.ldt;
    const int a = t[s], b = t[s + 1];
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    atomicAdd(I.acc + (size_t)lo * ld + hi, I.q[k]);
  }
}

// One CTA of 32 x 8 threads per 32 x 32 tile (bi, bj), bi <= bj, of the upper
// triangle: each thread updates four cells (i, j), j > i, with coalesced
// row accesses, and the tile's new tau and choice_info go through shared
// memory to the mirrored tile (bj, bi), written with coalesced rows as well.
constexpr int kSymTile = 32;

__global__ void __launch_bounds__(256) apply_symmetric_kernel(Instance I, int bump_iteration) {
  __shared__ float tile_tau[kSymTile][kSymTile + 1];
  __shared__ float tile_ch[kSymTile][kSymTile + 1];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bump_iteration && bi == 0 && bj == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    I.st->iteration += 1;
  if (bi > bj) return;
  const int n = I.n, ld = I.ld;
  const float keep = __fsub_rn(1.0f, I.rho);
  const float inv = inv_scale_of(I.st->deposit_shift);
  const float alpha = I.alpha;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = bj * kSymTile + tx;
#pragma unroll
  for (int r = 0; r < kSymTile; r += 8) {
    const int i = bi * kSymTile + ty + r;
    if (i < n && j < n && j > i) {
      const size_t e = (size_t)i * ld + j;
      const float t = apply_deposit(I.tau[e], I.acc[e], keep, inv);
      const float c = choice_of(t, I.heta[e], alpha);
      I.tau[e] = t;
      I.choice[e] = c;
      I.acc[e] = 0ull;
      tile_tau[ty + r][tx] = t;
      tile_ch[ty + r][tx] = c;
    }
  }
  __syncthreads();
  const int jt = bi * kSymTile + tx;  // column of the mirrored tile
#pragma unroll
  for (int r = 0; r < kSymTile; r += 8) {
    const int it = bj * kSymTile + ty + r;  // row of the mirrored tile
    if (it < n && jt < n && jt < it) {
      const size_t e = (size_t)it * ld + jt;
      I.tau[e] = tile_tau[tx][ty + r];
      I.choice[e] = tile_ch[tx][ty + r];
    }
  }
}

// MAX-MIN Ant System update (the variant of Stutzle and Hoos, cited by the
// paper in Section II-B): tau' = clamp(fl(fl((1-rho) tau) + [ij on the
// depositing tour] dtau), tau_min, tau_max) off the diagonal, then
// choice_info; one streaming pass of 16-byte accesses.  Every city has
// exactly two neighbours on the depositing tour (dep_nb), so the deposit
// needs no atomics and no accumulator.
__global__ void mmas_update_kernel(Instance I, int bump_iteration) {
  const int n = I.n, ld = I.ld;
  const size_t total4 = (size_t)n * ld / 4;
  const float keep = __fsub_rn(1.0f, I.rho);
  const float dtau = I.st->mmas_dtau, lo = I.st->tau_min, hi = I.st->tau_max;
  const float alpha = I.alpha;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total4;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(4 * e / ld), j0 = (int)(4 * e % ld);
    const uint32_t nb = I.dep_nb[i];
    const int pred = (int)(nb >> 16), succ = (int)(nb & 0xffffu);
    float4 t4 = reinterpret_cast<const float4*>(I.tau)[e];
    const float4 h4 = reinterpret_cast<const float4*>(I.heta)[e];
    float tv[4] = {t4.x, t4.y, t4.z, t4.w};
    const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
    float cv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      tv[c] = mmas_cell(tv[c], i, j0 + c, n, pred, succ, keep, dtau, lo, hi);
      cv[c] = choice_of(tv[c], hv[c], alpha);
    }
    reinterpret_cast<float4*>(I.tau)[e] = make_float4(tv[0], tv[1], tv[2], tv[3]);
    reinterpret_cast<float4*>(I.choice)[e] = make_float4(cv[0], cv[1], cv[2], cv[3]);
  }
  if (bump_iteration && blockIdx.x == 0 && threadIdx.x == 0) I.st->iteration += 1;
}

// MAX-MIN Ant System start: tau = tau_max computed from C_nn off the
// diagonal, the limits stored, choice_info recomputed.
__global__ void mmas_init_kernel(Instance I) {
  float lo, hi;
  mmas_limits(I, I.st->nn_len, &lo, &hi);
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)n * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    const float t = (j != i && j < n) ? hi : 0.0f;
    I.tau[e] = t;
    I.choice[e] = choice_of(t, I.heta[e], I.alpha);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    I.st->tau_min = lo;
    I.st->tau_max = hi;
  }
}

// The paper's atomic kernel: evaporation first (Eq. 2) ...
__global__ void evaporate_kernel(Instance I) {
  const size_t total4 = (size_t)I.n * I.ld / 4;
  const float keep = __fsub_rn(1.0f, I.rho);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total4;
       e += (size_t)gridDim.x * blockDim.x) {
    float4 t4 = reinterpret_cast<const float4*>(I.tau)[e];
    t4.x = __fmul_rn(keep, t4.x);
    t4.y = __fmul_rn(keep, t4.y);
    t4.z = __fmul_rn(keep, t4.z);
    t4.w = __fmul_rn(keep, t4.w);
    reinterpret_cast<float4*>(I.tau)[e] = t4;
  }
}

// ... then red.global.add.f32 of dtau^k on both directions of every tour edge
// (Eqs. 3-4; the order of the float additions is not deterministic).
__global__ void deposit_atomic_f32_kernel(Instance I) {
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)I.m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n), s = (int)(e % n);
    const int32_t* t = I.tours + (size_t)k * I.ldt;
    const int a = t[s], b = t[s + 1];
    const float dk = I.delta[k];
    atomicAdd(I.tau + (size_t)a * ld + b, dk);
    atomicAdd(I.tau + (size_t)b * ld + a, dk);
  }
}

// ---------------------------------------------------------------------------
// Batched forms: one CTA (best) or one warp (update row) per list entry.
// ---------------------------------------------------------------------------
__global__ void best_slots_kernel(const Instance* __restrict__ insts, const int* __restrict__ slots,
                                  int count) {
  if ((int)blockIdx.x >= count) return;
  best_body(insts[slots[blockIdx.x]]);
}

__global__ void update_rows_kernel(const Instance* __restrict__ insts, const int2* __restrict__ rows,
                                   int count, int max_ld) {
  extern __shared__ unsigned long long acc_rows[];
  const int warps = blockDim.x >> 5;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * warps + wi;
  if (idx >= count) return;
  const int2 it = rows[idx];
  const Instance& I = insts[it.x];
  if (it.y == 0 && lane == 0) I.st->iteration += 1;
  if (I.variant == kVariantMmas)
    mmas_row(I, it.y, lane);
  else
    gather_row(I, it.y, acc_rows + (size_t)wi * max_ld, lane);
}

// Rounded Euclidean distances (TSPLIB EUC_2D): d = floor(sqrt(dx^2 + dy^2) +
// 0.5) in IEEE double (exact squares for |coordinates| <= 2^25), written into
// the instance's padded distance matrix.
__global__ void dist_from_coords_kernel(Instance I, const int32_t* __restrict__ xy) {
  const int n = I.n, ld = I.ld;
  const size_t total = (size_t)n * ld;
  int32_t* dist = const_cast<int32_t*>(I.dist);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    int32_t d = 0;
    if (j < n && j != i) {
      const double dx = (double)xy[2 * i] - (double)xy[2 * j];
      const double dy = (double)xy[2 * i + 1] - (double)xy[2 * j + 1];
      d = (int32_t)floor(__dsqrt_rn(dx * dx + dy * dy) + 0.5);
    }
    dist[e] = d;
  }
}

// Optional check of the constructed tours (ACO_OPT_CHECK): one warp per
// ant; every city must occur exactly once among tour[0..n), tour[n] must be
// tour[0], and the stored length must equal the sum of the distances.  The
// visited cities are counted in a shared-memory bitmap per warp.
__global__ void check_tours_kernel(Instance I) {
  extern __shared__ uint32_t check_bits[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * (blockDim.x >> 5) + warp;
  if (k >= I.m) return;
  const int n = I.n, ld = I.ld, words = (n + 31) >> 5;
  uint32_t* bits = check_bits + (size_t)warp * words;
  for (int w = lane; w < words; w += 32) bits[w] = 0u;
  __syncwarp();
  const int32_t* t = I.tours + (size_t)k * I.ldt;
  bool ok = true;
  long long len = 0;
  for (int s = lane; s < n; s += 32) {
    const int a = t[s], b = t[s + 1];
    if ((unsigned)a >= (unsigned)n || (unsigned)b >= (unsigned)n) {
      ok = false;
      continue;
    }
    const uint32_t old = atomicOr(&bits[a >> 5], 1u << (a & 31));
    if (old & (1u << (a & 31))) ok = false;  // a city twice
    len += I.dist[(size_t)a * ld + b];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(FULL, len, o);
  ok = __all_sync(FULL, ok);
  if (lane == 0 && (!ok || t[n] != t[0] || len != I.lens[k]))
    atomicOr(&I.st->status, kStatusCheckFailed);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
static int grid_for(size_t work, int threads, int sms) {
  size_t blocks = (work + threads - 1) / threads;
  const size_t cap = (size_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

cudaError_t launch_setup(const Instance& I, int sms, cudaStream_t st) {
  nn_tour_kernel<<<1, kNnTourThreads, 0, st>>>(I);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  init_matrices_kernel<<<grid_for((size_t)I.n * I.ld, 256, sms), 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_choice(const Instance& I, int sms, cudaStream_t st) {
  choice_kernel<<<grid_for((size_t)I.n * I.ld, 256, sms), 256, 0, st>>>(I, 0);
  return cudaGetLastError();
}

cudaError_t launch_best(const Instance& I, cudaStream_t st) {
  best_kernel<<<1, 1024, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_best_slots(const Instance* insts, const int* slots, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  best_slots_kernel<<<count, 256, 0, st>>>(insts, slots, count);
  return cudaGetLastError();
}

cudaError_t launch_update_rows(const Instance* insts, const int2* rows, int count, int max_ld,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int w = gather_warps_per_cta(max_ld);
  const size_t smem = (size_t)w * max_ld * sizeof(unsigned long long);
  static std::atomic<unsigned long long> attr_set{0};
  once_per_device(attr_set, [] {
    return cudaFuncSetAttribute(update_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                100 * 1024);
  });
  update_rows_kernel<<<(count + w - 1) / w, 32 * w, smem, st>>>(insts, rows, count, max_ld);
  return cudaGetLastError();
}

cudaError_t launch_dist_from_coords(const Instance& I, const int32_t* xy, cudaStream_t st) {
  const size_t total = (size_t)I.n * I.ld;
  size_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dist_from_coords_kernel<<<(int)blocks, 256, 0, st>>>(I, xy);
  return cudaGetLastError();
}

int gather_warps_per_cta(int ld) {
  // Shared memory per warp: one u64 row.  Keep a CTA at or below 96 KB.
  int w = (96 * 1024) / (8 * ld);
  if (w > 8) w = 8;
  if (w < 1) w = 1;
  return w;
}

cudaError_t launch_deposit(const Instance& I, int variant, int sms, cudaStream_t st) {
  if (variant == kDepositAtomicU64) {
    deposit_atomic_u64_kernel<<<grid_for((size_t)I.m * I.n, 256, sms), 256, 0, st>>>(I);
  } else if (variant == kDepositSymmetric) {
    deposit_symmetric_kernel<<<grid_for((size_t)I.m * I.n, 256, sms), 256, 0, st>>>(I);
  } else if (variant == kDepositAtomicF32) {
    evaporate_kernel<<<grid_for((size_t)I.n * I.ld / 4, 256, sms), 256, 0, st>>>(I);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    deposit_atomic_f32_kernel<<<grid_for((size_t)I.m * I.n, 256, sms), 256, 0, st>>>(I);
  }
  return cudaGetLastError();
}

cudaError_t launch_update(const Instance& I, int variant, int sms, cudaStream_t st) {
  if (variant == kDepositGather) {
    const int w = gather_warps_per_cta(I.ld);
    const size_t smem = (size_t)w * I.ld * sizeof(unsigned long long);
    static std::atomic<unsigned long long> attr_set{0};
    once_per_device(attr_set, [] {
      return cudaFuncSetAttribute(update_gather_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    });
    update_gather_kernel<<<(I.n + w - 1) / w, 32 * w, smem, st>>>(I, 1);
  } else if (variant == kDepositAtomicU64) {
    apply_acc_kernel<<<grid_for((size_t)I.n * I.ld / 4, 256, sms), 256, 0, st>>>(I, 1);
  } else if (variant == kDepositSymmetric) {
    const int nb = (I.n + kSymTile - 1) / kSymTile;
    apply_symmetric_kernel<<<dim3(nb, nb), dim3(kSymTile, 8), 0, st>>>(I, 1);
  } else {
    choice_kernel<<<grid_for((size_t)I.n * I.ld, 256, sms), 256, 0, st>>>(I, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_check_tours(const Instance& I, cudaStream_t st) {
  const int warps = 4;
  const size_t smem = (size_t)warps * ((I.n + 31) / 32) * sizeof(uint32_t);
  check_tours_kernel<<<(I.m + warps - 1) / warps, 32 * warps, smem, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_mmas_init(const Instance& I, int sms, cudaStream_t st) {
  mmas_init_kernel<<<grid_for((size_t)I.n * I.ld, 256, sms), 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_mmas_update(const Instance& I, int sms, cudaStream_t st) {
  mmas_update_kernel<<<grid_for((size_t)I.n * I.ld / 4, 256, sms), 256, 0, st>>>(I, 1);
  return cudaGetLastError();
}

int launches_for_variant(int variant) {
  // construct + best + deposit kernels + update kernel
  if (variant == kDepositGather) return 3;
  if (variant == kDepositAtomicU64 || variant == kDepositSymmetric) return 4;
  return 5;
}

}  // namespace aco
