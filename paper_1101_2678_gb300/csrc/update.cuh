// Device bodies of the iteration-best and gather-update kernels, shared by the
// single-instance kernels and the batched pool kernels.
#pragma once

#include <climits>

#include "aco_device.cuh"

namespace aco {

// Block-wide (any blockDim multiple of 32, <= 1024): argmin of C^k (ties to
// the lower ant), best-so-far update, deposit scale S and the per-ant dtau^k,
// q_k of Eqs. 3-4.
// MAX-MIN Ant System trail limits for best-so-far length c_gb, in double,
// each rounded to float once: tau_max = 1 / (rho c_gb), tau_min = tau_max * f
// (f precomputed on the host), tau_min = tau_max where that is larger.
__device__ __forceinline__ void mmas_limits(const Instance& I, long long c_gb, float* tau_min,
                                            float* tau_max) {
  const double tmax = 1.0 / ((double)I.rho * (double)c_gb);
  double tmin = tmax * I.mmas_f;
  if (tmin > tmax) tmin = tmax;
  *tau_max = (float)tmax;
  *tau_min = (float)tmin;
}

// One MAX-MIN Ant System cell (i, j): evaporation, dtau on the depositing
// tour's edges at row i (its predecessor and successor of city i), the clamp
// into [lo, hi] off the diagonal and the padding.
__device__ __forceinline__ float mmas_cell(float tau, int i, int j, int n, int pred, int succ,
                                           float keep, float dtau, float lo, float hi) {
  float t = __fmul_rn(keep, tau);
  if (j == pred || j == succ) t = __fadd_rn(t, dtau);
  if (j != i && j < n) t = fminf(fmaxf(t, lo), hi);
  return t;
}

__device__ __forceinline__ void best_body(const Instance& I) {
  __shared__ long long red_l[32];
  __shared__ int red_k[32];
  __shared__ int s_best, s_shift, s_improved;
  const int m = I.m, n = I.n;
  long long bl = LLONG_MAX;
  int bk = INT_MAX;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const long long L = I.lens[k];
    if (L < bl) {
      bl = L;
      bk = k;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ol = __shfl_xor_sync(FULL, bl, o);
    const int ok = __shfl_xor_sync(FULL, bk, o);
    if (ol < bl || (ol == bl && ok < bk)) {
      bl = ol;
      bk = ok;
    }
  }
  if (lane == 0) {
    red_l[warp] = bl;
    red_k[warp] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (red_l[w] < bl || (red_l[w] == bl && red_k[w] < bk)) {
        bl = red_l[w];
        bk = red_k[w];
      }
    const float dmax = (float)(1.0 / (double)bl);
    const int S = 62 - ceil_log2_u32((uint32_t)m) - exponent_of_bits(__float_as_uint(dmax));
    IterState* st = I.st;
    st->iter_best_len = bl;
    st->iter_best_ant = bk;
    st->deposit_shift = S;
    s_improved = bl < st->best_len;
    if (s_improved) st->best_len = bl;
    s_best = bk;
    s_shift = S;
  }
  __syncthreads();
  const double scale = pow2d(s_shift);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const float dk = (float)(1.0 / (double)I.lens[k]);
    I.delta[k] = dk;
    I.q[k] = __double2ull_rz((double)dk * scale);
  }
  if (s_improved) {
    const int32_t* src = I.tours + (size_t)s_best * I.ldt;
    for (int s = threadIdx.x; s <= n; s += blockDim.x) I.best_tour[s] = src[s];
  }
  if (I.variant == kVariantMmas) {
    // The depositing tour (the iteration best, or the best-so-far tour,
    // which is this iteration's best when it just improved), its neighbours
    // per city, its deposit and the trail limits from the best-so-far length.
    const int32_t* dep = (I.mmas_best_so_far && !s_improved)
                             ? I.best_tour
                             : I.tours + (size_t)s_best * I.ldt;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
      const uint32_t pred = (uint32_t)dep[s == 0 ? n - 1 : s - 1], succ = (uint32_t)dep[s + 1];
      I.dep_nb[dep[s]] = (pred << 16) | succ;
    }
    if (threadIdx.x == 0) {
      IterState* st = I.st;
      const long long c_dep = I.mmas_best_so_far ? st->best_len : st->iter_best_len;
      st->mmas_dtau = (float)(1.0 / (double)c_dep);
      mmas_limits(I, st->best_len, &st->tau_min, &st->tau_max);
    }
  }
}

// tau' = fl(fl((1-rho) tau) + dep), dep = fl(acc) * 2^-S (Eqs. 2-4).
__device__ __forceinline__ float apply_deposit(float tau, unsigned long long acc, float keep,
                                               float inv_scale) {
  const float dep = __fmul_rn(__ull2float_rn(acc), inv_scale);
  return __fadd_rn(__fmul_rn(keep, tau), dep);
}

__device__ __forceinline__ float inv_scale_of(int S) {
  // 2^-S.  3 <= C^k < 2^44 (n <= 4096, int32 distances) and m <= 16384 put S
  // in [50, 106], inside the normal float range.
  return pow2f(-S);
}

// Atomic-free "scatter to gather" deposit fused with evaporation and
// choice_info.  One warp per row i: the construction kernel bucketed every
// tour edge under both of its cities (nbr[i][k] = predecessor and successor of
// i in tour k), so row i's deposit is a segmented reduction of 2m (column,
// q_k) pairs.  Lanes holding the same column are grouped with match.any and
// summed by shuffles; the group leader adds the group sum to the warp's
// private u64 row in shared memory.  No atomics, exact, deterministic.
__device__ __forceinline__ void gather_row(const Instance& I, const int i,
                                           unsigned long long* acc, const int lane) {
  const int ld = I.ld, m = I.m;
  for (int j = lane; j < ld; j += 32) acc[j] = 0ull;
  __syncwarp();
  const uint32_t* nb = I.nbr + (size_t)i * I.ldm;
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int k = k0 + lane;
    const bool valid = k < m;
    const uint32_t ps = valid ? nb[k] : 0u;
    const unsigned long long qk = valid ? I.q[k] : 0ull;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t col = valid ? (half ? (ps & 0xffffu) : (ps >> 16)) : 0xffffffffu;
      const uint32_t grp = __match_any_sync(FULL, col);
      const int rounds = (int)__reduce_max_sync(FULL, (uint32_t)__popc(grp));
      uint32_t rem = grp;
      unsigned long long sum = 0;
      for (int r = 0; r < rounds; ++r) {
        const int src = rem ? __ffs(rem) - 1 : lane;
        const unsigned long long val = shfl_u64(qk, src);
        if (rem) {
          sum += val;
          rem &= rem - 1;
        }
      }
      if (valid && lane == __ffs(grp) - 1) acc[col] += sum;
      __syncwarp();
    }
  }
  const float keep = __fsub_rn(1.0f, I.rho);
  const float inv = inv_scale_of(I.st->deposit_shift);
  const float alpha = I.alpha;
  float* tau = I.tau + (size_t)i * ld;
  const float* heta = I.heta + (size_t)i * ld;
  float* ch = I.choice + (size_t)i * ld;
  for (int j = lane * 4; j < ld; j += 128) {
    const float4 t4 = *reinterpret_cast<const float4*>(tau + j);
    const float4 h4 = *reinterpret_cast<const float4*>(heta + j);
    float4 o, c;
    o.x = apply_deposit(t4.x, acc[j + 0], keep, inv);
    o.y = apply_deposit(t4.y, acc[j + 1], keep, inv);
    o.z = apply_deposit(t4.z, acc[j + 2], keep, inv);
    o.w = apply_deposit(t4.w, acc[j + 3], keep, inv);
    c.x = choice_of(o.x, h4.x, alpha);
    c.y = choice_of(o.y, h4.y, alpha);
    c.z = choice_of(o.z, h4.z, alpha);
    c.w = choice_of(o.w, h4.w, alpha);
    *reinterpret_cast<float4*>(tau + j) = o;
    *reinterpret_cast<float4*>(ch + j) = c;
  }
}

}  // namespace aco

namespace aco {

// Row i of the MAX-MIN Ant System update by one warp (the pool's row list).
__device__ __forceinline__ void mmas_row(const Instance& I, const int i, const int lane) {
  const int n = I.n, ld = I.ld;
  const float keep = __fsub_rn(1.0f, I.rho);
  const float dtau = I.st->mmas_dtau, lo = I.st->tau_min, hi = I.st->tau_max;
  const float alpha = I.alpha;
  const uint32_t nb = I.dep_nb[i];
  const int pred = (int)(nb >> 16), succ = (int)(nb & 0xffffu);
  float* tau = I.tau + (size_t)i * ld;
  const float* heta = I.heta + (size_t)i * ld;
  float* ch = I.choice + (size_t)i * ld;
  for (int j = lane * 4; j < ld; j += 128) {
    const float4 t4 = *reinterpret_cast<const float4*>(tau + j);
    const float4 h4 = *reinterpret_cast<const float4*>(heta + j);
    float4 o, c;
    o.x = mmas_cell(t4.x, i, j + 0, n, pred, succ, keep, dtau, lo, hi);
    o.y = mmas_cell(t4.y, i, j + 1, n, pred, succ, keep, dtau, lo, hi);
    o.z = mmas_cell(t4.z, i, j + 2, n, pred, succ, keep, dtau, lo, hi);
    o.w = mmas_cell(t4.w, i, j + 3, n, pred, succ, keep, dtau, lo, hi);
    c.x = choice_of(o.x, h4.x, alpha);
    c.y = choice_of(o.y, h4.y, alpha);
    c.z = choice_of(o.z, h4.z, alpha);
    c.w = choice_of(o.w, h4.w, alpha);
    *reinterpret_cast<float4*>(tau + j) = o;
    *reinterpret_cast<float4*>(ch + j) = c;
  }
}

}  // namespace aco
