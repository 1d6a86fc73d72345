// Device-side building blocks shared by the Ant System kernels (sm_103a).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace aco {

constexpr unsigned FULL = 0xffffffffu;

// Host: run `set` (a kernel attribute setting, which holds per device) the
// first time it succeeds on the current device.  `done` keeps one bit per
// device ordinal (ordinals >= 64 run `set` every time); concurrent first
// calls may both run it, which is harmless for an idempotent setting.
template <class F>
inline cudaError_t once_per_device(std::atomic<unsigned long long>& done, F set) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set();
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  const cudaError_t e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Per-instance iteration state, resident on the device.
struct IterState {
  unsigned long long iteration;  // completed pheromone updates (Philox counter word 2)
  long long best_len;            // best-so-far tour length (INT64_MAX before the first)
  long long iter_best_len;       // shortest C^k of the last construction
  long long nn_len;              // nearest-neighbour tour length C_nn
  int iter_best_ant;
  int deposit_shift;             // S of the fixed-point deposit
  float tau0;
  int status;                    // device error bits (kStatus*)
  float tau_min, tau_max;        // MAX-MIN Ant System trail limits
  float mmas_dtau;               // MAX-MIN Ant System deposit of this iteration
  float acs_tau0;                // Ant Colony System tau0 = 1 / (n C_nn)
};

constexpr int kStatusTimeout = 1;
constexpr int kStatusBadTour = 2;
constexpr int kStatusCheckFailed = 4;  // a tour failed the optional check (ACO_OPT_CHECK)

// Everything a kernel needs to know about one instance.  Matrices are n rows
// of `ld` elements (ld = n rounded up to a multiple of 4, padding zero).
struct Instance {
  int n, m, ld;
  int ldt;   // tour row stride (>= n + 1, multiple of 4)
  int ldm;   // nbr row stride (>= m, multiple of 32)
  float alpha, beta, rho;
  int rule;                     // 0: Eq. 1 (integer roulette); 1: product of a uniform and the
                                // weight, highest wins (the paper's data-parallel kernel);
                                // 2: the exponential race (smallest E_j / w_j)
  int stage;                    // row staging: 0 bulk copy (TMA) + mbarrier, 1 lane copies
  unsigned long long seed;
  const int32_t* dist;          // [n][ld]
  float* heta;                  // [n][ld]  eta^beta
  float* tau;                   // [n][ld]
  float* choice;                // [n][ld]  choice_info
  int32_t* tours;               // [m][ldt]
  long long* lens;              // [m]
  uint32_t* nbr;                // [n][ldm]  (pred << 16 | succ) of city i in tour k
  unsigned long long* q;        // [m]   fixed-point deposit per ant
  float* delta;                 // [m]   dtau^k as float
  unsigned long long* acc;      // [n][ld] fixed-point accumulator (atomic u64 variant)
  int32_t* best_tour;           // [n + 1]
  IterState* st;
  // Nearest-neighbour lists (optional; nn = 0: off): list(i) in nnlist[i][0..nn)
  // (rows of kNnStride), and their choice_info values in list order.
  int nn;
  int32_t* nnlist;              // [n][kNnStride]
  float* nnchoice;              // [n][kNnStride]
  // Update rule: kVariantAs (Eqs. 2-4) or kVariantMmas (the MAX-MIN Ant
  // System: one depositing tour, trails clamped into [tau_min, tau_max]).
  int variant;
  int mmas_best_so_far;         // 1: the best-so-far tour deposits, 0: the iteration best
  double mmas_f;                // tau_min / tau_max = (1 - p^(1/n)) / ((n/2 - 1) p^(1/n))
  uint32_t* dep_nb;             // [n]  (pred << 16 | succ) of city i in the depositing tour
  // Ant Colony System: a step exploits when its Philox word x2 is below
  // acs_threshold = floor(q0 2^32); local evaporation xi.
  unsigned long long acs_threshold;
  float acs_xi;
};

constexpr int kVariantAs = 0;
constexpr int kVariantMmas = 1;
constexpr int kVariantAcs = 2;

constexpr int kNnStride = 32;   // longest supported list

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by 0x9E3779B9 /
// 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
struct Philox4 {
  uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

// Uniform in (0, 1] of candidate j at one construction step:
// (floor(x / 2^8) + 1) * 2^-24 with x word (j mod 4) of Philox counter
// (step, ant, iteration, 1 + j / 4); this returns all four words' uniforms.
__device__ __forceinline__ float candidate_uniform_of(uint32_t x) {
  return __fmaf_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-08f, 5.9604644775390625e-08f);
}

// The draw of one construction step: counter (step, ant, iteration, 0).
__device__ __forceinline__ Philox4 step_draw(unsigned long long seed, uint32_t step, uint32_t ant,
                                             uint32_t iteration) {
  return philox4x32_10(step, ant, iteration, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ceil(log2 v) for v >= 1.
__host__ __device__ __forceinline__ int ceil_log2_u32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return v <= 1 ? 0 : 32 - __clz(v - 1);
#else
  int c = 0;
  while ((1ull << c) < v) ++c;
  return c;
#endif
}

// Unbiased exponent floor(log2 x) of a positive finite float given its bits
// (subnormals included: 2^-149 has exponent -149).
__device__ __forceinline__ int exponent_of_bits(uint32_t b) {
  return b >= 0x00800000u ? (int)(b >> 23) - 127 : -118 - __clz(b);
}

// 2^e as a float, for -126 <= e <= 127.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// 2^e as a double, for -1022 <= e <= 1023.
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src) {
  return __shfl_sync(FULL, v, src);
}

// choice_info = tau^alpha * eta^beta (alpha == 1: one rounding).
__device__ __forceinline__ float choice_of(float tau, float heta, float alpha) {
  if (alpha == 1.0f) return __fmul_rn(tau, heta);
  if (alpha == 0.0f) return heta;
  return __fmul_rn(powf(tau, alpha), heta);
}

// ---------------------------------------------------------------------------
// Shared-memory staging with the bulk-copy (TMA) engine and mbarriers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make initialised mbarriers visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread: expect `bytes` on `bar`, then copy them global -> shared with
// the bulk-copy engine.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Every device-side wait in this library gives up after this many polls
// (each poll may suspend the thread briefly), records kStatusTimeout and
// lets the kernel run to its end instead of hanging.
constexpr int kWaitPolls = 1 << 20;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  int polls = kWaitPolls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace aco
