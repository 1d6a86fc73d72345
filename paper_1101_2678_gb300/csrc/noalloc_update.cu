// Pheromone update (evaporation + fixed-point atomic deposit + choice_info)
// on caller-owned device buffers, with its scratch in a file-scope device
// array instead of allocated memory (aco_update_pheromone_noalloc in aco.h).
//
// Some callers cannot call cudaMalloc at all: code running inside a region
// being captured into a CUDA graph by someone else, allocator-less embedded
// runtimes, or hosts that pre-plan every byte of device memory and forbid
// allocations after start-up.  For them this entry point needs no memory
// beyond the arrays they pass and one fixed static array that the module
// reserves on every GPU where the library is loaded.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "../../include/aco.h"
#include "aco_device.cuh"
#include "runtime.h"

namespace aco {
namespace {

constexpr int kNoallocMaxN = ACO_NOALLOC_MAX_N;
constexpr int kNoallocMaxM = ACO_NOALLOC_MAX_M;
// [0, N*N): u64 accumulator, [N*N, N*N + M): q_k, then one slot for S.
constexpr size_t kScratchWords = (size_t)kNoallocMaxN * kNoallocMaxN + kNoallocMaxM + 32;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int scratch_for_current_device(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(ACO_EINVAL, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_ptr[dev];
  return ACO_OK;
}

// Clear the accumulator rows this call uses.
__global__ void noalloc_zero_kernel(unsigned long long* acc, int n) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    acc[e] = 0ull;
}

// Deposit scale S and q_k = floor(dtau^k * 2^S), dtau^k = (float)(1/C^k).
__global__ void noalloc_prep_kernel(const long long* __restrict__ lens, int m,
                                    unsigned long long* q, unsigned long long* shift_slot) {
  __shared__ long long red[32];
  __shared__ int s_shift;
  long long bl = LLONG_MAX;
  for (int k = threadIdx.x; k < m; k += blockDim.x) bl = min(bl, lens[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bl = min(bl, __shfl_xor_sync(FULL, bl, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bl;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bl = min(bl, red[w]);
    const float dmax = (float)(1.0 / (double)bl);
    s_shift = 62 - ceil_log2_u32((uint32_t)m) - exponent_of_bits(__float_as_uint(dmax));
    *shift_slot = (unsigned long long)s_shift;
  }
  __syncthreads();
  const double scale = pow2d(s_shift);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const float dk = (float)(1.0 / (double)lens[k]);
    q[k] = __double2ull_rz((double)dk * scale);
  }
}

// red.global.add.u64 of q_k on (a,b) and (b,a) of every tour edge; tours are
// m rows of n+1 cities.  Entries outside [0, n) are skipped.
__global__ void noalloc_deposit_kernel(const int32_t* __restrict__ tours, int n, int m,
                                       const unsigned long long* __restrict__ q,
                                       unsigned long long* acc) {
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n), s = (int)(e % n);
    const int32_t* t = tours + (size_t)k * (n + 1);
    const int a = t[s], b = t[s + 1];
    if ((unsigned)a >= (unsigned)n || (unsigned)b >= (unsigned)n) continue;
    const unsigned long long qk = q[k];
    atomicAdd(acc + (size_t)a * n + b, qk);
    atomicAdd(acc + (size_t)b * n + a, qk);
  }
}

// tau' = fl(fl((1-rho) tau) + fl(acc) * 2^-S), choice = tau'^alpha * eta^beta.
__global__ void noalloc_apply_kernel(float* tau, const float* __restrict__ heta, float* choice,
                                     const unsigned long long* __restrict__ acc,
                                     const unsigned long long* __restrict__ shift_slot, int n,
                                     float alpha, float rho) {
  const size_t total = (size_t)n * n;
  const float keep = __fsub_rn(1.0f, rho);
  const float inv = pow2f(-(int)*shift_slot);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const float dep = __fmul_rn(__ull2float_rn(acc[e]), inv);
    const float t = __fadd_rn(__fmul_rn(keep, tau[e]), dep);
    tau[e] = t;
    choice[e] = choice_of(t, heta[e], alpha);
  }
}

}  // namespace
}  // namespace aco

using namespace aco;

extern "C" int aco_update_pheromone_noalloc(int32_t n, int32_t m, const int32_t* tours,
                                            const int64_t* lens, const float* heta, float* tau,
                                            float* choice, float alpha, float rho,
                                            int64_t stream) {
  if (n < 3 || n > kNoallocMaxN)
    return fail(ACO_EINVAL, "n=%d outside [3, %d] (the static scratch holds %d x %d)", n,
                kNoallocMaxN, kNoallocMaxN, kNoallocMaxN);
  if (m < 1 || m > kNoallocMaxM)
    return fail(ACO_EINVAL, "m=%d outside [1, %d]", m, kNoallocMaxM);
  if (!tours || !lens || !heta || !tau || !choice) return fail(ACO_EINVAL, "NULL device pointer");
  if (!std::isfinite(alpha) || alpha < 0.0f) return fail(ACO_EINVAL, "alpha must be finite and >= 0");
  if (!(rho > 0.0f && rho <= 1.0f)) return fail(ACO_EINVAL, "rho must lie in (0, 1]");
  unsigned long long* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  unsigned long long* acc = scratch;
  unsigned long long* q = scratch + (size_t)kNoallocMaxN * kNoallocMaxN;
  unsigned long long* shift_slot = q + kNoallocMaxM;
  cudaStream_t st = (cudaStream_t)(intptr_t)stream;
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  auto blocks = [](size_t work) { return (int)std::min<size_t>((work + 255) / 256, 4096); };
  noalloc_zero_kernel<<<blocks(nn), 256, 0, st>>>(acc, n);
  noalloc_prep_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const long long*>(lens), m, q,
                                          shift_slot);
  noalloc_deposit_kernel<<<blocks(mn), 256, 0, st>>>(tours, n, m, q, acc);
  noalloc_apply_kernel<<<blocks(nn), 256, 0, st>>>(tau, heta, choice, acc, shift_slot, n, alpha,
                                                   rho);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc update launch");
  return ACO_OK;
}
