// C ABI of the single-instance Ant System (include/aco.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/aco.h"
#include "aco_device.cuh"
#include "construct_chunks.h"
#include "kernels.h"
#include "runtime.h"
#include "checkpoint.h"

namespace aco {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  // Clear the runtime's last-error state so that a later, unrelated launch
  // check does not report this error again (a failed allocation is not
  // sticky).
  (void)cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? ACO_ENOMEM : ACO_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Construction tilings
// ---------------------------------------------------------------------------
// Cities per thread: the widths each tiling's launch table compiles.
static const int* c_set(int G, int H, int* cnt) {
  if (G == 1 && (H == 8 || H == 16 || H == 32)) {
    *cnt = chunk_count(ChunksOneWarp{});
    return chunk_values(ChunksOneWarp{});
  }
  if (H == 32 && G == 2) {
    *cnt = chunk_count(ChunksTwoWarps{});
    return chunk_values(ChunksTwoWarps{});
  }
  if (H == 32 && G == 4) {
    *cnt = chunk_count(ChunksFourWarps{});
    return chunk_values(ChunksFourWarps{});
  }
  *cnt = 0;
  return nullptr;
}

bool construct_supported(int C, int G, int H) {
  int cnt = 0;
  const int* set = c_set(G, H, &cnt);
  for (int i = 0; i < cnt; ++i)
    if (set[i] == C) return true;
  return false;
}

int ants_per_cta(ConstructTiling t) { return t.H == 32 ? t.W / t.G : t.W * (32 / t.H); }

ConstructTiling construct_tiling(int n, int G, int H, int ants) {
  int cnt = 0;
  const int* set = c_set(G, H, &cnt);
  const int W = H == 32 ? G * ants : (ants * H + 31) / 32;
  for (int i = 0; i < cnt; ++i)
    if (H * G * set[i] >= n) return ConstructTiling{set[i], G, H, W};
  return ConstructTiling{0, G, H, W};
}

ConstructTiling default_construct_tiling(int n) {
  if (n <= 32 * 76) return construct_tiling(n, 1, 32, 4);
  return construct_tiling(n, 2, 32, 4);
}

// Batched instances use the same whole-warp tiling: packing 2 or 4 ants per
// warp (H = 16, 8) measured about 4% slower on the 256-instance batch (the
// per-step work it shares is smaller than the segment shuffles it adds).
ConstructTiling batched_construct_tiling(int n) { return default_construct_tiling(n); }

cudaError_t launch_construct(const Instance& I, ConstructTiling t, cudaStream_t st) {
  if (t.W < 1 || t.W > 8) return cudaErrorInvalidValue;
  if (I.rule == 1) return launch_construct_rule1(I, t, st);
  if (I.rule == 2) return launch_construct_rule2(I, t, st);
  if (t.G == 1 && t.H == 8) return launch_construct_g1h8(I, t.C, t.W, st);
  if (t.G == 1 && t.H == 16) return launch_construct_g1h16(I, t.C, t.W, st);
  if (t.G == 1 && t.H == 32) return launch_construct_g1h32(I, t.C, t.W, st);
  if (t.G == 2 && t.H == 32) return launch_construct_g2h32(I, t.C, t.W, st);
  if (t.G == 4 && t.H == 32) return launch_construct_g4h32(I, t.C, t.W, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_construct_items(const Instance* insts, const int2* items, int count,
                                   ConstructTiling t, cudaStream_t st) {
  if (t.W < 1 || t.W > 8) return cudaErrorInvalidValue;
  if (t.G == 1 && t.H == 8) return launch_construct_items_g1h8(insts, items, count, t.C, t.W, t.S, st);
  if (t.G == 1 && t.H == 16) return launch_construct_items_g1h16(insts, items, count, t.C, t.W, t.S, st);
  if (t.G == 1 && t.H == 32) return launch_construct_items_g1h32(insts, items, count, t.C, t.W, t.S, st);
  if (t.G == 2 && t.H == 32) return launch_construct_items_g2h32(insts, items, count, t.C, t.W, t.S, st);
  if (t.G == 4 && t.H == 32) return launch_construct_items_g4h32(insts, items, count, t.C, t.W, t.S, st);
  return cudaErrorInvalidValue;
}

// floor(q0 2^32) for q0 in [0, 1]; q0 = 1 gives 2^32 (every step exploits).
unsigned long long acs_threshold_of(double q0) {
  return q0 >= 1.0  ? (1ull << 32)
         : q0 > 0.0 ? (unsigned long long)std::floor(q0 * 4294967296.0)
                    : 0ull;
}

// MAX-MIN Ant System f = tau_min / tau_max before the tau_min <= tau_max cap:
// (1 - p^(1/n)) / ((n/2 - 1) p^(1/n)), in double.
double mmas_f_of(int n, double p_best) {
  const double root = std::pow(p_best, 1.0 / (double)n);
  return (1.0 - root) / (((double)n / 2.0 - 1.0) * root);
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return sms;
}

int validate_instance(int32_t n, const int32_t* dist, float alpha, float beta, float rho,
                      int32_t m) {
  if (n < 3 || n > ACO_MAX_N) return fail(ACO_EINVAL, "n=%d outside [3, %d]", n, ACO_MAX_N);
  if (m < 1 || m > ACO_MAX_M) return fail(ACO_EINVAL, "m=%d outside [1, %d]", m, ACO_MAX_M);
  if (!dist) return fail(ACO_EINVAL, "dist is NULL");
  if (!std::isfinite(alpha) || alpha < 0.0f) return fail(ACO_EINVAL, "alpha must be finite and >= 0");
  if (!std::isfinite(beta) || beta < 0.0f) return fail(ACO_EINVAL, "beta must be finite and >= 0");
  if (!(rho > 0.0f && rho <= 1.0f)) return fail(ACO_EINVAL, "rho must lie in (0, 1]");
  for (int i = 0; i < n; ++i) {
    if (dist[(size_t)i * n + i] != 0) return fail(ACO_EINVAL, "dist[%d][%d] != 0", i, i);
    for (int j = i + 1; j < n; ++j) {
      const int32_t a = dist[(size_t)i * n + j], b = dist[(size_t)j * n + i];
      if (a != b) return fail(ACO_EINVAL, "dist not symmetric at (%d,%d)", i, j);
      if (a < 1) return fail(ACO_EINVAL, "dist[%d][%d]=%d, must be >= 1", i, j, a);
    }
  }
  return ACO_OK;
}

}  // namespace aco

using namespace aco;

// ---------------------------------------------------------------------------
// The handle
// ---------------------------------------------------------------------------
struct aco_colony {
  Instance I{};
  void* arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int sms = 148;
  int deposit = kDepositSymmetric;
  int use_graph = 1;
  int profile = 0;
  int warps_per_ant = 0;
  int lanes_per_ant = 0;
  int ants_per_cta = 0;
  int check = 0;  // ACO_OPT_CHECK
  bool tours_valid = false;
  bool constructed = false;
  bool nn_lists_built = false;
  long long host_iteration = 0;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[ACO_NUM_PHASES + 1] = {};
  void* sort_scratch = nullptr;  // keys, values and digit counts of the sort deposit
};

static ConstructTiling tiling_of(const aco_colony* h) {
  const int n = h->I.n;
  if (h->warps_per_ant == 0 && h->lanes_per_ant == 0) {
    ConstructTiling t = default_construct_tiling(n);
    if (h->ants_per_cta) t = construct_tiling(n, t.G, t.H, h->ants_per_cta);
    return t;
  }
  const int G = h->warps_per_ant ? h->warps_per_ant : 1;
  const int H = h->lanes_per_ant ? h->lanes_per_ant : 32;
  const int A = h->ants_per_cta ? h->ants_per_cta
                                : (H < 32 ? 4 * (32 / H) : G == 1 ? 4 : G == 2 ? 2 : 1);
  return construct_tiling(n, G, H, A);
}

static bool tiling_ok(ConstructTiling t, int rule) {
  if (t.C == 0 || t.W < 1 || t.W > 8) return false;
  if (t.H < 32 && t.G != 1) return false;
  if (rule != 0 && (t.H != 32 || t.G > 2)) return false;
  return ants_per_cta(t) >= 1;
}

// External records so that the events also become graph nodes under capture.
static cudaError_t record_event(aco_colony* h, cudaEvent_t ev, cudaStream_t st) {
  (void)h;
  return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
}

static void drop_graph(aco_colony* h) {
  if (h->exec) {
    cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
  }
}

static int enqueue_construct(aco_colony* h) {
  const ConstructTiling t = tiling_of(h);
  if (!tiling_ok(t, h->I.rule)) return fail(ACO_EINVAL, "no construction tiling for n=%d", h->I.n);
  cudaError_t e;
  if (h->profile && (e = record_event(h, h->ev[0], h->stream)) != cudaSuccess)
    return cuda_fail(e, "event");
  e = h->I.variant == kVariantAcs ? launch_acs_construct(h->I, h->stream)
      : h->I.nn > 0               ? launch_construct_nn(h->I, h->stream)
                                  : launch_construct(h->I, t, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "construct");
  if (h->profile && (e = record_event(h, h->ev[1], h->stream)) != cudaSuccess)
    return cuda_fail(e, "event");
  if (h->check && (e = launch_check_tours(h->I, h->stream)) != cudaSuccess)
    return cuda_fail(e, "check tours");
  if ((e = launch_best(h->I, h->stream)) != cudaSuccess) return cuda_fail(e, "best");
  if (h->profile && (e = record_event(h, h->ev[2], h->stream)) != cudaSuccess)
    return cuda_fail(e, "event");
  return ACO_OK;
}

static int enqueue_update(aco_colony* h) {
  cudaError_t e;
  const int variant = h->I.variant;
  if (variant == kVariantAs) {
    e = h->deposit == kDepositSort ? launch_sort_deposit(h->I, h->sort_scratch, h->sms, h->stream)
                                   : launch_deposit(h->I, h->deposit, h->sms, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "deposit");
  }
  if (h->profile && (e = record_event(h, h->ev[3], h->stream)) != cudaSuccess)
    return cuda_fail(e, "event");
  e = variant == kVariantMmas ? launch_mmas_update(h->I, h->sms, h->stream)
      : variant == kVariantAcs ? launch_acs_global(h->I, h->stream)
                               : launch_update(h->I,
                                               h->deposit == kDepositSort ? kDepositSymmetric
                                                                          : h->deposit,
                                               h->sms, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "update");
  // (the Ant Colony System reads its list weights from choice_info itself)
  if (h->I.nn > 0 && variant != kVariantAcs && (e = launch_nn_choice(h->I, h->stream)) != cudaSuccess)
    return cuda_fail(e, "nn choice");
  if (h->profile && (e = record_event(h, h->ev[4], h->stream)) != cudaSuccess)
    return cuda_fail(e, "event");
  return ACO_OK;
}

static int check_status(aco_colony* h) {
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, &h->I.st->status, sizeof(int), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  if (status & kStatusTimeout) return fail(ACO_ETIMEOUT, "a device-side wait gave up");
  if (status & kStatusCheckFailed)
    return fail(ACO_ECUDA, "a constructed tour failed the check (device status 0x%x)", status);
  if (status) return fail(ACO_ECUDA, "device status 0x%x", status);
  return ACO_OK;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

extern "C" {

const char* aco_strerror(int code) {
  switch (code) {
    case ACO_OK:
      return "ACO_OK";
    case ACO_EINVAL:
      return "ACO_EINVAL: invalid argument";
    case ACO_ENOMEM:
      return "ACO_ENOMEM: out of memory";
    case ACO_ECUDA:
      return "ACO_ECUDA: CUDA error";
    case ACO_ESTATE:
      return "ACO_ESTATE: call not valid in this state";
    case ACO_ETIMEOUT:
      return "ACO_ETIMEOUT: device-side wait gave up";
    case ACO_EBUSY:
      return "ACO_EBUSY: no free slot or memory budget";
    default:
      return "unknown ACO error code";
  }
}

const char* aco_last_error_message(void) { return g_err; }

static int create_common(int32_t n, const int32_t* dist, const int32_t* xy, float alpha,
                         float beta, float rho, int32_t m, uint64_t seed, aco_handle* out);

int aco_create(int32_t n, const int32_t* dist, float alpha, float beta, float rho, int32_t m,
               uint64_t seed, aco_handle* out) {
  if (!out) return fail(ACO_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_instance(n, dist, alpha, beta, rho, m);
  if (rc) return rc;
  return create_common(n, dist, nullptr, alpha, beta, rho, m, seed, out);
}

int aco_create_coords(int32_t n, const int32_t* xy, float alpha, float beta, float rho, int32_t m,
                      uint64_t seed, aco_handle* out) {
  if (!out) return fail(ACO_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_coords_public(n, xy);
  if (rc) return rc;
  if (m < 1 || m > ACO_MAX_M) return fail(ACO_EINVAL, "m=%d outside [1, %d]", m, ACO_MAX_M);
  if (!std::isfinite(alpha) || alpha < 0.0f || !std::isfinite(beta) || beta < 0.0f)
    return fail(ACO_EINVAL, "alpha and beta must be finite and >= 0");
  if (!(rho > 0.0f && rho <= 1.0f)) return fail(ACO_EINVAL, "rho must lie in (0, 1]");
  return create_common(n, nullptr, xy, alpha, beta, rho, m, seed, out);
}

static int create_common(int32_t n, const int32_t* dist, const int32_t* xy, float alpha,
                         float beta, float rho, int32_t m, uint64_t seed, aco_handle* out) {
  NvtxRange nvtx_range("aco_create");
  int rc;
  aco_colony* h = new (std::nothrow) aco_colony();
  if (!h) return fail(ACO_ENOMEM, "host allocation");
  Instance& I = h->I;
  I.n = n;
  I.m = m;
  I.ld = (int)align_up((size_t)n, 4);
  I.ldt = (int)align_up((size_t)n + 1, 4);
  I.ldm = (int)align_up((size_t)m, 32);
  I.alpha = alpha;
  I.beta = beta;
  I.rho = rho;
  I.seed = seed;
  const size_t mat = (size_t)n * I.ld;
  // Arena layout (every block 256-byte aligned).
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_dist = take(mat * 4), o_heta = take(mat * 4), o_tau = take(mat * 4),
               o_choice = take(mat * 4), o_tours = take((size_t)m * I.ldt * 4),
               o_lens = take((size_t)m * 8), o_nbr = take((size_t)n * I.ldm * 4),
               o_q = take((size_t)m * 8), o_delta = take((size_t)m * 4),
               o_acc = take(mat * 8), o_best = take(((size_t)n + 1) * 4),
               o_st = take(sizeof(IterState)), o_nnl = take((size_t)n * kNnStride * 4),
               o_nnc = take((size_t)n * kNnStride * 4), o_depnb = take((size_t)n * 4);
  h->arena_bytes = off;
  cudaError_t e = cudaMalloc(&h->arena, off);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaMalloc");
  }
  char* b = (char*)h->arena;
  I.dist = (const int32_t*)(b + o_dist);
  I.heta = (float*)(b + o_heta);
  I.tau = (float*)(b + o_tau);
  I.choice = (float*)(b + o_choice);
  I.tours = (int32_t*)(b + o_tours);
  I.lens = (long long*)(b + o_lens);
  I.nbr = (uint32_t*)(b + o_nbr);
  I.q = (unsigned long long*)(b + o_q);
  I.delta = (float*)(b + o_delta);
  I.acc = (unsigned long long*)(b + o_acc);
  I.best_tour = (int32_t*)(b + o_best);
  I.st = (IterState*)(b + o_st);
  I.nnlist = (int32_t*)(b + o_nnl);
  I.nnchoice = (float*)(b + o_nnc);
  I.nn = 0;
  // Row staging: the bulk copy is faster from n = 1002 on (1.22 vs 1.96 ms at
  // n = 1002, 6.15 vs 8.23 ms at n = 2392); lane copies win for rows of a few
  // hundred bytes (0.034 vs 0.038 ms at n = 48).
  I.stage = n <= 64 ? 1 : 0;
  I.dep_nb = (uint32_t*)(b + o_depnb);
  I.variant = kVariantAs;
  h->sms = device_sms();
  rc = ACO_OK;
  do {
    if ((e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
      rc = cuda_fail(e, "stream");
      break;
    }
    h->stream = h->own_stream;
    for (int i = 0; i <= ACO_NUM_PHASES; ++i)
      if ((e = cudaEventCreate(&h->ev[i])) != cudaSuccess) break;
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "event");
      break;
    }
    if ((e = cudaMemsetAsync(h->arena, 0, off, h->stream)) != cudaSuccess) {
      rc = cuda_fail(e, "memset");
      break;
    }
    IterState st0{};
    st0.best_len = INT64_MAX;
    if ((e = cudaMemcpyAsync(I.st, &st0, sizeof st0, cudaMemcpyHostToDevice, h->stream)) !=
        cudaSuccess) {
      rc = cuda_fail(e, "upload state");
      break;
    }
    if (dist) {
      // dist: n rows of n int32 into rows of ld (padding stays zero).
      e = cudaMemcpy2DAsync((void*)I.dist, (size_t)I.ld * 4, dist, (size_t)n * 4, (size_t)n * 4,
                            (size_t)n, cudaMemcpyHostToDevice, h->stream);
    } else {
      // coordinates staged in the choice_info block, distances built on the device
      e = cudaMemcpyAsync(I.choice, xy, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = launch_dist_from_coords(I, (const int32_t*)I.choice, h->stream);
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "upload instance");
      break;
    }
    if ((e = launch_setup(I, h->sms, h->stream)) != cudaSuccess) {
      rc = cuda_fail(e, "setup");
      break;
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
      rc = cuda_fail(e, "setup sync");
      break;
    }
  } while (0);
  if (rc) {
    aco_destroy(h);
    return rc;
  }
  *out = h;
  return ACO_OK;
}

int aco_destroy(aco_handle h) {
  if (!h) return ACO_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  for (int i = 0; i <= ACO_NUM_PHASES; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->arena) cudaFree(h->arena);
  if (h->sort_scratch) cudaFree(h->sort_scratch);
  delete h;
  return ACO_OK;
}

int aco_choice_info(aco_handle h, float* out) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  cudaError_t e = launch_choice(h->I, h->sms, h->stream);
  if (e == cudaSuccess && h->I.nn > 0) e = launch_nn_choice(h->I, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "choice");
  if (out) {
    const int n = h->I.n;
    e = cudaMemcpy2DAsync(out, (size_t)n * 4, h->I.choice, (size_t)h->I.ld * 4, (size_t)n * 4, n,
                          cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy choice");
    return check_status(h);
  }
  return ACO_OK;
}

int aco_construct_tours(aco_handle h, int32_t* tours, int64_t* lens) {
  NvtxRange nvtx_range("aco_construct_tours");
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  int rc = enqueue_construct(h);
  if (rc) return rc;
  h->tours_valid = true;
  h->constructed = true;
  cudaError_t e;
  const int n = h->I.n, m = h->I.m;
  if (tours &&
      (e = cudaMemcpy2DAsync(tours, (size_t)(n + 1) * 4, h->I.tours, (size_t)h->I.ldt * 4,
                             (size_t)(n + 1) * 4, m, cudaMemcpyDeviceToHost, h->stream)) !=
          cudaSuccess)
    return cuda_fail(e, "copy tours");
  if (lens && (e = cudaMemcpyAsync(lens, h->I.lens, (size_t)m * 8, cudaMemcpyDeviceToHost,
                                   h->stream)) != cudaSuccess)
    return cuda_fail(e, "copy lens");
  if (tours || lens) return check_status(h);
  return ACO_OK;
}

int aco_update_pheromone(aco_handle h) {
  NvtxRange nvtx_range("aco_update_pheromone");
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (!h->tours_valid) return fail(ACO_ESTATE, "no tours constructed since the last update");
  int rc = enqueue_update(h);
  if (rc) return rc;
  h->tours_valid = false;
  h->host_iteration += 1;
  return ACO_OK;
}

int aco_iterate(aco_handle h, int32_t iterations) {
  NvtxRange nvtx_range("aco_iterate");
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (iterations < 0) return fail(ACO_EINVAL, "iterations < 0");
  if (iterations == 0) return ACO_OK;
  cudaError_t e;
  if (h->use_graph) {
    if (!h->exec) {
      cudaGraph_t g = nullptr;
      if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
      int rc = enqueue_construct(h);
      if (!rc) rc = enqueue_update(h);
      e = cudaStreamEndCapture(h->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&h->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        h->exec = nullptr;
        return cuda_fail(e, "instantiate");
      }
    }
    for (int i = 0; i < iterations; ++i)
      if ((e = cudaGraphLaunch(h->exec, h->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
  } else {
    for (int i = 0; i < iterations; ++i) {
      int rc = enqueue_construct(h);
      if (!rc) rc = enqueue_update(h);
      if (rc) return rc;
    }
  }
  h->constructed = true;
  h->tours_valid = false;
  h->host_iteration += iterations;
  return ACO_OK;
}

int aco_best_tour(aco_handle h, int32_t* tour, int64_t* len) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (!h->constructed) return fail(ACO_ESTATE, "no tour constructed yet");
  cudaError_t e;
  if (tour && (e = cudaMemcpyAsync(tour, h->I.best_tour, ((size_t)h->I.n + 1) * 4,
                                   cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
    return cuda_fail(e, "copy best tour");
  if (len && (e = cudaMemcpyAsync(len, &h->I.st->best_len, 8, cudaMemcpyDeviceToHost,
                                  h->stream)) != cudaSuccess)
    return cuda_fail(e, "copy best len");
  return check_status(h);
}

int aco_get_pheromone(aco_handle h, float* tau) {
  if (!h || !tau) return fail(ACO_EINVAL, "NULL argument");
  const int n = h->I.n;
  cudaError_t e = cudaMemcpy2DAsync(tau, (size_t)n * 4, h->I.tau, (size_t)h->I.ld * 4,
                                    (size_t)n * 4, n, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy tau");
  return check_status(h);
}

int aco_get_heuristic(aco_handle h, float* heta) {
  if (!h || !heta) return fail(ACO_EINVAL, "NULL argument");
  const int n = h->I.n;
  cudaError_t e = cudaMemcpy2DAsync(heta, (size_t)n * 4, h->I.heta, (size_t)h->I.ld * 4,
                                    (size_t)n * 4, n, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy heta");
  return check_status(h);
}

int aco_get_iteration(aco_handle h, int64_t* iteration) {
  if (!h || !iteration) return fail(ACO_EINVAL, "NULL argument");
  unsigned long long it = 0;
  cudaError_t e = cudaMemcpyAsync(&it, &h->I.st->iteration, 8, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy iteration");
  int rc = check_status(h);
  *iteration = (int64_t)it;
  return rc;
}

int aco_get_tau0(aco_handle h, float* tau0, int64_t* nn_len) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  IterState st{};
  cudaError_t e = cudaMemcpyAsync(&st, h->I.st, sizeof st, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy state");
  int rc = check_status(h);
  if (tau0) *tau0 = st.tau0;
  if (nn_len) *nn_len = st.nn_len;
  return rc;
}

int aco_set_mmas(aco_handle h, double p_best, int32_t best_so_far) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (!(p_best > 0.0 && p_best < 1.0)) return fail(ACO_EINVAL, "p_best must lie in (0, 1)");
  if (best_so_far != 0 && best_so_far != 1) return fail(ACO_EINVAL, "best_so_far must be 0 or 1");
  if (h->constructed || h->host_iteration != 0 || h->I.variant != kVariantAs)
    return fail(ACO_ESTATE, "the update rule is chosen once, before the first construction");
  h->I.mmas_f = mmas_f_of(h->I.n, p_best);
  h->I.mmas_best_so_far = best_so_far;
  h->I.variant = kVariantMmas;
  drop_graph(h);
  cudaError_t e = launch_mmas_init(h->I, h->sms, h->stream);
  if (e == cudaSuccess && h->I.nn > 0) e = launch_nn_choice(h->I, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mmas init");
  return check_status(h);
}

int aco_set_acs(aco_handle h, double q0, float xi) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (!(q0 >= 0.0 && q0 <= 1.0)) return fail(ACO_EINVAL, "q0 must lie in [0, 1]");
  if (!(xi >= 0.0f && xi <= 1.0f)) return fail(ACO_EINVAL, "xi must lie in [0, 1]");
  if (h->I.m > kAcsMaxAnts)
    return fail(ACO_EINVAL, "the Ant Colony System runs at most %d ants (m=%d)", kAcsMaxAnts,
                h->I.m);
  if (h->I.rule != 0)
    return fail(ACO_EINVAL, "the Ant Colony System uses its own rule (no selection option)");
  if (h->constructed || h->host_iteration != 0 || h->I.variant != kVariantAs)
    return fail(ACO_ESTATE, "the update rule is chosen once, before the first construction");
  h->I.acs_threshold = acs_threshold_of(q0);
  h->I.acs_xi = xi;
  h->I.variant = kVariantAcs;
  drop_graph(h);
  cudaError_t e = launch_acs_init(h->I, h->sms, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "acs init");
  return check_status(h);
}

int aco_save_state(aco_handle h, void* buf, uint64_t capacity, uint64_t* size) {
  NvtxRange nvtx_range("aco_save_state");
  if (!h || !size) return fail(ACO_EINVAL, "NULL argument");
  const int n = h->I.n;
  *size = checkpoint_bytes(n);
  if (!buf) return ACO_OK;
  if (capacity < *size) return fail(ACO_EINVAL, "buffer holds %llu bytes, %llu needed",
                                    (unsigned long long)capacity, (unsigned long long)*size);
  CheckpointHeader hd = checkpoint_header(h->I);
  hd.constructed = h->constructed ? 1 : 0;
  hd.host_iteration = h->host_iteration;
  char* b = static_cast<char*>(buf);
  std::memcpy(b, &hd, sizeof hd);
  char* st = b + sizeof hd;
  float* tau = reinterpret_cast<float*>(st + sizeof(IterState));
  int32_t* best = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(tau) + (size_t)n * n * 4);
  cudaError_t e = cudaMemcpyAsync(st, h->I.st, sizeof(IterState), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(tau, (size_t)n * 4, h->I.tau, (size_t)h->I.ld * 4, (size_t)n * 4, n,
                          cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(best, h->I.best_tour, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost,
                        h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "save state");
  return check_status(h);
}

int aco_restore_state(aco_handle h, const void* buf, uint64_t size) {
  NvtxRange nvtx_range("aco_restore_state");
  if (!h || !buf) return fail(ACO_EINVAL, "NULL argument");
  CheckpointHeader hd{};
  IterState st{};
  const float* tau = nullptr;
  const int32_t* best = nullptr;
  int rc = checkpoint_parse(h->I, buf, size, hd, st, tau, best);
  if (rc) return rc;
  if (hd.variant == kVariantAcs && (h->I.rule != 0 || h->I.m > kAcsMaxAnts))
    return fail(ACO_EINVAL, "the Ant Colony System uses its own construction");
  const int n = hd.n;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->I.st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(h->I.tau, (size_t)h->I.ld * 4, tau, (size_t)n * 4, (size_t)n * 4, n,
                          cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->I.best_tour, best, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice,
                        h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "restore state");
  h->I.variant = hd.variant;
  h->I.mmas_best_so_far = hd.mmas_best_so_far;
  h->I.mmas_f = hd.mmas_f;
  h->I.acs_threshold = hd.acs_threshold;
  h->I.acs_xi = hd.acs_xi;
  h->constructed = hd.constructed != 0;
  h->tours_valid = false;
  h->host_iteration = hd.host_iteration;
  drop_graph(h);
  // choice_info from the restored tau (and the list-ordered copy)
  e = launch_choice(h->I, h->sms, h->stream);
  if (e == cudaSuccess && h->I.nn > 0) e = launch_nn_choice(h->I, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "restore choice");
  // the host copies above read caller memory: finish them before returning
  return check_status(h);
}

int aco_get_mmas_limits(aco_handle h, float* tau_min, float* tau_max) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  if (h->I.variant != kVariantMmas) return fail(ACO_ESTATE, "the handle runs the Ant System");
  IterState st{};
  cudaError_t e = cudaMemcpyAsync(&st, h->I.st, sizeof st, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy state");
  int rc = check_status(h);
  if (tau_min) *tau_min = st.tau_min;
  if (tau_max) *tau_max = st.tau_max;
  return rc;
}

int aco_set_option(aco_handle h, int32_t key, int64_t value) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  switch (key) {
    case ACO_OPT_DEPOSIT:
      if (value < 0 || value > 4) return fail(ACO_EINVAL, "deposit variant %lld", (long long)value);
      if (value == kDepositSort && !h->sort_scratch) {
        const cudaError_t e = cudaMalloc(&h->sort_scratch, sort_deposit_bytes(h->I.n, h->I.m));
        if (e != cudaSuccess) {
          h->sort_scratch = nullptr;
          return cuda_fail(e, "sort deposit scratch");
        }
      }
      h->deposit = (int)value;
      break;
    case ACO_OPT_STREAM:
      h->stream = value ? (cudaStream_t)(intptr_t)value : h->own_stream;
      break;
    case ACO_OPT_USE_GRAPH:
      h->use_graph = value != 0;
      break;
    case ACO_OPT_NN_LIST: {
      const int most = h->I.n - 1 < kNnStride ? h->I.n - 1 : kNnStride;
      if (value < 0 || value > most)
        return fail(ACO_EINVAL, "nearest-neighbour list length must be in [0, %d]", most);
      if (value > 0 && h->I.rule != 0)
        return fail(ACO_EINVAL, "nearest-neighbour lists use Eq. 1 (ACO_SELECT_EQ1)");
      cudaError_t e = cudaSuccess;
      if (value > 0 && !h->nn_lists_built) {
        e = launch_nn_lists(h->I, most, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "nn lists");
        h->nn_lists_built = true;
      }
      h->I.nn = (int)value;
      if (value > 0 && (e = launch_nn_choice(h->I, h->stream)) != cudaSuccess)
        return cuda_fail(e, "nn choice");
      break;
    }
    case ACO_OPT_SELECTION: {
      if (value != ACO_SELECT_EQ1 && value != ACO_SELECT_DATA_PARALLEL &&
          value != ACO_SELECT_EXP_RACE)
        return fail(ACO_EINVAL, "selection rule %lld", (long long)value);
      if (value != ACO_SELECT_EQ1 && h->I.nn > 0)
        return fail(ACO_EINVAL, "nearest-neighbour lists use Eq. 1 (ACO_SELECT_EQ1)");
      if (value != ACO_SELECT_EQ1 && h->I.variant == kVariantAcs)
        return fail(ACO_EINVAL, "the Ant Colony System uses its own construction");
      const int old = h->I.rule;
      h->I.rule = (int)value;
      if (!tiling_ok(tiling_of(h), h->I.rule)) {
        h->I.rule = old;
        return fail(ACO_EINVAL, "per-candidate rules need whole warps per ant (H = 32, G <= 2)");
      }
      break;
    }
    case ACO_OPT_PROFILE:
      h->profile = value != 0;
      break;
    case ACO_OPT_STAGING:
      if (value != 0 && value != 1) return fail(ACO_EINVAL, "staging must be 0 or 1");
      h->I.stage = (int)value;
      break;
    case ACO_OPT_CHECK:
      if (value != 0 && value != 1) return fail(ACO_EINVAL, "check must be 0 or 1");
      h->check = (int)value;
      break;
    case ACO_OPT_WARPS_PER_ANT:
    case ACO_OPT_LANES_PER_ANT:
    case ACO_OPT_ANTS_PER_CTA: {
      if (key == ACO_OPT_WARPS_PER_ANT && value != 0 && value != 1 && value != 2 && value != 4)
        return fail(ACO_EINVAL, "warps per ant must be 0, 1, 2 or 4");
      if (key == ACO_OPT_LANES_PER_ANT && value != 0 && value != 8 && value != 16 && value != 32)
        return fail(ACO_EINVAL, "lanes per ant must be 0, 8, 16 or 32");
      if (key == ACO_OPT_ANTS_PER_CTA && (value < 0 || value > 32))
        return fail(ACO_EINVAL, "ants per CTA must be in [0, 32]");
      int* field = key == ACO_OPT_WARPS_PER_ANT   ? &h->warps_per_ant
                   : key == ACO_OPT_LANES_PER_ANT ? &h->lanes_per_ant
                                                  : &h->ants_per_cta;
      const int old = *field;
      *field = (int)value;
      if (!tiling_ok(tiling_of(h), h->I.rule)) {
        *field = old;
        return fail(ACO_EINVAL, "no construction tiling for n=%d with this option", h->I.n);
      }
      break;
    }
    default:
      return fail(ACO_EINVAL, "unknown option %d", key);
  }
  drop_graph(h);
  return ACO_OK;
}

int aco_get_option(aco_handle h, int32_t key, int64_t* value) {
  if (!h || !value) return fail(ACO_EINVAL, "NULL argument");
  switch (key) {
    case ACO_OPT_DEPOSIT:
      *value = h->deposit;
      break;
    case ACO_OPT_STREAM:
      *value = (int64_t)(intptr_t)h->stream;
      break;
    case ACO_OPT_USE_GRAPH:
      *value = h->use_graph;
      break;
    case ACO_OPT_SELECTION:
      *value = h->I.rule;
      break;
    case ACO_OPT_STAGING:
      *value = h->I.stage;
      break;
    case ACO_OPT_CHECK:
      *value = h->check;
      break;
    case ACO_OPT_NN_LIST:
      *value = h->I.nn;
      break;
    case ACO_OPT_PROFILE:
      *value = h->profile;
      break;
    case ACO_OPT_WARPS_PER_ANT:
      *value = tiling_of(h).G;
      break;
    case ACO_OPT_LANES_PER_ANT:
      *value = tiling_of(h).H;
      break;
    case ACO_OPT_ANTS_PER_CTA:
      *value = ants_per_cta(tiling_of(h));
      break;
    default:
      return fail(ACO_EINVAL, "unknown option %d", key);
  }
  return ACO_OK;
}

int aco_get_kernel_times(aco_handle h, float* ms) {
  if (!h || !ms) return fail(ACO_EINVAL, "NULL argument");
  if (!h->profile) return fail(ACO_ESTATE, "profiling is off");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  for (int p = 0; p < ACO_NUM_PHASES; ++p) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, h->ev[p], h->ev[p + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "elapsed time");
    ms[p] = t;
  }
  return ACO_OK;
}

int aco_synchronize(aco_handle h) {
  if (!h) return fail(ACO_EINVAL, "NULL handle");
  return check_status(h);
}

int aco_kernel_launches_per_iteration(aco_handle h, int32_t* count) {
  if (!h || !count) return fail(ACO_EINVAL, "NULL argument");
  *count = (h->I.variant != kVariantAs     ? 3
            : h->deposit == kDepositSort ? 3 + sort_deposit_launches(h->I.n)
                                         : launches_for_variant(h->deposit)) +
           (h->I.nn > 0 && h->I.variant != kVariantAcs ? 1 : 0) + (h->check ? 1 : 0);
  return ACO_OK;
}

}  // extern "C"
