// Host-side launch interface of the Ant System kernels.
#pragma once

#include <cuda_runtime.h>

#include "aco_device.cuh"

namespace aco {

constexpr int kDepositGather = 0;
constexpr int kDepositAtomicU64 = 1;
constexpr int kDepositAtomicF32 = 2;
constexpr int kDepositSymmetric = 3;
constexpr int kDepositSort = 4;

// Tiling of the construction kernel: C cities per thread, G warps per ant
// group, H lanes per ant (H < 32: 32/H ants share a warp, G = 1), W warps
// per CTA.
struct ConstructTiling {
  int C, G, H, W;
  int S = 0;  // row staging of batched launches: 0 bulk copy, 1 lane copies
};

// Smallest supported C for n cities with G warps and H lanes per ant, and
// `ants_per_cta` ants per CTA (C = 0 if there is none).
ConstructTiling construct_tiling(int n, int G, int H, int ants_per_cta);
// Default tiling of a single instance (latency: whole warps per ant).
ConstructTiling default_construct_tiling(int n);
// Default tiling of batched instances (throughput: the fewest issued
// instructions per ant step).
ConstructTiling batched_construct_tiling(int n);
cudaError_t launch_construct(const Instance& I, ConstructTiling t, cudaStream_t st);
// Ants per CTA of a tiling.
int ants_per_cta(ConstructTiling t);

cudaError_t launch_setup(const Instance& I, int sms, cudaStream_t st);
cudaError_t launch_choice(const Instance& I, int sms, cudaStream_t st);
cudaError_t launch_best(const Instance& I, cudaStream_t st);
cudaError_t launch_deposit(const Instance& I, int variant, int sms, cudaStream_t st);
cudaError_t launch_update(const Instance& I, int variant, int sms, cudaStream_t st);
int launches_for_variant(int variant);
// MAX-MIN Ant System: trails to tau_max(C_nn); one update (evaporation, the
// depositing tour's dtau, clamp, choice_info).
cudaError_t launch_mmas_init(const Instance& I, int sms, cudaStream_t st);
// Optional check of the constructed tours (ACO_OPT_CHECK).
cudaError_t launch_check_tours(const Instance& I, cudaStream_t st);
cudaError_t launch_mmas_update(const Instance& I, int sms, cudaStream_t st);
// Ant Colony System: trails to 1/(n C_nn); construction with the local
// update (one CTA, m <= kAcsMaxAnts); the global update on the best tour.
constexpr int kAcsMaxAnts = 32;
cudaError_t launch_acs_init(const Instance& I, int sms, cudaStream_t st);
cudaError_t launch_acs_construct(const Instance& I, cudaStream_t st);
cudaError_t launch_acs_global(const Instance& I, cudaStream_t st);
// The same for `count` colonies insts[slots[b]] per launch (one CTA each,
// sized for the largest m and n among them; lists: all of them construct
// with their nearest-neighbour lists).
cudaError_t launch_acs_construct_slots(const Instance* insts, const int* slots, int count,
                                       int max_m, int max_n, bool lists, cudaStream_t st);
cudaError_t launch_acs_global_slots(const Instance* insts, const int* slots, int count,
                                    cudaStream_t st);
int gather_warps_per_cta(int ld);
// Atomic-free deposit by a radix sort of the tour edges (sort_deposit.cu):
// scratch bytes for n cities and m ants, the deposit into the upper-triangle
// accumulator (apply with the symmetric update), and its kernel launches.
size_t sort_deposit_bytes(int n, int m);
cudaError_t launch_sort_deposit(const Instance& I, void* scratch, int sms, cudaStream_t st);
int sort_deposit_launches(int n);

// Per-(G, H) dispatchers (one translation unit each, compiled in parallel).
#define ACO_DECLARE_CONSTRUCT(tag)                                                              \
  cudaError_t launch_construct_##tag(const Instance& I, int C, int warps, cudaStream_t st);     \
  cudaError_t launch_construct_items_##tag(const Instance* insts, const int2* items, int count, \
                                           int C, int warps, int lane_copy, cudaStream_t st);
ACO_DECLARE_CONSTRUCT(g1h8)
ACO_DECLARE_CONSTRUCT(g1h16)
ACO_DECLARE_CONSTRUCT(g1h32)
ACO_DECLARE_CONSTRUCT(g2h32)
ACO_DECLARE_CONSTRUCT(g4h32)
#undef ACO_DECLARE_CONSTRUCT
bool construct_supported(int C, int G, int H);
// The paper's data-parallel selection rule (Instance::rule == 1); H = 32, G = 1 or 2.
cudaError_t launch_construct_rule1(const Instance& I, ConstructTiling t, cudaStream_t st);
cudaError_t launch_construct_rule2(const Instance& I, ConstructTiling t, cudaStream_t st);
cudaError_t launch_construct_items(const Instance* insts, const int2* items, int count,
                                   ConstructTiling t, cudaStream_t st);
// One persistent launch over the items of several classes (whole warps per
// ant): class k holds items [begin[k], begin[k] + count[k]) of chunk width
// C[k]; the classes are taken in the order listed.
struct SingleClasses {
  int begin[8], count[8], C[8], lane_copy[8];
  int n;
};
bool single_launch_supports(int C);
cudaError_t launch_construct_single(const Instance* insts, const int2* items,
                                    const SingleClasses& cls, int total, int* ticket, int sms,
                                    cudaStream_t st);

// Nearest-neighbour lists: build list(i) (nn <= kNnStride), refresh their
// choice_info values, and the list-restricted construction.
cudaError_t launch_nn_lists(const Instance& I, int nn, cudaStream_t st);
cudaError_t launch_nn_choice(const Instance& I, cudaStream_t st);
cudaError_t launch_construct_nn(const Instance& I, cudaStream_t st);
// The same for many instances (pool slots): one warp per (slot, ant) item,
// bitmaps sized for the largest n; and the list-ordered choice_info refresh
// of `count` slots after their update.
cudaError_t launch_construct_nn_items(const Instance* insts, const int2* items, int count,
                                      int max_n, cudaStream_t st);
cudaError_t launch_nn_choice_slots(const Instance* insts, const int* slots, int count,
                                   int max_n, cudaStream_t st);

// Batched best / gather update over device-side lists.
cudaError_t launch_best_slots(const Instance* insts, const int* slots, int count, cudaStream_t st);
cudaError_t launch_update_rows(const Instance* insts, const int2* rows, int count, int max_ld,
                               cudaStream_t st);
// Device-side setup of one instance from city coordinates (TSPLIB EUC_2D).
cudaError_t launch_dist_from_coords(const Instance& I, const int32_t* xy, cudaStream_t st);

}  // namespace aco
