// Host-side launch interface of the Ant System kernels.
#pragma once

#include <cuda_runtime.h>

#include "aco_device.cuh"

namespace aco {

constexpr int kDepositGather = 0;
constexpr int kDepositAtomicU64 = 1;
constexpr int kDepositAtomicF32 = 2;

// Tiling of the construction kernel: C cities per thread, G warps per ant,
// A ants per CTA.
struct ConstructTiling {
  int C, G, A;
};

// Smallest supported tiling for n cities with G warps per ant (C = 0 if none).
ConstructTiling construct_tiling(int n, int G, int A);
// Default choice of G and A for n cities.
ConstructTiling default_construct_tiling(int n);
cudaError_t launch_construct(const Instance& I, ConstructTiling t, cudaStream_t st);

cudaError_t launch_setup(const Instance& I, int sms, cudaStream_t st);
cudaError_t launch_choice(const Instance& I, int sms, cudaStream_t st);
cudaError_t launch_best(const Instance& I, cudaStream_t st);
cudaError_t launch_deposit(const Instance& I, int variant, int sms, cudaStream_t st);
cudaError_t launch_update(const Instance& I, int variant, int sms, cudaStream_t st);
int launches_for_variant(int variant);
int gather_warps_per_cta(int ld);

// Per-G dispatchers (one translation unit each, compiled in parallel).
cudaError_t launch_construct_g1(const Instance& I, int C, int A, cudaStream_t st);
cudaError_t launch_construct_g2(const Instance& I, int C, int A, cudaStream_t st);
cudaError_t launch_construct_g4(const Instance& I, int C, int A, cudaStream_t st);
bool construct_supported(int C, int G);
cudaError_t launch_construct_items_g1(const Instance* insts, const int2* items, int count, int C,
                                      int A, cudaStream_t st);
cudaError_t launch_construct_items_g2(const Instance* insts, const int2* items, int count, int C,
                                      int A, cudaStream_t st);
cudaError_t launch_construct_items_g4(const Instance* insts, const int2* items, int count, int C,
                                      int A, cudaStream_t st);
cudaError_t launch_construct_items(const Instance* insts, const int2* items, int count,
                                   ConstructTiling t, cudaStream_t st);

// Batched best / gather update over device-side lists.
cudaError_t launch_best_slots(const Instance* insts, const int* slots, int count, cudaStream_t st);
cudaError_t launch_update_rows(const Instance* insts, const int2* rows, int count, int max_ld,
                               cudaStream_t st);
// Device-side setup of one instance from city coordinates (TSPLIB EUC_2D).
cudaError_t launch_dist_from_coords(const Instance& I, const int32_t* xy, cudaStream_t st);

}  // namespace aco
