// Host-side helpers shared by the C ABI translation units.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace aco {

// NVTX range around a host API call (visible to Nsight tools; a no-op when
// no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Record a message for aco_last_error_message() and return `code`.
int fail(int code, const char* fmt, ...);
// Map a CUDA error to ACO_ENOMEM / ACO_ECUDA with a message.
int cuda_fail(cudaError_t e, const char* what);
// Streaming multiprocessors of the current device.
int device_sms();
// Ant Colony System exploitation threshold floor(q0 2^32), q0 in [0, 1].
unsigned long long acs_threshold_of(double q0);
// MAX-MIN Ant System trail-limit ratio f for n cities and p_best.
double mmas_f_of(int n, double p_best);
// Argument checks shared by aco_create and the batch/pool admission.
int validate_instance(int32_t n, const int32_t* dist, float alpha, float beta, float rho,
                      int32_t m);

// Coordinates for aco_create_coords / aco_pool_admit_coords: range and
// pairwise distinctness.
int validate_coords_public(int32_t n, const int32_t* xy);

}  // namespace aco
