// Checkpoint blob shared by instance handles and pool slots: header, the
// device iteration state, tau (n*n, unpadded) and the best-so-far tour
// (n+1).  The instance itself (distances, eta^beta, nearest-neighbour lists)
// is not stored: it is rebuilt by creating the handle, or admitting the pool
// slot, again with the same arguments, which the header checks.
#pragma once

#include <cstdint>
#include <cstring>

#include "../../include/aco.h"
#include "aco_device.cuh"
#include "runtime.h"

namespace aco {

struct CheckpointHeader {
  uint32_t magic, version;
  int32_t n, m;
  float alpha, beta, rho;
  int32_t variant, mmas_best_so_far;
  double mmas_f;
  unsigned long long acs_threshold;
  float acs_xi;
  int32_t constructed;
  unsigned long long seed;
  long long host_iteration;
  uint32_t state_bytes, reserved;
};
constexpr uint32_t kCheckpointMagic = 0x31434f41u;  // "ACO1"

inline uint64_t checkpoint_bytes(int n) {
  return sizeof(CheckpointHeader) + sizeof(IterState) + (uint64_t)n * n * 4 +
         ((uint64_t)n + 1) * 4;
}

// The header for instance I (its rule and parameters); the caller fills in
// constructed and host_iteration.
inline CheckpointHeader checkpoint_header(const Instance& I) {
  CheckpointHeader hd{};
  hd.magic = kCheckpointMagic;
  hd.version = 1;
  hd.n = I.n;
  hd.m = I.m;
  hd.alpha = I.alpha;
  hd.beta = I.beta;
  hd.rho = I.rho;
  hd.variant = I.variant;
  hd.mmas_best_so_far = I.mmas_best_so_far;
  hd.mmas_f = I.mmas_f;
  hd.acs_threshold = I.acs_threshold;
  hd.acs_xi = I.acs_xi;
  hd.seed = I.seed;
  hd.state_bytes = (uint32_t)sizeof(IterState);
  return hd;
}

// Check a blob against instance I (same n, m, seed and parameters; a known
// rule; a clean device state; a best tour inside [0, n)) and point into it.
inline int checkpoint_parse(const Instance& I, const void* buf, uint64_t size,
                            CheckpointHeader& hd, IterState& st, const float*& tau,
                            const int32_t*& best) {
  if (size < sizeof hd) return fail(ACO_EINVAL, "checkpoint too short");
  std::memcpy(&hd, buf, sizeof hd);
  if (hd.magic != kCheckpointMagic || hd.version != 1 || hd.state_bytes != sizeof(IterState))
    return fail(ACO_EINVAL, "not a checkpoint of this library");
  if (hd.n != I.n || hd.m != I.m || hd.seed != I.seed || hd.alpha != I.alpha ||
      hd.beta != I.beta || hd.rho != I.rho)
    return fail(ACO_EINVAL, "the checkpoint is of another instance (n, m, seed or parameters)");
  if (size < checkpoint_bytes(hd.n)) return fail(ACO_EINVAL, "checkpoint truncated");
  if (hd.variant < kVariantAs || hd.variant > kVariantAcs)
    return fail(ACO_EINVAL, "checkpoint names an unknown update rule");
  const int n = hd.n;
  const char* b = static_cast<const char*>(buf);
  std::memcpy(&st, b + sizeof hd, sizeof st);
  if (st.status != 0) return fail(ACO_EINVAL, "the checkpoint records a device error");
  tau = reinterpret_cast<const float*>(b + sizeof hd + sizeof st);
  best = reinterpret_cast<const int32_t*>(b + sizeof hd + sizeof st + (size_t)n * n * 4);
  if (hd.constructed)
    for (int i = 0; i <= n; ++i)
      if (best[i] < 0 || best[i] >= n) return fail(ACO_EINVAL, "checkpoint tour out of range");
  return ACO_OK;
}

}  // namespace aco
