// Construction kernels with the exponential race (a per-candidate random
// rule that samples Eq. 1).
#include "construct_rule.cuh"

namespace aco {

cudaError_t launch_construct_rule2(const Instance& I, ConstructTiling t, cudaStream_t st) {
  return launch_construct_rule<2>(I, t, st);
}

}  // namespace aco
