// Construction kernels with the paper's data-parallel selection rule.
#include "construct_rule.cuh"

namespace aco {

cudaError_t launch_construct_rule1(const Instance& I, ConstructTiling t, cudaStream_t st) {
  return launch_construct_rule<1>(I, t, st);
}

}  // namespace aco
