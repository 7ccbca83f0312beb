// Kernel instantiations: e+e- -> u ubar (Born) and e+e- -> u ubar g (tree, FKS real).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ee(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid == P_EE_UU) { ME_PREC_SWITCH(P_EE_UU) }
  if (pid == P_EE_UUG) { ME_PREC_SWITCH(P_EE_UUG) }
  return cudaErrorInvalidValue;
}
cudaError_t launch_items_ee(const LaunchArgs& a, cudaStream_t st) { return launch_items_one<P_EE_UUG>(a, st); }
}  // namespace me
