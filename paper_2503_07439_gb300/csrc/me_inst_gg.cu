// Kernel instantiations: g g -> t tbar (Born) and g g -> t tbar g (tree, FKS real).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_gg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid == P_GG_TT) { ME_PREC_SWITCH(P_GG_TT) }
  if (pid == P_GG_TTG) { ME_PREC_SWITCH(P_GG_TTG) }
  return cudaErrorInvalidValue;
}
cudaError_t launch_items_gg(const LaunchArgs& a, cudaStream_t st) { return launch_items_one<P_GG_TTG>(a, st); }
}  // namespace me
