// Kernel instantiations: u ubar -> t tbar (Born) and u ubar -> t tbar g (tree, FKS real).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_uu(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid == P_UU_TT) { ME_PREC_SWITCH(P_UU_TT) }
  if (pid == P_UU_TTG) { ME_PREC_SWITCH(P_UU_TTG) }
  return cudaErrorInvalidValue;
}
cudaError_t launch_items_uu(const LaunchArgs& a, cudaStream_t st) { return launch_items_one<P_UU_TTG>(a, st); }
}  // namespace me
