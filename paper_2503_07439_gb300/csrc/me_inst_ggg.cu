// Kernel instantiations: g g -> t tbar g g (tree; float32 also with the tensor-core colour sum).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ggg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid == P_GG_TTGG && kind == K_TREE && !fp64 && lpe == 32) return launch_tree_tc<P_GG_TTGG>(a, st);
  if (pid == P_GG_TTGG) { ME_PREC_SWITCH(P_GG_TTGG) }
  return cudaErrorInvalidValue;
}
}  // namespace me
