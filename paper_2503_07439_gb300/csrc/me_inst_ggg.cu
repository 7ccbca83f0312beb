// Kernel instantiations: g g -> t tbar g g (tree; the float32 kernel sums colours on tensor cores).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ggg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid == P_GG_TTGG) { ME_PREC_SWITCH(P_GG_TTGG) }
  return cudaErrorInvalidValue;
}
}  // namespace me
