// Kernel instantiations: g g -> t tbar g g tree in float64.
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ggg64(int kind, int lpe, const LaunchArgs& a, cudaStream_t st) {
  ME_LPE_SWITCH8(P_GG_TTGG, double)
}
}  // namespace me
