// Kernel instantiations: g g -> t tbar g g tree in float32 (colour sums on tensor cores).
// The float64 kernels are in me_inst_ggg64.cu so that the two compile in parallel.
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ggg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid != P_GG_TTGG) return cudaErrorInvalidValue;
  if (fp64) return launch_ggg64(kind, lpe, a, st);
  ME_LPE_SWITCH8(P_GG_TTGG, float)
}
}  // namespace me
