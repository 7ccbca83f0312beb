// Kernel instantiations: g g -> t tbar g g tree in float32 (k_tree_tc4: shared-memory helicity
// blocks, colour sums on tensor cores).
// The float64 kernels are in me_inst_ggg64.cu so that the two compile in parallel.
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_ggg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  if (pid != P_GG_TTGG) return cudaErrorInvalidValue;
  if (fp64) return launch_ggg64(kind, lpe, a, st);
  // float32 runs the cooperative tensor-core kernel: four lanes per event
  if (lpe != 4) return cudaErrorInvalidValue;
  return launch_one<P_GG_TTGG, float, 4>(kind, a, st);
}
}  // namespace me
