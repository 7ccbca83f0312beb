// Kernel instantiations: the queued mixed-precision subtracted real of e+e- -> u ubar g
// and u ubar -> t tbar g, and the dispatcher (g g -> t tbar g is in me_inst_queued_gg.cu
// so that the two compile in parallel).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_queued(int pid, const LaunchArgs& a, cudaStream_t st) {
  switch (pid) {
    case P_EE_UUG: return launch_queued_one<P_EE_UUG>(a, st);
    case P_GG_TTG: return launch_queued_gg(a, st);
    case P_UU_TTG: return launch_queued_one<P_UU_TTG>(a, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace me
