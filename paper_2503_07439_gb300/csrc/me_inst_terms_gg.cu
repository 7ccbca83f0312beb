// Kernel instantiation: per-term queues of g g -> t tbar g.
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_terms_gg(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts,
                            cudaStream_t st) {
  return launch_terms_one<P_GG_TTG>(phase, mixed, a, tb, counts, st);
}
}  // namespace me
