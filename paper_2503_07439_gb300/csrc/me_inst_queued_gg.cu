// Kernel instantiation: the queued mixed-precision subtracted real of g g -> t tbar g.
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_queued_gg(const LaunchArgs& a, cudaStream_t st) { return launch_queued_one<P_GG_TTG>(a, st); }
}  // namespace me
