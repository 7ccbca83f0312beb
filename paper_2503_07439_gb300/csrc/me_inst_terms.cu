// Kernel instantiations: per-term queues of e+e- -> u ubar g and u ubar -> t tbar g, and
// the cut lists of the tree entries (g g -> t tbar g is in me_inst_terms_gg.cu so that the
// two compile in parallel).
#include "me_kernels.cuh"
namespace me {
cudaError_t launch_terms_ee(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts,
                            cudaStream_t st) {
  return launch_terms_one<P_EE_UUG>(phase, mixed, a, tb, counts, st);
}
cudaError_t launch_terms_uu(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts,
                            cudaStream_t st) {
  return launch_terms_one<P_UU_TTG>(phase, mixed, a, tb, counts, st);
}
cudaError_t launch_cut_list(int pid, const LaunchArgs& a, int* list, int* listed, cudaStream_t st) {
  (void)cudaGetLastError();
  const long blocks = (a.groups + 127) / 128;
  if (blocks <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(listed, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const unsigned b = (unsigned)blocks;
  switch (pid) {
    case P_EE_UU: k_cut_list<P_EE_UU><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_EE_UUG: k_cut_list<P_EE_UUG><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_GG_TT: k_cut_list<P_GG_TT><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_GG_TTG: k_cut_list<P_GG_TTG><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_GG_TTGG: k_cut_list<P_GG_TTGG><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_UU_TT: k_cut_list<P_UU_TT><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    case P_UU_TTG: k_cut_list<P_UU_TTG><<<b, 128, 0, st>>>(a.p, a.n, a.count, a.out, a.kp, list, listed); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace me
