// Kernel instantiations: the persistent serving kernels of the e+e- and u ubar families
// and the launcher (the g g family is in me_inst_serve_gg.cu, compiled in parallel).
#include "me_persist.cuh"
namespace me {
cudaError_t launch_serve_gg(bool mixed, unsigned blocks, const PDesc* descs, PDone* dones, PCtl* ctl, PDev* dev,
                            const KParams& kpB, const KParams& kpR, unsigned pos0, unsigned long long idle_ns,
                            cudaStream_t st);

cudaError_t launch_serve(int family, bool mixed, unsigned blocks, const PDesc* descs, PDone* dones, PCtl* ctl,
                         PDev* dev, const KParams& kpB, const KParams& kpR, unsigned pos0, unsigned long long idle_ns,
                         cudaStream_t st) {
  (void)cudaGetLastError();
  if (family == 1) return launch_serve_gg(mixed, blocks, descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns, st);
  if (family == 0) {
    if (mixed)
      k_serve<P_EE_UU, P_EE_UUG, true><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
    else
      k_serve<P_EE_UU, P_EE_UUG, false><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
  } else if (family == 2) {
    if (mixed)
      k_serve<P_UU_TT, P_UU_TTG, true><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
    else
      k_serve<P_UU_TT, P_UU_TTG, false><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace me
