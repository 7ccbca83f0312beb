// Kernel instantiation: the persistent serving kernel of the g g family (gg_tt, gg_ttg).
#include "me_persist.cuh"
namespace me {
cudaError_t launch_serve_gg(bool mixed, unsigned blocks, const PDesc* descs, PDone* dones, PCtl* ctl, PDev* dev,
                            const KParams& kpB, const KParams& kpR, unsigned pos0, unsigned long long idle_ns,
                            cudaStream_t st) {
  if (mixed)
    k_serve<P_GG_TT, P_GG_TTG, true><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
  else
    k_serve<P_GG_TT, P_GG_TTG, false><<<blocks, QT, 0, st>>>(descs, dones, ctl, dev, kpB, kpR, pos0, idle_ns);
  return cudaGetLastError();
}
}  // namespace me
