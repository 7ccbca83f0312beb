// Allocation-free evaluation of the subtracted real weight.
//
// Callers that cannot allocate GPU memory -- for example code whose device memory is
// entirely owned by another allocator (a caching pool of the host application), code
// that must not trigger the implicit device-wide synchronisation of cudaMalloc and
// cudaFree, or code running where allocation is forbidden -- evaluate the FKS
// real-minus-counterterm weights through this one entry point.  Its only scratch
// memory is the file-scope device array below (the mixed-precision rescue list and
// its counter); the process tables live in a second file-scope device object.  Both
// exist on every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_kernels.cuh"

namespace {

constexpr int64_t kMaxPoints = ME_NOALLOC_MAX_POINTS;
constexpr int kCountSlot = 0;   // rescue counter
constexpr int kListOffset = 64; // rescue list starts 256 bytes in

// rescue counter + rescue index list: (1 << 20) + 64 int32 = 4 MiB + 256 B
static __device__ __align__(256) int g_noalloc_scratch[kListOffset + kMaxPoints];
static __device__ __align__(256) me::ColourTables g_noalloc_tables;

struct DeviceSlot {
  bool ready = false;
  int* scratch = nullptr;             // device address of g_noalloc_scratch on this device
  me::ColourTables* tables = nullptr; // device address of g_noalloc_tables on this device
};
std::mutex g_mu;
DeviceSlot g_slots[64];
me::ColourTables g_host_tables;  // host copy built once (static storage)
bool g_host_ready = false;

// once per device, with that device current: resolve the symbols' device addresses
// (a host-side symbol name is not a device address) and upload the process tables
int setup(int dev, DeviceSlot** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return me_internal_fail(ME_ERR_ARG, "me_eval_real_subtracted_noalloc: bad device");
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    if (!g_host_ready) {
      int rc = me_internal_build_tables(&g_host_tables);
      if (rc != ME_OK) return rc;
      g_host_ready = true;
    }
    cudaError_t e = cudaGetSymbolAddress((void**)&s.scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
    e = cudaGetSymbolAddress((void**)&s.tables, g_noalloc_tables);
    if (e != cudaSuccess) return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
    e = cudaMemcpyToSymbol(g_noalloc_tables, &g_host_tables, sizeof(me::ColourTables));
    if (e != cudaSuccess) return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
    s.ready = true;
  }
  *out = &s;
  return ME_OK;
}

// A buffer is usable when it is device memory of `dev` or managed memory; device memory
// of another GPU is refused (without peer access the kernel could not read it).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return me_internal_buffer_usable((int)at.type, at.device, dev) != 0;
}

// The caller's current device is put back on every return path.
struct CurrentDeviceGuard {
  int prev = -1;
  CurrentDeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
  }
  ~CurrentDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cudaError_t launch(int pid, int kind, bool fp64, int lpe, const me::LaunchArgs& a, cudaStream_t st) {
  switch (pid) {
    case me::P_EE_UUG: return me::launch_ee(pid, kind, fp64, lpe, a, st);
    case me::P_GG_TTG: return me::launch_gg(pid, kind, fp64, lpe, a, st);
    case me::P_UU_TTG: return me::launch_uu(pid, kind, fp64, lpe, a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// Pure argument rule of on_device(), exported (not part of me.h) so that the rule can be
// checked without a second GPU: cudaMemoryTypeDevice (2) memory must belong to
// `want_device`; cudaMemoryTypeManaged (3) memory is reachable from every device; host
// and unregistered memory are refused.
extern "C" int me_internal_buffer_usable(int mem_type, int mem_device, int want_device) {
  if (mem_type == (int)cudaMemoryTypeManaged) return 1;
  return mem_type == (int)cudaMemoryTypeDevice && mem_device == want_device;
}

extern "C" int me_eval_real_subtracted_noalloc(const char* process, const me_params* params, const double* momenta,
                                               const double* ps_weights, int64_t n, double* out, void* cuda_stream) {
  me::KParams kp;
  int pid = -1;
  int rc = me_internal_kparams(process, params, &kp, &pid);
  if (rc != ME_OK) return rc;
  if (pid != me::P_EE_UUG && pid != me::P_GG_TTG && pid != me::P_UU_TTG)
    return me_internal_fail(ME_ERR_PROCESS, "me_eval_real_subtracted_noalloc: process has no FKS sectors");
  if (n < 0 || n > kMaxPoints)
    return me_internal_fail(ME_ERR_ARG, "me_eval_real_subtracted_noalloc: n must be in [0, 1048576] "
                                        "(size of the built-in scratch)");
  const int lpe = params->lanes_per_event ? params->lanes_per_event : 4;
  if (lpe != 1 && lpe != 2 && lpe != 4 && lpe != 8 && lpe != 16)
    return me_internal_fail(ME_ERR_ARG, "me_eval_real_subtracted_noalloc: lanes_per_event");
  CurrentDeviceGuard keep_current;
  if (cudaSetDevice(params->device) != cudaSuccess)
    return me_internal_fail(ME_ERR_CUDA, "me_eval_real_subtracted_noalloc: cudaSetDevice failed");
  DeviceSlot* slot = nullptr;
  if ((rc = setup(params->device, &slot)) != ME_OK) return rc;
  if (n == 0) return ME_OK;
  const int dev = params->device;
  if (!momenta || !out || !on_device(momenta, dev) || !on_device(out, dev) ||
      (ps_weights && !on_device(ps_weights, dev)))
    return me_internal_fail(ME_ERR_ARG, "me_eval_real_subtracted_noalloc: buffers must be device memory of "
                                        "params->device (or managed memory)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  kp.tab = slot->tables;
  int* count = slot->scratch + kCountSlot;
  int* list = slot->scratch + kListOffset;
  const bool mixed = params->precision == ME_PREC_MIXED;
  me::LaunchArgs a{};
  a.p = momenta;
  a.wgt = ps_weights;
  a.n = n;
  a.out = out;
  a.kp = kp;
  a.groups = n;
  a.resc_list = list;
  a.resc_count = count;
  cudaError_t e;
  if (mixed) {
    // the counter keeps the previous call's value: clear it on the stream first
    if ((e = cudaMemsetAsync(count, 0, sizeof(int), st)) != cudaSuccess)
      return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
    a.kp.flag_unstable = 1;
  }
  if ((e = launch(pid, me::K_REAL, !mixed, lpe, a, st)) != cudaSuccess)
    return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
  if (mixed) {
    me::LaunchArgs r = a;
    r.kp.flag_unstable = 0;
    r.idx = list;
    r.count = count;
    if ((e = launch(pid, me::K_REAL, true, lpe, r, st)) != cudaSuccess)
      return me_internal_fail(ME_ERR_CUDA, cudaGetErrorString(e));
  }
  return ME_OK;
}
