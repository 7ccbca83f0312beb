// Host side of the C ABI: process set-up (colour algebra), handles, dispatch,
// host<->device staging, FP64 rescue, accumulators, autotuning.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_kernels.cuh"

namespace me {

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
#define ME_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(ME_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------- reductions
__global__ void k_partials(const double* __restrict__ w, long n, double* __restrict__ part, const int* __restrict__ cnt) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  if (cnt) n = *cnt;
  for (long i = (long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long)gridDim.x * 256) {
    const double x = w[i];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

// One warp: lane l adds the partials l, l + 32, ... in order, then a fixed butterfly adds
// the lanes.  The order is fixed, so the result is reproducible; a single thread adding
// all partials in a dependent chain would take tens of microseconds of float64 latency.
__global__ void k_finish(const double* __restrict__ part, int nblk, double* __restrict__ acc, long n,
                         const int* __restrict__ cnt) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double a = 0.0, b = 0.0;
  for (int i = (int)threadIdx.x; i < nblk; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) {
    if (cnt) n = *cnt;
    acc[0] += a;
    acc[1] += b;
    acc[2] += (double)n;
  }
}
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
// Item rescue: a flagged point re-evaluates items in float64, largest error scale first,
// until the float32 error left is at most this fraction of tol |W| -- half the budget of
// an unflagged point, so that flagged points add little to the tail that the calibration
// of me_eps bounds (2^20 flat points: the 99.9th percentile of the error stays at 8.2e-6
// (g g -> t tbar g), 8.0e-6 (u ubar -> t tbar g) and 7.3e-6 (e+e- -> u ubar g) of tol =
// 1e-5; at 1 it reaches 1.5e-5).  A compile-time setting, like ME_MINB, for calibration
// studies: -DME_ITEM_BUDGET=x.
#ifndef ME_ITEM_BUDGET
#define ME_ITEM_BUDGET 0.5
#endif
constexpr double kItemBudget = ME_ITEM_BUDGET;

// ---------------------------------------------------------------- colour algebra (host)
using cd = std::complex<double>;
struct Gen {
  cd T[8][3][3];
  double f[8][8][8];
};
static Gen make_generators() {
  Gen g{};
  const double r3 = 1.0 / std::sqrt(3.0);
  cd l[8][3][3] = {};
  l[0][0][1] = l[0][1][0] = 1.0;
  l[1][0][1] = cd(0, -1);
  l[1][1][0] = cd(0, 1);
  l[2][0][0] = 1.0;
  l[2][1][1] = -1.0;
  l[3][0][2] = l[3][2][0] = 1.0;
  l[4][0][2] = cd(0, -1);
  l[4][2][0] = cd(0, 1);
  l[5][1][2] = l[5][2][1] = 1.0;
  l[6][1][2] = cd(0, -1);
  l[6][2][1] = cd(0, 1);
  l[7][0][0] = l[7][1][1] = r3;
  l[7][2][2] = -2.0 * r3;
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) g.T[a][i][j] = 0.5 * l[a][i][j];
  // f^abc = -2 i Tr([T^a, T^b] T^c)
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        cd tr = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
              tr += (g.T[a][i][j] * g.T[b][j][k] - g.T[b][i][j] * g.T[a][j][k]) * g.T[c][k][i];
        g.f[a][b][c] = (cd(0, -2) * tr).real();
      }
  return g;
}

// A colour tensor over legs with dimensions dims[], stored dense.
struct Tensor {
  std::vector<int> dims;
  std::vector<cd> v;
  size_t size() const { return v.size(); }
};
enum Rep { ADJ, FUND, ANTI };

// apply the colour-charge generator a of leg `axis` (representation rep) to t
static Tensor charge(const Gen& G, const Tensor& t, int axis, Rep rep, int a) {
  Tensor o = t;
  std::fill(o.v.begin(), o.v.end(), cd(0));
  size_t inner = 1;
  for (size_t k = axis + 1; k < t.dims.size(); ++k) inner *= t.dims[k];
  const int d = t.dims[axis];
  const size_t outer = t.size() / (inner * d);
  for (size_t o1 = 0; o1 < outer; ++o1)
    for (int x = 0; x < d; ++x)
      for (int y = 0; y < d; ++y) {
        cd m;
        if (rep == FUND) m = G.T[a][x][y];
        else if (rep == ANTI) m = -G.T[a][y][x];
        else m = cd(0, -1) * G.f[a][x][y];
        if (m == cd(0)) continue;
        for (size_t i = 0; i < inner; ++i) o.v[(o1 * d + x) * inner + i] += m * t.v[(o1 * d + y) * inner + i];
      }
  return o;
}

static cd inner(const Tensor& a, const Tensor& b) {
  cd s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += std::conj(a.v[i]) * b.v[i];
  return s;
}

struct ProcColour {
  std::vector<Tensor> basis;
  std::vector<Rep> reps;  // per axis
};

// string basis (T^{a_s0} ... T^{a_s(n-1)})_{ij} over axes (gluon_0..gluon_{n-1}, i, j)
static ProcColour ttng_basis(const Gen& G, int ng) {
  ProcColour pc;
  std::vector<int> perm(ng);
  for (int i = 0; i < ng; ++i) perm[i] = i;
  std::vector<int> dims(ng, 8);
  dims.push_back(3);
  dims.push_back(3);
  size_t ncol = 1;
  for (int i = 0; i < ng; ++i) ncol *= 8;
  do {
    Tensor t;
    t.dims = dims;
    t.v.assign(ncol * 9, cd(0));
    std::vector<int> a(ng);
    for (size_t c = 0; c < ncol; ++c) {
      size_t r = c;
      for (int i = ng - 1; i >= 0; --i) {
        a[i] = (int)(r % 8);
        r /= 8;
      }
      cd m[3][3], tmp[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m[i][j] = (i == j) ? 1.0 : 0.0;
      for (int q = 0; q < ng; ++q) {
        const int ai = a[perm[q]];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            cd s = 0;
            for (int k = 0; k < 3; ++k) s += m[i][k] * G.T[ai][k][j];
            tmp[i][j] = s;
          }
        std::memcpy(m, tmp, sizeof(m));
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t.v[c * 9 + i * 3 + j] = m[i][j];
    }
    pc.basis.push_back(std::move(t));
  } while (std::next_permutation(perm.begin(), perm.end()));
  for (int i = 0; i < ng; ++i) pc.reps.push_back(ADJ);
  pc.reps.push_back(FUND);  // t  (outgoing quark)
  pc.reps.push_back(ANTI);  // tbar (outgoing antiquark)
  return pc;
}

static double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

// axes (k: incoming u, l: incoming ubar, i: t, j: tbar [, a: gluon])
static ProcColour uu_basis(const Gen& G, bool gluon) {
  ProcColour pc;
  std::vector<int> dims = {3, 3, 3, 3};
  if (gluon) dims.push_back(8);
  const int na = gluon ? 8 : 1;
  const int nb = gluon ? 4 : 2;
  for (int e = 0; e < nb; ++e) {
    Tensor t;
    t.dims = dims;
    t.v.assign(81 * na, cd(0));
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int a = 0; a < na; ++a) {
              cd v;
              if (!gluon) {
                v = e == 0 ? delta(i, k) * delta(l, j) : delta(i, j) * delta(l, k);
              } else if (e == 0) v = G.T[a][i][k] * delta(l, j);
              else if (e == 1) v = delta(i, k) * G.T[a][l][j];
              else if (e == 2) v = G.T[a][i][j] * delta(l, k);
              else v = delta(i, j) * G.T[a][l][k];
              t.v[(((k * 3 + l) * 3 + i) * 3 + j) * na + a] = v;
            }
    pc.basis.push_back(std::move(t));
  }
  pc.reps = {ANTI, FUND, FUND, ANTI};
  if (gluon) pc.reps.push_back(ADJ);
  return pc;
}

// axes (i: u, j: ubar [, a])
static ProcColour ee_basis(const Gen& G, bool gluon) {
  ProcColour pc;
  Tensor t;
  const int na = gluon ? 8 : 1;
  t.dims = {3, 3};
  if (gluon) t.dims.push_back(8);
  t.v.assign(9 * na, cd(0));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int a = 0; a < na; ++a) t.v[(i * 3 + j) * na + a] = gluon ? G.T[a][i][j] : cd(delta(i, j));
  pc.basis.push_back(std::move(t));
  pc.reps = {FUND, ANTI};
  if (gluon) pc.reps.push_back(ADJ);
  return pc;
}

// Build all tables; verifies colour conservation of every basis tensor and
// that the Gram matrices are real.
static int build_tables(ColourTables& tab) {
  std::memset(&tab, 0, sizeof(tab));
  const Gen G = make_generators();
  struct Item {
    int pid;
    ProcColour pc;
  };
  std::vector<Item> items;
  items.push_back({P_EE_UU, ee_basis(G, false)});
  items.push_back({P_EE_UUG, ee_basis(G, true)});
  items.push_back({P_GG_TT, ttng_basis(G, 2)});
  items.push_back({P_GG_TTG, ttng_basis(G, 3)});
  items.push_back({P_GG_TTGG, ttng_basis(G, 4)});
  items.push_back({P_UU_TT, uu_basis(G, false)});
  items.push_back({P_UU_TTG, uu_basis(G, true)});
  for (auto& it : items) {
    const auto& B = it.pc.basis;
    const int nf = (int)B.size();
    for (int x = 0; x < nf; ++x) {
      // colour conservation: sum over legs of T_leg^a e_x = 0 for every a
      for (int a = 0; a < 8; ++a) {
        Tensor s = B[x];
        std::fill(s.v.begin(), s.v.end(), cd(0));
        for (size_t ax = 0; ax < B[x].dims.size(); ++ax) {
          if (B[x].dims[ax] == 1) continue;
          Tensor c = charge(G, B[x], (int)ax, it.pc.reps[ax], a);
          for (size_t q = 0; q < s.size(); ++q) s.v[q] += c.v[q];
        }
        double mx = 0;
        for (auto& v : s.v) mx = std::max(mx, std::abs(v));
        if (mx > 1e-12) return fail(ME_ERR_PROCESS, "colour basis not invariant for process table");
      }
      for (int y = 0; y < nf; ++y) {
        const cd c = inner(B[x], B[y]);
        if (std::abs(c.imag()) > 1e-12) return fail(ME_ERR_PROCESS, "complex colour matrix");
        tab.C[it.pid][x * nf + y] = c.real();
        tab.Cf[it.pid][x * nf + y] = (float)c.real();
      }
    }
    for (int x = 0; x < nf; ++x)
      for (int y = x; y < nf; ++y) {
        if (tab.C[it.pid][x * nf + y] != tab.C[it.pid][y * nf + x]) return fail(ME_ERR_PROCESS, "colour matrix not symmetric");
        const double u = (y == x ? 1.0 : 2.0) * tab.C[it.pid][x * nf + y];
        tab.U[it.pid][x * nf + y] = u;
        tab.Uf[it.pid][x * nf + y] = (float)u;
      }
    // Born colour correlators C^{kl}_{xy} = sum_a <T_k^a e_x | T_l^a e_y>
    if (it.pid == P_GG_TT || it.pid == P_UU_TT) {
      const int ci = it.pid == P_GG_TT ? 0 : 1;
      int pr = 0;
      for (int k = 0; k < 4; ++k)
        for (int l = k; l < 4; ++l, ++pr)
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              cd s = 0;
              for (int a = 0; a < 8; ++a)
                s += inner(charge(G, B[x], k, it.pc.reps[k], a), charge(G, B[y], l, it.pc.reps[l], a));
              if (std::abs(s.imag()) > 1e-12) return fail(ME_ERR_PROCESS, "complex colour correlator");
              tab.Ccorr[ci][pr][x * 2 + y] = s.real();
            }
    }
  }
  return ME_OK;
}

// ---------------------------------------------------------------- per-device state
struct DeviceState {
  bool ready = false;
  ColourTables* d_tab = nullptr;
};
static std::mutex g_dev_mu;
static DeviceState g_dev[64];
static ColourTables* g_host_tab = nullptr;

static int device_setup(int dev, ColourTables** d_tab) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev < 0 || dev >= 64) return fail(ME_ERR_ARG, "device ordinal out of range");
  if (!g_host_tab) {
    g_host_tab = new ColourTables;
    int rc = build_tables(*g_host_tab);
    if (rc != ME_OK) {
      delete g_host_tab;
      g_host_tab = nullptr;
      return rc;
    }
  }
  if (!g_dev[dev].ready) {
    ME_CUDA(cudaSetDevice(dev));
    ME_CUDA(cudaMalloc(&g_dev[dev].d_tab, sizeof(ColourTables)));
    cudaStream_t st;  // a private stream: no legacy-stream synchronisation
    ME_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const cudaError_t e1 = cudaMemcpyAsync(g_dev[dev].d_tab, g_host_tab, sizeof(ColourTables), cudaMemcpyHostToDevice, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    ME_CUDA(e1);
    ME_CUDA(e2);
    g_dev[dev].ready = true;
  }
  *d_tab = g_dev[dev].d_tab;
  return ME_OK;
}

// ---------------------------------------------------------------- process registry
struct ProcDesc {
  const char* name;
  int pid;
  int n_ext;
  int born_pid;   // underlying Born for the FKS entry (-1 if none)
  double avg;     // initial spin x colour average / identical factor
};
static const ProcDesc kProcs[] = {
    {"ee_uu", P_EE_UU, 4, -1, 4.0},
    {"ee_uug", P_EE_UUG, 5, P_EE_UU, 4.0},
    {"gg_tt", P_GG_TT, 4, -1, 256.0},
    {"gg_ttg", P_GG_TTG, 5, P_GG_TT, 256.0},
    {"gg_ttgg", P_GG_TTGG, 6, -1, 512.0},
    {"uu_tt", P_UU_TT, 4, -1, 36.0},
    {"uu_ttg", P_UU_TTG, 5, P_UU_TT, 36.0},
};

}  // namespace me

using namespace me;

struct me_handle {
  const ProcDesc* proc;
  me_params prm;
  KParams kp;
  int device;
  cudaStream_t own_stream;
  cudaStream_t stream;
  // device scratch (grown on demand)
  double* d_p = nullptr;
  double* d_w = nullptr;
  double* d_out = nullptr;
  size_t cap = 0;
  int* d_resc = nullptr;     // rescue index list (capacity cap)
  int* d_nresc = nullptr;    // [0]: points re-evaluated in float64, [1]: tile counter (queued kernel),
                             // [2] / [3]: real-block / Born items of the item rescue,
                             // [8]: points passing the cuts (tree entries with per-term queues)
  // item rescue (mixed-precision subtracted real): records and item lists, capacity icap
  ItemBufs ib{};
  size_t icap = 0;
  // per-term queues (term_queues = 1): records, configurations and queues, capacity tcap
  TermBufs tb{};
  size_t tcap = 0;
  double* d_part = nullptr;  // reduction partials
  double* d_acc = nullptr;   // accumulators (3)
  int lpe[2][2] = {{0, 0}, {0, 0}};  // [kind][fp64] chosen lanes per event
  int lpe_class[2][2] = {{-1, -1}, {-1, -1}};  // batch-size class they were chosen for
  int last_kind = K_TREE;
  // stage timers: per timed call, events before the main kernel, after it, after the
  // rescue kernel and after the reduction
  bool timers = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::array<cudaEvent_t, 4>> ev_used;
};

static void free_items(me_handle* h) {
  cudaFree(h->ib.ev);
  cudaFree(h->ib.mask);
  cudaFree(h->ib.a);
  cudaFree(h->ib.v);
  cudaFree(h->ib.list_r);
  cudaFree(h->ib.list_b);
  h->ib = ItemBufs{};
  h->icap = 0;
}

// Records and item lists of the item rescue for n points (grown on demand).
static int ensure_item_capacity(me_handle* h, size_t n) {
  if (n <= h->icap) return ME_OK;
  free_items(h);
  const size_t c = std::max(n, (size_t)1024);
  ItemBufs& b = h->ib;
  if (cudaMalloc(&b.ev, c * sizeof(int)) != cudaSuccess || cudaMalloc(&b.mask, c * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b.a, c * MAX_ITEMS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b.v, c * MAX_ITEMS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b.list_r, c * 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b.list_b, c * sizeof(int)) != cudaSuccess) {
    free_items(h);
    return fail(ME_ERR_OOM, "item-rescue scratch allocation failed");
  }
  b.cap = (long)c;
  h->icap = c;
  return ME_OK;
}

static void free_terms(me_handle* h) {
  TermBufs& t = h->tb;
  void* ptrs[] = {t.ev, t.flags, t.grow, t.a, t.v, t.m, t.cfg, t.bp, t.bx, t.bslot, t.q_real, t.r_real, t.r_born,
                  t.flagged, t.cnt};
  for (void* q : ptrs) cudaFree(q);
  h->tb = TermBufs{};
  h->tcap = 0;
}

// Records, Born configurations and queues of the per-term queues for n points.
static int ensure_term_capacity(me_handle* h, size_t n) {
  if (n <= h->tcap) return ME_OK;
  free_terms(h);
  const size_t c = std::max(n, (size_t)1024);
  TermBufs& t = h->tb;
  bool ok = cudaMalloc(&t.ev, c * sizeof(int)) == cudaSuccess && cudaMalloc(&t.flags, c * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.grow, c * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&t.a, c * MAX_ITEMS * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&t.v, c * MAX_ITEMS * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&t.m, c * 6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&t.cfg, c * 2 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.bp, c * 2 * 16 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&t.bx, c * 2 * 4 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&t.bslot, c * 2 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.q_real, c * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.r_real, c * 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.r_born, c * 2 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t.flagged, c * sizeof(int)) == cudaSuccess && cudaMalloc(&t.cnt, 8 * sizeof(int)) == cudaSuccess;
  if (!ok) {
    free_terms(h);
    return fail(ME_ERR_OOM, "per-term queue scratch allocation failed");
  }
  t.cap = (long)c;
  h->tcap = c;
  return ME_OK;
}

static int ensure_capacity(me_handle* h, size_t n) {
  if (n <= h->cap) return ME_OK;
  size_t c = std::max(n, (size_t)1024);
  cudaFree(h->d_p);
  cudaFree(h->d_w);
  cudaFree(h->d_out);
  cudaFree(h->d_resc);
  h->d_p = h->d_w = h->d_out = nullptr;
  h->d_resc = nullptr;
  h->cap = 0;
  if (cudaMalloc(&h->d_p, c * 4 * h->proc->n_ext * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_w, c * sizeof(double)) != cudaSuccess || cudaMalloc(&h->d_out, c * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_resc, c * sizeof(int)) != cudaSuccess)
    return fail(ME_ERR_OOM, "device scratch allocation failed");
  h->cap = c;
  return ME_OK;
}

// Address under which the kernels can use a caller's buffer, or nullptr if it has to be
// staged: device and managed memory as is; pinned (page-locked, mapped) host memory under
// its device address -- on GB300 the kernels then read and write it over the coherent
// CPU-GPU link while they compute, with no staging copy.  Pageable memory is staged.
struct PtrView {
  void* dev;  // address the kernels use, or nullptr if the buffer has to be staged
  bool host;  // host memory (pinned or pageable): results are in place when the call returns
};
static PtrView view_of(const void* p) {
  if (!p) return {nullptr, false};
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return {nullptr, true};  // unregistered: pageable host memory
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return {const_cast<void*>(p), false};
  if (at.type == cudaMemoryTypeHost) return {at.devicePointer, true};
  return {nullptr, at.type == cudaMemoryTypeUnregistered};
}

static cudaError_t dispatch(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st) {
  switch (pid) {
    case P_EE_UU:
    case P_EE_UUG: return launch_ee(pid, kind, fp64, lpe, a, st);
    case P_GG_TT:
    case P_GG_TTG: return launch_gg(pid, kind, fp64, lpe, a, st);
    case P_GG_TTGG: return launch_ggg(pid, kind, fp64, lpe, a, st);
    case P_UU_TT:
    case P_UU_TTG: return launch_uu(pid, kind, fp64, lpe, a, st);
  }
  return cudaErrorInvalidValue;
}

// The item rescue (mixed-precision subtracted real, two-launch organisation) unless the
// caller asked for whole points; item lists encode slot * 4 + block, so batches stay
// below 2^29 points on this path.
static bool use_items(const me_handle* h, int64_t n) {
  return h->prm.rescue == ME_RESCUE_ITEMS && n < (int64_t)1 << 29;
}

// Float64 work for the points the bulk-precision launch `a` flagged, on the handle's
// stream, counts read on the device: the item rescue (float64 items, then W recombined
// from the coefficients), or every flagged point re-evaluated whole.
static cudaError_t launch_rescue(me_handle* h, const LaunchArgs& a, int lpe64) {
  if (a.kp.item_rescue) {
    switch (h->proc->pid) {
      case P_EE_UUG: return launch_items_ee(a, h->stream);
      case P_GG_TTG: return launch_items_gg(a, h->stream);
      case P_UU_TTG: return launch_items_uu(a, h->stream);
    }
    return cudaErrorInvalidValue;
  }
  LaunchArgs r = a;
  r.kp.flag_unstable = 0;
  r.idx = h->d_resc;
  r.count = h->d_nresc;
  return dispatch(h->proc->pid, K_REAL, true, lpe64, r, h->stream);
}

// Whether a subtracted-real call of n points runs the per-term queues.
constexpr int64_t kTermsAutoMin = (int64_t)1 << 19;
static bool use_terms(const me_handle* h, int64_t n) {
  const int t = h->prm.term_queues;
  // the automatic choice leaves the masked path's own rescue options (whole points, the
  // per-block queue) to the masked path
  return t == ME_TERMS_QUEUED || (t == ME_TERMS_AUTO && h->prm.precision == ME_PREC_MIXED && n >= kTermsAutoMin &&
                                  h->prm.queued_rescue == 0 && h->prm.rescue == ME_RESCUE_ITEMS);
}

// Per-term queues of the subtracted real (phase 0: float64 pass, bulk items and
// recombination; phase 1: float64 rescue and recombination of the flagged points).
static cudaError_t launch_terms(me_handle* h, int phase, bool mixed, const LaunchArgs& a) {
  switch (h->proc->pid) {
    case P_EE_UUG: return launch_terms_ee(phase, mixed, a, h->tb, h->d_nresc, h->stream);
    case P_GG_TTG: return launch_terms_gg(phase, mixed, a, h->tb, h->d_nresc, h->stream);
    case P_UU_TTG: return launch_terms_uu(phase, mixed, a, h->tb, h->d_nresc, h->stream);
  }
  return cudaErrorInvalidValue;
}

// pick lanes-per-event by timing each candidate once on the caller's batch (first use)
// Lane layouts chosen by timing, shared by every handle of the process (key: device,
// process, kind, precision, batch-size class), so that later handles -- e.g. the slots
// of a server -- reuse the first handle's choice instead of tuning again.  The best
// layout depends on the batch size (small batches favour more lanes per point, which
// fill the GPU with fewer points), so the key holds floor(log2 n), capped at 15: the
// tuning runs on min(n, 2^15) points.
static std::mutex g_lpe_mu;
static std::map<std::tuple<int, int, int, int, int>, int> g_lpe_cache;

static int size_class(long n) {
  int c = 0;
  while (c < 15 && (2L << c) <= n) ++c;
  return c;
}

static int choose_lpe(me_handle* h, int kind, bool fp64, const LaunchArgs& a) {
  int& slot = h->lpe[kind][fp64 ? 1 : 0];
  if (h->prm.lanes_per_event) return slot = h->prm.lanes_per_event;
  const int cls = size_class(a.groups);
  if (slot && h->lpe_class[kind][fp64 ? 1 : 0] == cls) return slot;
  h->lpe_class[kind][fp64 ? 1 : 0] = cls;
  const auto key = std::make_tuple(h->prm.device, h->proc->pid, kind, fp64 ? 1 : 0, cls);
  {
    std::lock_guard<std::mutex> lk(g_lpe_mu);
    auto it = g_lpe_cache.find(key);
    if (it != g_lpe_cache.end()) return slot = it->second;
  }
  const int cands[5] = {1, 2, 4, 8, 16};
  const int ncand = 5;
  LaunchArgs t = a;
  t.groups = std::min<long>(a.groups, 1L << 15);
  t.kp.flag_unstable = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int pick = 8;
  for (int ic = 0; ic < ncand; ++ic) {
    const int c = cands[ic];
    if (dispatch(h->proc->pid, kind, fp64, c, t, h->stream) != cudaSuccess) continue;  // warm-up
    // the fastest of three timed launches: work of other streams (a server's other
    // slots) running at the same time only ever slows a launch down
    float ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, h->stream);
      dispatch(h->proc->pid, kind, fp64, c, t, h->stream);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float m1 = 0;
      cudaEventElapsedTime(&m1, e0, e1);
      ms = std::min(ms, m1);
    }
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_lpe_mu);
    g_lpe_cache.emplace(key, pick);
  }
  return slot = pick;
}

// The cuts of me_params as the kernels take them (Cuts in me_kernels.cuh), for process pid.
static bool cuts_valid(const me_params* p) {
  return std::isfinite(p->cut_pt_min) && p->cut_pt_min >= 0.0 && p->cut_abs_y_max > 0.0 &&
         !std::isnan(p->cut_abs_y_max) && p->cut_abs_cos_axis_max > 0.0 && !std::isnan(p->cut_abs_cos_axis_max) &&
         p->cut_thrust_max > 0.0 && !std::isnan(p->cut_thrust_max) && p->term_queues >= ME_TERMS_MASKED &&
         p->term_queues <= ME_TERMS_AUTO;
}
static Cuts cuts_of(int pid, const me_params* p) {
  Cuts c{};
  const bool heavy = pid == P_GG_TT || pid == P_GG_TTG || pid == P_GG_TTGG || pid == P_UU_TT || pid == P_UU_TTG;
  if (heavy) {
    if (p->cut_pt_min > 0.0) {
      c.mask |= CUT_PT;
      c.pt2_min = p->cut_pt_min * p->cut_pt_min;
    }
    if (std::isfinite(p->cut_abs_y_max)) {
      c.mask |= CUT_Y;
      c.ey2 = std::exp(2.0 * p->cut_abs_y_max);
    }
  } else {
    if (p->cut_abs_cos_axis_max < 1.0) {
      c.mask |= CUT_AXIS;
      c.cos2_max = p->cut_abs_cos_axis_max * p->cut_abs_cos_axis_max;
    }
    if (p->cut_thrust_max < 1.0) {
      c.mask |= CUT_THRUST;
      c.thrust_max = p->cut_thrust_max;
    }
  }
  return c;
}

extern "C" {

void me_default_params(me_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->version = ME_PARAMS_VERSION;
  p->precision = ME_PREC_FP64;
  p->alpha = 1.0 / 132.507;
  p->alpha_s = 0.118;
  p->mt = 173.0;
  p->xi_cut = 0.5;
  p->delta = 1.0;
  p->xi_thr = 1e-3;
  p->y_thr = 1e-3;
  p->tol = 1e-5;
  p->me_eps = 4e-7;
  p->device = 0;
  p->lanes_per_event = 0;
  p->rescue = ME_RESCUE_ITEMS;
  p->term_queues = ME_TERMS_AUTO;
  p->cut_pt_min = 0.0;
  p->cut_abs_y_max = HUGE_VAL;
  p->cut_abs_cos_axis_max = 1.0;
  p->cut_thrust_max = 1.0;
}

const char* me_last_error(void) { return g_err.c_str(); }

int me_init(const char* process, const me_params* params, me_handle** out) {
  if (!process || !params || !out) return fail(ME_ERR_ARG, "me_init: NULL argument");
  *out = nullptr;
  if (params->version != ME_PARAMS_VERSION) return fail(ME_ERR_ARG, "me_init: params version mismatch");
  if (params->precision != ME_PREC_FP64 && params->precision != ME_PREC_MIXED)
    return fail(ME_ERR_ARG, "me_init: precision must be ME_PREC_FP64 or ME_PREC_MIXED");
  if (!(params->xi_cut > 0 && params->xi_cut <= 1) || !(params->delta > 0 && params->delta <= 2) ||
      !(params->alpha_s > 0) || !(params->alpha > 0) || !(params->mt > 0))
    return fail(ME_ERR_ARG, "me_init: parameter out of range");
  const int l = params->lanes_per_event;
  if (l != 0 && l != 1 && l != 2 && l != 4 && l != 8 && l != 16) return fail(ME_ERR_ARG, "me_init: lanes_per_event");
  if (params->rescue != ME_RESCUE_POINTS && params->rescue != ME_RESCUE_ITEMS)
    return fail(ME_ERR_ARG, "me_init: rescue must be ME_RESCUE_POINTS or ME_RESCUE_ITEMS");
  if (!cuts_valid(params)) return fail(ME_ERR_ARG, "me_init: cut or term_queues parameter out of range");
  const ProcDesc* pd = nullptr;
  for (const auto& d : kProcs)
    if (std::strcmp(d.name, process) == 0) pd = &d;
  if (!pd) return fail(ME_ERR_PROCESS, std::string("me_init: unknown process ") + process);
  ColourTables* d_tab = nullptr;
  int rc = device_setup(params->device, &d_tab);
  if (rc != ME_OK) return rc;
  me_handle* h = new me_handle();
  h->proc = pd;
  h->prm = *params;
  h->device = params->device;
  if (cudaSetDevice(h->device) != cudaSuccess || cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail(ME_ERR_CUDA, "me_init: stream creation failed");
  }
  h->stream = h->own_stream;
  if (cudaMalloc(&h->d_nresc, 16 * sizeof(int)) != cudaSuccess || cudaMalloc(&h->d_part, 2 * RED_BLOCKS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_acc, 3 * sizeof(double)) != cudaSuccess) {
    me_destroy(h);
    return fail(ME_ERR_OOM, "me_init: allocation failed");
  }
  KParams& kp = h->kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.cp.gs = std::sqrt(4.0 * M_PI * params->alpha_s);
  kp.cp.ee = std::sqrt(4.0 * M_PI * params->alpha);
  kp.cp.mt = params->mt;
  kp.avg_inv = 1.0 / pd->avg;
  kp.born_avg_inv = pd->born_pid >= 0 ? 1.0 / kProcs[pd->born_pid].avg : 0.0;
  kp.nlo_factor = 1.0;
  kp.xi_cut = params->xi_cut;
  kp.delta = params->delta;
  kp.xi_thr = params->xi_thr;
  kp.y_thr = params->y_thr;
  kp.me_eps = params->me_eps;
  kp.tol = params->tol;
  kp.item_budget = kItemBudget;
  kp.cut = cuts_of(pd->pid, params);
  kp.tab = d_tab;
  // stream-ordered on the handle's own stream: no device-wide synchronisation, so a
  // handle can be created while other threads capture CUDA graphs
  if (cudaMemsetAsync(h->d_acc, 0, 3 * sizeof(double), h->own_stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_nresc, 0, 16 * sizeof(int), h->own_stream) != cudaSuccess ||
      cudaStreamSynchronize(h->own_stream) != cudaSuccess) {
    me_destroy(h);
    return fail(ME_ERR_CUDA, "me_init: device error");
  }
  *out = h;
  return ME_OK;
}

int me_n_external(const me_handle* h) { return h ? h->proc->n_ext : 0; }

static int run(me_handle* h, int kind, double nlo_factor, const double* momenta, const double* wgt, int64_t n,
               double* out) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  if (n < 0 || n > (int64_t)INT32_MAX) return fail(ME_ERR_ARG, "n out of range [0, 2^31)");
  if (n > 0 && (!momenta || !out)) return fail(ME_ERR_ARG, "NULL momenta/out");
  ME_CUDA(cudaSetDevice(h->device));
  h->last_kind = K_TREE;
  if (n == 0) return ME_OK;
  const int next = h->proc->n_ext;
  const PtrView pv = view_of(momenta), wv = view_of(wgt), ov = view_of(out);
  const double* vp = static_cast<const double*>(pv.dev);
  const double* vw = static_cast<const double*>(wv.dev);
  double* vo = static_cast<double*>(ov.dev);
  // host buffers (pinned or pageable): results are in place when the call returns
  const bool on_host = pv.host || wv.host || ov.host;
  int rc = ensure_capacity(h, (size_t)n);
  if (rc != ME_OK) return rc;
  const double* P = vp;
  const double* Wt = wgt ? vw : nullptr;
  double* O = vo;
  if (!vp) {
    ME_CUDA(cudaMemcpyAsync(h->d_p, momenta, (size_t)n * 4 * next * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    P = h->d_p;
  }
  if (wgt && !vw) {
    ME_CUDA(cudaMemcpyAsync(h->d_w, wgt, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    Wt = h->d_w;
  }
  if (!vo) O = h->d_out;
  const bool mixed = h->prm.precision == ME_PREC_MIXED;
  LaunchArgs a{};
  a.p = P;
  a.wgt = Wt;
  a.n = n;
  a.out = O;
  a.kp = h->kp;
  a.kp.nlo_factor = nlo_factor;
  a.groups = n;
  a.resc_list = h->d_resc;
  a.resc_count = h->d_nresc;
  a.tiles = h->d_nresc + 1;
  const bool terms = kind == K_REAL && use_terms(h, n);
  const bool cut_list = kind == K_TREE && h->prm.term_queues == ME_TERMS_QUEUED && a.kp.cut.mask;
  const bool queued = kind == K_REAL && mixed && h->prm.queued_rescue && !terms;
  // the queues encode slot * 4 + block in 32 bits
  if (terms && n >= (int64_t)1 << 29) return fail(ME_ERR_ARG, "term_queues: at most 2^29 - 1 points per call");
  if (terms && (rc = ensure_term_capacity(h, (size_t)n)) != ME_OK) return rc;
  // host momenta read in place: the float64 pass copies them to the device for the item
  // kernels, so that they cross the CPU-GPU link once
  if (terms && vp && pv.host) a.p_copy = h->d_p;
  if (kind == K_REAL && mixed) {
    a.kp.flag_unstable = 1;
    if (!queued && !terms && use_items(h, n)) {
      if ((rc = ensure_item_capacity(h, (size_t)n)) != ME_OK) return rc;
      a.kp.item_rescue = 1;
      a.items = h->ib;
    }
    ME_CUDA(cudaMemsetAsync(h->d_nresc, 0, 6 * sizeof(int), h->stream));
    h->last_kind = K_REAL;
  }
  // the first call per (kind, precision) times the lane layouts (synchronising);
  // both are chosen before the launches whose results are kept.  The queued kernel
  // runs one lane per point in both precisions; the per-term queues one lane per item.
  if (queued) h->lpe[kind][0] = h->lpe[kind][1] = 1;
  const int lpe64 = (kind == K_REAL && mixed && !queued && !terms) ? choose_lpe(h, kind, true, a) : 0;
  const int lpe = queued ? 1 : (terms ? std::max(1, h->lpe[kind][mixed ? 0 : 1]) : choose_lpe(h, kind, !mixed, a));
  if (terms) h->lpe[kind][0] = h->lpe[kind][1] = lpe;  // a counted launch needs a layout on record
  std::array<cudaEvent_t, 4> ev{};
  const bool timed = h->timers && h->ev_used.size() < 4096;
  if (timed) {
    for (auto& e : ev) {
      if (h->ev_pool.empty()) {
        cudaEvent_t x;
        ME_CUDA(cudaEventCreate(&x));
        h->ev_pool.push_back(x);
      }
      e = h->ev_pool.back();
      h->ev_pool.pop_back();
    }
    h->ev_used.push_back(ev);
    ME_CUDA(cudaEventRecord(ev[0], h->stream));
  }
  if (terms) {
    ME_CUDA(launch_terms(h, 0, mixed, a));
  } else if (queued) {
    ME_CUDA(launch_queued(h->proc->pid, a, h->stream));
  } else {
    if (cut_list) {
      // per-term queues of a tree entry: only the points that pass the cuts are evaluated
      ME_CUDA(launch_cut_list(h->proc->pid, a, h->d_resc, h->d_nresc + 8, h->stream));
      a.idx = h->d_resc;
      a.count = h->d_nresc + 8;
    }
    ME_CUDA(dispatch(h->proc->pid, kind, !mixed, lpe, a, h->stream));
  }
  if (timed) ME_CUDA(cudaEventRecord(ev[1], h->stream));
  if (terms && mixed) ME_CUDA(launch_terms(h, 1, mixed, a));
  if (kind == K_REAL && mixed && !queued && !terms) ME_CUDA(launch_rescue(h, a, lpe64));
  if (timed) ME_CUDA(cudaEventRecord(ev[2], h->stream));
  k_partials<<<RED_BLOCKS, 256, 0, h->stream>>>(O, n, h->d_part, nullptr);
  k_finish<<<1, 32, 0, h->stream>>>(h->d_part, RED_BLOCKS, h->d_acc, n, nullptr);
  ME_CUDA(cudaGetLastError());
  if (timed) ME_CUDA(cudaEventRecord(ev[3], h->stream));
  if (!vo) ME_CUDA(cudaMemcpyAsync(out, O, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (on_host) ME_CUDA(cudaStreamSynchronize(h->stream));
  return ME_OK;
}

int me_eval_born(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out) {
  return run(h, K_TREE, 1.0, momenta, ps_weights, n, out);
}

// n-body NLO factor of e+e- -> u ubar: 1 + a_s [5 - 2 pi^2/3 - (3 + 4 ln xi_c) ln(delta/2)]
static double nbody_factor(const me_handle* h) {
  const double a_s = h->prm.alpha_s * (4.0 / 3.0) / (2.0 * M_PI);
  const double c = 5.0 - 2.0 * M_PI * M_PI / 3.0 - (3.0 + 4.0 * std::log(h->prm.xi_cut)) * std::log(0.5 * h->prm.delta);
  return 1.0 + a_s * c;
}

int me_eval_nbody_nlo(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  if (h->proc->pid != P_EE_UU) return fail(ME_ERR_PROCESS, "me_eval_nbody_nlo: only defined for ee_uu");
  return run(h, K_TREE, nbody_factor(h), momenta, ps_weights, n, out);
}

int me_eval_real_subtracted(me_handle* h, const double* momenta, const double* ps_weights, int64_t n, double* out) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  if (h->proc->born_pid < 0) return fail(ME_ERR_PROCESS, "me_eval_real_subtracted: process has no FKS sectors");
  return run(h, K_REAL, 1.0, momenta, ps_weights, n, out);
}

int me_last_rescued(me_handle* h, int64_t* n_rescued) {
  if (!h || !n_rescued) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  int c = 0;
  if (h->prm.precision == ME_PREC_MIXED && h->last_kind == K_REAL) {
    ME_CUDA(cudaMemcpyAsync(&c, h->d_nresc, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    ME_CUDA(cudaStreamSynchronize(h->stream));
  }
  *n_rescued = c;
  return ME_OK;
}

int me_last_rescue_work(me_handle* h, int64_t* points, int64_t* real_blocks, int64_t* born_sets) {
  if (!h || !points || !real_blocks || !born_sets) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  int c[4] = {0, 0, 0, 0};
  if (h->prm.precision == ME_PREC_MIXED && h->last_kind == K_REAL) {
    ME_CUDA(cudaMemcpyAsync(c, h->d_nresc, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    ME_CUDA(cudaStreamSynchronize(h->stream));
  }
  *points = c[0];
  *real_blocks = c[2];
  *born_sets = c[3];
  return ME_OK;
}

int me_last_rescue_configs(me_handle* h, int64_t* set0, int64_t* set1) {
  if (!h || !set0 || !set1) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  int c[6] = {0, 0, 0, 0, 0, 0};
  if (h->prm.precision == ME_PREC_MIXED && h->last_kind == K_REAL) {
    ME_CUDA(cudaMemcpyAsync(c, h->d_nresc, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    ME_CUDA(cudaStreamSynchronize(h->stream));
  }
  *set0 = c[4];
  *set1 = c[5];
  return ME_OK;
}

int me_get_accumulators(me_handle* h, double out[3]) {
  if (!h || !out) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  ME_CUDA(cudaMemcpyAsync(out, h->d_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ME_CUDA(cudaStreamSynchronize(h->stream));
  return ME_OK;
}

int me_set_accumulators(me_handle* h, const double in[3]) {
  if (!h || !in) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  ME_CUDA(cudaMemcpyAsync(h->d_acc, in, 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  ME_CUDA(cudaStreamSynchronize(h->stream));
  return ME_OK;
}

int me_enable_stage_timers(me_handle* h, int on) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  h->timers = on != 0;
  return ME_OK;
}

int me_stage_times(me_handle* h, double out_ms[3], int64_t* calls) {
  if (!h || !out_ms || !calls) return fail(ME_ERR_ARG, "NULL argument");
  ME_CUDA(cudaSetDevice(h->device));
  ME_CUDA(cudaStreamSynchronize(h->stream));
  double t[3] = {0, 0, 0};
  for (auto& ev : h->ev_used) {
    for (int k = 0; k < 3; ++k) {
      float ms = 0;
      ME_CUDA(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
      t[k] += ms;
    }
    for (auto e : ev) h->ev_pool.push_back(e);
  }
  *calls = (int64_t)h->ev_used.size();
  h->ev_used.clear();
  for (int k = 0; k < 3; ++k) out_ms[k] = t[k];
  return ME_OK;
}

int me_set_stream(me_handle* h, void* s) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  h->stream = s ? (cudaStream_t)s : h->own_stream;
  return ME_OK;
}

int me_synchronize(me_handle* h) {
  if (!h) return fail(ME_ERR_ARG, "NULL handle");
  ME_CUDA(cudaSetDevice(h->device));
  ME_CUDA(cudaStreamSynchronize(h->stream));
  return ME_OK;
}

void me_destroy(me_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->d_p);
  cudaFree(h->d_w);
  cudaFree(h->d_out);
  cudaFree(h->d_resc);
  cudaFree(h->d_nresc);
  free_items(h);
  free_terms(h);
  cudaFree(h->d_part);
  cudaFree(h->d_acc);
  for (auto& ev : h->ev_used)
    for (auto e : ev) cudaEventDestroy(e);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

}  // extern "C"

// kernel kind and Born factor of an ME_KIND_* request
static int kind_of(const me_handle* h, int me_kind, double* nlo) {
  *nlo = 1.0;
  if (me_kind == ME_KIND_REAL_SUBTRACTED) {
    if (h->proc->born_pid < 0) return -1;
    return K_REAL;
  }
  if (me_kind == ME_KIND_NBODY_NLO) {
    if (h->proc->pid != P_EE_UU) return -1;
    *nlo = nbody_factor(h);
  }
  return K_TREE;
}

int me_internal_prepare_counted(me_handle* h, int me_kind, int64_t cap) {
  double nlo;
  const int kind = kind_of(h, me_kind, &nlo);
  if (kind < 0) return fail(ME_ERR_PROCESS, "counted launch: kind not defined for the process");
  const bool mixed = h->prm.precision == ME_PREC_MIXED;
  if (!h->lpe[kind][mixed ? 0 : 1] || (kind == K_REAL && mixed && !h->lpe[kind][1]))
    return fail(ME_ERR_ARG, "counted launch: run one ordinary call of this kind first");
  ME_CUDA(cudaSetDevice(h->device));
  int rc = ensure_capacity(h, (size_t)cap);
  if (rc == ME_OK && kind == K_REAL && use_terms(h, cap)) {
    if (cap >= (int64_t)1 << 29) return fail(ME_ERR_ARG, "term_queues: at most 2^29 - 1 points per call");
    return ensure_term_capacity(h, (size_t)cap);
  }
  if (rc == ME_OK && kind == K_REAL && mixed && !h->prm.queued_rescue && use_items(h, cap))
    rc = ensure_item_capacity(h, (size_t)cap);
  return rc;
}

int me_internal_launch_counted(me_handle* h, int me_kind, const double* d_p, const double* d_w, int64_t cap,
                               const int* d_n, double* d_out) {
  double nlo;
  const int kind = kind_of(h, me_kind, &nlo);
  const bool mixed = h->prm.precision == ME_PREC_MIXED;
  if (kind < 0 || cap <= 0 || (size_t)cap > h->cap || !d_p || !d_n || !d_out)
    return fail(ME_ERR_ARG, "counted launch: bad arguments or handle not prepared");
  const int lpe = h->lpe[kind][mixed ? 0 : 1], lpe64 = h->lpe[kind][1];
  LaunchArgs a{};
  a.p = d_p;
  a.wgt = d_w;
  a.n = cap;
  a.out = d_out;
  a.kp = h->kp;
  a.kp.nlo_factor = nlo;
  a.count = d_n;
  a.groups = cap;
  a.resc_list = h->d_resc;
  a.resc_count = h->d_nresc;
  a.tiles = h->d_nresc + 1;
  const bool terms = kind == K_REAL && use_terms(h, cap);
  const bool cut_list = kind == K_TREE && h->prm.term_queues == ME_TERMS_QUEUED && a.kp.cut.mask;
  const bool queued = kind == K_REAL && mixed && h->prm.queued_rescue && !terms;
  h->last_kind = K_TREE;
  if (terms && (size_t)cap > h->tcap) return fail(ME_ERR_ARG, "counted launch: handle not prepared");
  if (kind == K_REAL && mixed) {
    a.kp.flag_unstable = 1;
    if (!queued && !terms && use_items(h, cap)) {
      if ((size_t)cap > h->icap) return fail(ME_ERR_ARG, "counted launch: handle not prepared");
      a.kp.item_rescue = 1;
      a.items = h->ib;
    }
    ME_CUDA(cudaMemsetAsync(h->d_nresc, 0, 6 * sizeof(int), h->stream));
    h->last_kind = K_REAL;
  }
  if (terms) {
    ME_CUDA(launch_terms(h, 0, mixed, a));
    if (mixed) ME_CUDA(launch_terms(h, 1, mixed, a));
  } else if (queued) {
    ME_CUDA(launch_queued(h->proc->pid, a, h->stream));
  } else {
    if (cut_list) {
      ME_CUDA(launch_cut_list(h->proc->pid, a, h->d_resc, h->d_nresc + 8, h->stream));
      a.idx = h->d_resc;
      a.count = h->d_nresc + 8;
    }
    ME_CUDA(dispatch(h->proc->pid, kind, !mixed, lpe, a, h->stream));
  }
  if (kind == K_REAL && mixed && !queued && !terms) ME_CUDA(launch_rescue(h, a, lpe64));
  k_partials<<<RED_BLOCKS, 256, 0, h->stream>>>(d_out, cap, h->d_part, d_n);
  k_finish<<<1, 32, 0, h->stream>>>(h->d_part, RED_BLOCKS, h->d_acc, cap, d_n);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int me_internal_final_masses(me_handle* h, double* masses, int* n_out, cudaStream_t* stream) {
  if (!h || !masses || !n_out || !stream) return fail(ME_ERR_ARG, "NULL argument");
  const int pid = h->proc->pid;
  const int nout = h->proc->n_ext - 2;
  const bool tops = pid == P_GG_TT || pid == P_GG_TTG || pid == P_GG_TTGG || pid == P_UU_TT || pid == P_UU_TTG;
  for (int j = 0; j < nout; ++j) masses[j] = (tops && j < 2) ? h->prm.mt : 0.0;
  *n_out = nout;
  *stream = h->stream;
  ME_CUDA(cudaSetDevice(h->device));
  return ME_OK;
}

int me_internal_rescued_async(me_handle* h, int* dst) {
  if (!h || !dst) return fail(ME_ERR_ARG, "NULL argument");
  if (h->prm.precision != ME_PREC_MIXED || h->last_kind != K_REAL) {
    *dst = 0;
    return ME_OK;
  }
  ME_CUDA(cudaMemcpyAsync(dst, h->d_nresc, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  return ME_OK;
}

int me_internal_fail(int code, const char* msg) { return fail(code, msg ? msg : ""); }

int me_internal_build_tables(me::ColourTables* tab) {
  if (!tab) return fail(ME_ERR_ARG, "NULL table");
  return build_tables(*tab);
}

int me_internal_kparams(const char* process, const me_params* params, me::KParams* kp, int* pid) {
  if (!process || !params || !kp || !pid) return fail(ME_ERR_ARG, "NULL argument");
  if (params->version != ME_PARAMS_VERSION) return fail(ME_ERR_ARG, "params version mismatch");
  if (params->precision != ME_PREC_FP64 && params->precision != ME_PREC_MIXED)
    return fail(ME_ERR_ARG, "precision must be ME_PREC_FP64 or ME_PREC_MIXED");
  if (!(params->xi_cut > 0 && params->xi_cut <= 1) || !(params->delta > 0 && params->delta <= 2) ||
      !(params->alpha_s > 0) || !(params->alpha > 0) || !(params->mt > 0) || !cuts_valid(params))
    return fail(ME_ERR_ARG, "parameter out of range");
  const ProcDesc* pd = nullptr;
  for (const auto& d : kProcs)
    if (std::strcmp(d.name, process) == 0) pd = &d;
  if (!pd) return fail(ME_ERR_PROCESS, std::string("unknown process ") + process);
  std::memset(kp, 0, sizeof(*kp));
  kp->cp.gs = std::sqrt(4.0 * M_PI * params->alpha_s);
  kp->cp.ee = std::sqrt(4.0 * M_PI * params->alpha);
  kp->cp.mt = params->mt;
  kp->avg_inv = 1.0 / pd->avg;
  kp->born_avg_inv = pd->born_pid >= 0 ? 1.0 / kProcs[pd->born_pid].avg : 0.0;
  kp->nlo_factor = 1.0;
  kp->xi_cut = params->xi_cut;
  kp->delta = params->delta;
  kp->xi_thr = params->xi_thr;
  kp->y_thr = params->y_thr;
  kp->me_eps = params->me_eps;
  kp->tol = params->tol;
  kp->cut = cuts_of(pd->pid, params);
  *pid = pd->pid;
  return ME_OK;
}

int me_internal_handle_process(const me_handle* h) { return h ? h->proc->pid : -1; }

int me_internal_device_kparams(const char* process, const me_params* params, me::KParams* kp, int* pid) {
  int rc = me_internal_kparams(process, params, kp, pid);
  if (rc != ME_OK) return rc;
  ColourTables* d_tab = nullptr;
  if ((rc = device_setup(params->device, &d_tab)) != ME_OK) return rc;
  kp->tab = d_tab;
  kp->item_budget = kItemBudget;
  return ME_OK;
}

int me_internal_process_id(const char* name) {
  if (!name) return -1;
  for (const auto& d : kProcs)
    if (std::strcmp(d.name, name) == 0) return d.pid;
  return -1;
}
