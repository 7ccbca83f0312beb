// Kernels of the event-parallel NLO hot path (templates; instantiated in me_inst_*.cu).
//
// Layout: momenta are structure-of-arrays float64 p[comp][leg][n] (comp = E,px,py,pz),
// so that consecutive events are consecutive addresses; weights are float64 w[n].
// A group of LPE consecutive lanes handles one event: the lanes split the helicity
// blocks (and, for the subtracted real, the Born-kinematics tasks) and reduce with warp
// shuffles.  Helicity sums run over one member of each pair (h, -h) -- the
// configurations with leg 0 at + -- and are doubled: flipping every helicity leaves the
// colour-summed squared amplitude (and every colour/spin-correlated one) unchanged for
// these tree amplitudes with real couplings (pinned against the oracle).  A helicity
// block (me_procs.cuh) is one configuration of the other legs with the four helicities
// of the heavy pair, evaluated with shared gluon currents and quark-line rows.  Born, real, soft and collinear terms are evaluated for every point and
// masked afterwards (Sec. 4.3, Algorithm 2), so a warp never diverges on cuts.
#pragma once
#include <algorithm>
#include <atomic>

#include "me_procs.cuh"
#include "me_tc.cuh"

// minimum resident 128-thread blocks per SM requested from the register allocator: 2
// gives the subtracted-real kernels up to 255 registers (8 warps per SM, fewer spills);
// measured against 3 (168 registers, 12 warps): 9.56 against 9.64 ms per c2 step
#ifndef ME_MINB
#define ME_MINB 2
#endif

namespace me {

constexpr int MAX_FLOW = 24;
constexpr int N_PAIRS = 10;  // unordered pairs (k<=l) of the 4 coloured legs of a 2->2 Born

// Device-resident process constants (written once per device at set-up):
// colour matrices (row-major NFLOW x NFLOW, in double and float) and the 2->2 Born
// colour correlators C^{kl} (pair order (0,0),(0,1),..,(3,3); [0] gg->tt, [1] uu->tt).
// U holds the upper triangle of the symmetric C with the off-diagonal entries doubled
// (U_aa = C_aa, U_ab = 2 C_ab for b > a, zero below), so that
// J^dagger C J = sum_a Re(J_a^* sum_{b >= a} U_ab J_b).
struct ColourTables {
  double C[P_COUNT][MAX_FLOW * MAX_FLOW];
  float Cf[P_COUNT][MAX_FLOW * MAX_FLOW];
  double U[P_COUNT][MAX_FLOW * MAX_FLOW];
  float Uf[P_COUNT][MAX_FLOW * MAX_FLOW];
  double Ccorr[2][N_PAIRS][4];
};

// Cuts of one configuration (Algorithm 2's passCuts, applied to each term at its own
// kinematics).  Each decision is an integer result taken in float64 with the operations
// in a fixed order and no contraction, so that any implementation doing the same
// operations on the same momenta decides alike:
//   CUT_PT      both heavy quarks (legs 2, 3):  px*px + py*py >= pt2_min
//   CUT_Y       both heavy quarks:  E + |pz| <= ey2 * (E - |pz|),  ey2 = exp(2 y_max)
//   CUT_AXIS    e+e-: the most energetic final parton m (first of equal energies):
//               pz*pz <= cos2_max * ((px*px + py*py) + pz*pz)  (thrust axis along p_m)
//   CUT_THRUST  e+e-: 2 E_m <= thrust_max * (E_0 + E_1)  (thrust T = 2 E_m / sqrt(s))
enum : unsigned { CUT_PT = 1u, CUT_Y = 2u, CUT_AXIS = 4u, CUT_THRUST = 8u };
struct Cuts {
  unsigned mask;  // 0: no cut
  double pt2_min, ey2, cos2_max, thrust_max;
};

struct KParams {
  Couplings cp;
  double avg_inv;       // 1 / (initial spin x colour average), x identical-particle factor
  double born_avg_inv;  // same for the underlying Born of a real process
  double nlo_factor;    // Born -> Born * factor (n-body NLO entry), else 1
  double xi_cut, delta; // FKS plus-distribution cut-offs
  double xi_thr, y_thr; // points with xi < xi_thr or 1-y < y_thr go to the FP64 path
  double me_eps;        // assumed relative error of a bulk-precision matrix element
  double tol;           // target relative accuracy of a weight
  int flag_unstable;    // 1: append unstable points to the rescue list
  int item_rescue;      // with flag_unstable: records and float64 items instead of the point list
  double item_budget;   // item rescue: residual error allowed, as a fraction of tol |W|
  Cuts cut;             // cuts of every term (mask 0: none)
  const ColourTables* tab;
};

template <typename T> __device__ __forceinline__ const T* ctab(const ColourTables* t, int pid);
template <> __device__ __forceinline__ const double* ctab<double>(const ColourTables* t, int pid) { return t->C[pid]; }
template <> __device__ __forceinline__ const float* ctab<float>(const ColourTables* t, int pid) { return t->Cf[pid]; }
template <typename T> __device__ __forceinline__ const T* utab(const ColourTables* t, int pid);
template <> __device__ __forceinline__ const double* utab<double>(const ColourTables* t, int pid) { return t->U[pid]; }
template <> __device__ __forceinline__ const float* utab<float>(const ColourTables* t, int pid) { return t->Uf[pid]; }

template <int PID, typename T>
__device__ __forceinline__ T colour_sum(const ColourTables* tab, const cx<T>* J) {
  constexpr int NF = Proc<PID>::NFLOW;
  T s = T(0);
  if constexpr (NF <= 6) {
    // triangular form: NF (NF + 1) + 2 NF multiply-adds instead of 2 NF^2 + 2 NF
    const T* __restrict__ Um = utab<T>(tab, PID);
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      const T d = Um[a * NF + a];
      T zr = d * J[a].re, zi = d * J[a].im;
#pragma unroll
      for (int b = a + 1; b < NF; ++b) {
        const T c = Um[a * NF + b];
        zr += c * J[b].re;
        zi += c * J[b].im;
      }
      s += J[a].re * zr + J[a].im * zi;
    }
    return s;
  }
  const T* __restrict__ Cm = ctab<T>(tab, PID);
#pragma unroll 4
  for (int a = 0; a < NF; ++a) {
    T zr = T(0), zi = T(0);
#pragma unroll 8
    for (int b = 0; b < NF; ++b) {
      const T c = Cm[a * NF + b];
      zr += c * J[b].re;
      zi += c * J[b].im;
    }
    s += J[a].re * zr + J[a].im * zi;
  }
  return s;
}

// J^dagger M J for a real symmetric 2x2 matrix M (row-major)
template <typename T>
__device__ __forceinline__ T quad2(const T* M, const cx<T>* J) {
  return M[0] * norm2(J[0]) + M[3] * norm2(J[1]) + T(2) * M[1] * (J[0].re * J[1].re + J[0].im * J[1].im);
}

template <int LPE, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int o = LPE / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, LPE);
  return v;
}

template <int LPE>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (LPE == 32) {
    return 0xffffffffu;
  } else {
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << LPE) - 1u) << (lane & ~(unsigned)(LPE - 1));
  }
}

template <int NEXT>
__device__ __forceinline__ void load_event(const double* __restrict__ p, long n, long i, r4<double>* k) {
#pragma unroll
  for (int l = 0; l < NEXT; ++l) {
    k[l].e = __ldg(p + (0L * NEXT + l) * n + i);
    k[l].x = __ldg(p + (1L * NEXT + l) * n + i);
    k[l].y = __ldg(p + (2L * NEXT + l) * n + i);
    k[l].z = __ldg(p + (3L * NEXT + l) * n + i);
  }
}

// ---------------------------------------------------------------- cuts
__device__ __forceinline__ bool heavy_pass(const r4<double>& q, const Cuts& c) {
  bool ok = true;
  if (c.mask & CUT_PT) ok = ok && __dadd_rn(__dmul_rn(q.x, q.x), __dmul_rn(q.y, q.y)) >= c.pt2_min;
  if (c.mask & CUT_Y) {
    const double a = fabs(q.z);
    ok = ok && __dadd_rn(q.e, a) <= __dmul_rn(c.ey2, __dsub_rn(q.e, a));
  }
  return ok;
}

// passCuts of a configuration k of process PID (or of a Born counter-event of it)
template <int PID>
__device__ __forceinline__ bool pass_cuts(const r4<double>* k, const Cuts& c) {
  if constexpr (PID == P_EE_UU || PID == P_EE_UUG) {
    r4<double> m = k[2];
#pragma unroll
    for (int i = 3; i < Proc<PID>::NEXT; ++i)
      if (k[i].e > m.e) m = k[i];
    bool ok = true;
    if (c.mask & CUT_AXIS) {
      const double t = __dadd_rn(__dmul_rn(m.x, m.x), __dmul_rn(m.y, m.y));
      const double z2 = __dmul_rn(m.z, m.z);
      ok = ok && z2 <= __dmul_rn(c.cos2_max, __dadd_rn(t, z2));
    }
    if (c.mask & CUT_THRUST) ok = ok && 2.0 * m.e <= __dmul_rn(c.thrust_max, __dadd_rn(k[0].e, k[1].e));
    return ok;
  } else {
    return heavy_pass(k[2], c) && heavy_pass(k[3], c);
  }
}

// ---------------------------------------------------------------- tree |M|^2
// float32 trees of 2 -> 2 processes fit 128 registers: 4 blocks per SM (16 warps) hide
// their float64 preparation better than the 2 blocks of the heavier kernels
// (gg -> t tbar Born: 0.122 against 0.132 ms per 2^20 points)
template <int PID, typename T>
constexpr int tree_min_blocks() {
  return (Proc<PID>::NEXT == 4 && std::is_same<T, float>::value) ? 4 : ME_MINB;
}

// out[i] = wgt[i] * |M|^2(p_i) * nlo_factor.  `count` (optional): the number of events,
// read on the device; `idx` (optional): the list of events to process (its length in
// `count`).  Momenta have stride n either way.  (g g -> t tbar g g in float32 runs
// k_tree_tc4 below instead.)
template <int PID, typename T, int LPE>
__global__ void __launch_bounds__(128, tree_min_blocks<PID, T>()) k_tree(const double* __restrict__ p, const double* __restrict__ wgt,
                                                       long n, double* __restrict__ out, KParams kp,
                                                       const int* __restrict__ idx, const int* __restrict__ count) {
  static_assert(!(PID == P_GG_TTGG && std::is_same<T, float>::value), "float g g -> t tbar g g runs k_tree_tc4");
  constexpr int NEXT = Proc<PID>::NEXT;
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) / LPE;
  const int lane = threadIdx.x % LPE;
  const long nev = count ? (long)*count : n;
  if (gid >= nev) return;
  const long ev = idx ? (long)idx[gid] : gid;
  r4<double> k[NEXT];
  load_event<NEXT>(p, n, ev, k);
  // Algorithm 2: every point is evaluated, and zeroed below where it fails the cuts
  const bool pass = !kp.cut.mask || pass_cuts<PID>(k, kp.cut);
  const Kin<PID, T> K = prepare<PID, T>(k, kp.cp);
  T acc = T(0);
  for (int b = lane; b < n_live_blocks<PID>(); b += LPE)
    amplitude_block<PID, T>(K, live_block_hel<PID>(b), kp.cp,
                            [&](int, const cx<T>* J) { acc += colour_sum<PID, T>(kp.tab, J); });
  const double tot = 2.0 * (double)group_sum<LPE>(acc, group_mask<LPE>());
  if (lane == 0) {
    const double w = wgt ? wgt[ev] : 1.0;
    out[ev] = pass ? w * tot * kp.avg_inv * kp.nlo_factor : 0.0;
  }
}

// ---------------------------------------------------------------- g g -> t tbar g g, float32, tensor cores
// Four lanes share one event and one helicity block at a time (me_procs.cuh: the gluon
// helicities fixed, the four (t, tbar) helicities open):
//  1. the 34 gluon four-vectors of the block -- polarisations e[4], ordered currents
//     J(xy) (6, x < y), J(xyz) (12, one of each reversed pair), J(wxyz) (12, w < z) --
//     are built cooperatively (a quarter each) into the event's shared-memory area;
//  2. lane w extends the quark line for the six orderings that start with gluon w,
//     U(w) -> U(wx) -> U(wxy), for both top helicities, and writes the partial
//     amplitudes of both antitop helicities into shared-memory rows;
//  3. one warp-wide tensor-core colour sum (me_tc.cuh) takes the warp's 32 rows
//     (8 events x 4 heavy-pair helicities): lane 4e + h receives helicity h of event e.
// Everything a lane needs stays on chip, so the 5e5 flops of an event run from registers
// and shared memory.  In a warp that holds the end of the batch, events past it compute
// a fixed finite configuration and are discarded, so every warp-wide step stays
// converged; warps entirely past the end return at once.
constexpr int TC4_EV_FLOATS = 276;  // 34 four-vectors x 8 floats, padded so 8 events hit distinct banks
constexpr int TC4_ROW = 25;         // floats per amplitude row (24 flows, padded)
constexpr int TC4_WARP_FLOATS = 8 * TC4_EV_FLOATS + 2 * 32 * TC4_ROW;
constexpr int TC4_SMEM_PER_WARP = TC4_WARP_FLOATS * 4 + TC_SMEM_PER_WARP;
constexpr int TC4_THREADS = 128;
constexpr int TC4_SMEM = (TC4_THREADS / 32) * TC4_SMEM_PER_WARP;

// J(xyz) representatives, slot t = 3 * (missing gluon) + (position of the middle gluon
// among the three in increasing order); packed x | y << 4 | z << 8, x < z
__constant__ short kJ3Rep[12] = {0x312, 0x321, 0x231, 0x302, 0x320, 0x230,
                                 0x301, 0x310, 0x130, 0x201, 0x210, 0x120};
// J(wxyz) representatives (w < z), enumerated by w, then x, then y: packed w | x<<4 | y<<8 | z<<12
__constant__ short kJ4Rep[12] = {0x3210, 0x2310, 0x3120, 0x1320, 0x2130, 0x1230,
                                 0x3201, 0x2301, 0x3021, 0x2031, 0x3102, 0x3012};
// ordering f (lexicographic) -> +-(1 + representative of J(wxyz)); minus: reversed, J = -J(rep)
__constant__ signed char kJ4OfOrdering[24] = {1,  2,  3,   4,  5,  6,  7,   8,  9,  -6, 10, -4,
                                              11, -10, 12, -5, -8, -2, -12, -9, -11, -3, -7, -1};

__device__ __forceinline__ void st_c4(float* b, int slot, const c4<float>& v) {
  float4* p = reinterpret_cast<float4*>(b + 8 * slot);
  p[0] = make_float4(v.v[0].re, v.v[0].im, v.v[1].re, v.v[1].im);
  p[1] = make_float4(v.v[2].re, v.v[2].im, v.v[3].re, v.v[3].im);
}
__device__ __forceinline__ c4<float> ld_c4(const float* b, int slot) {
  const float4* p = reinterpret_cast<const float4*>(b + 8 * slot);
  const float4 a = p[0], c = p[1];
  return c4<float>{{{a.x, a.y}, {a.z, a.w}, {c.x, c.y}, {c.z, c.w}}};
}
__device__ __forceinline__ int pair_slot(int x, int y) {  // x < y
  return 4 + (x == 0 ? y - 1 : (x == 1 ? y + 1 : 5));
}
__device__ __forceinline__ c4<float> ld_j2(const float* b, int x, int y) {
  c4<float> J = ld_c4(b, pair_slot(x < y ? x : y, x < y ? y : x));
  if (x > y) cscale(J, -1.0f);
  return J;
}
// the same eight floats read as the chiral combinations (V0 - V3, V0 + V3, V1 - i V2,
// V1 + i V2) once a slot has been converted in place for the quark lines
__device__ __forceinline__ sl4<float> ld_sl4(const float* b, int slot) {
  const float4* p = reinterpret_cast<const float4*>(b + 8 * slot);
  const float4 a = p[0], c = p[1];
  return sl4<float>{{a.x, a.y}, {a.z, a.w}, {c.x, c.y}, {c.z, c.w}};
}
__device__ __forceinline__ void slash_in_place(float* b, int slot) {
  const sl4<float> S = slashed(ld_c4(b, slot));
  float4* p = reinterpret_cast<float4*>(b + 8 * slot);
  p[0] = make_float4(S.a.re, S.a.im, S.b.re, S.b.im);
  p[1] = make_float4(S.c.re, S.c.im, S.d.re, S.d.im);
}
__device__ __forceinline__ sl4<float> ld_sj2(const float* b, int x, int y) {
  sl4<float> S = ld_sl4(b, pair_slot(x < y ? x : y, x < y ? y : x));
  if (x > y) S = sl4<float>{-S.a, -S.b, -S.c, -S.d};
  return S;
}
__device__ __forceinline__ int triple_slot(int x, int y, int z) {  // any order: J(zyx) = J(xyz)
  const int miss = 6 - x - y - z;
  const int a = miss == 0 ? 1 : 0, c = miss == 3 ? 2 : 3;
  return 10 + 3 * miss + (y == a ? 0 : (y == c ? 2 : 1));
}

template <int LPE>
__global__ void __launch_bounds__(TC4_THREADS, 2) k_tree_tc4(const double* __restrict__ p, const double* __restrict__ wgt,
                                                             long n, double* __restrict__ out, KParams kp,
                                                             const int* __restrict__ idx, const int* __restrict__ count) {
  static_assert(LPE == 4, "four lanes per event");
  constexpr int PID = P_GG_TTGG;
  extern __shared__ __align__(16) float tc4_smem[];
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  float* wsm = tc4_smem + warp * (TC4_SMEM_PER_WARP / 4);
  float* cur = wsm + (wl >> 2) * TC4_EV_FLOATS;         // this event's four-vectors
  float* are = wsm + 8 * TC4_EV_FLOATS;                 // amplitude rows, real parts [32][TC4_ROW]
  float* aim = are + 32 * TC4_ROW;                      // imaginary parts
  unsigned char* stage = reinterpret_cast<unsigned char*>(wsm + TC4_WARP_FLOATS);
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) / 4;
  const int lane = threadIdx.x & 3;
  const long nev = count ? (long)*count : n;
  // a warp whose eight events all lie past the batch leaves together (every
  // synchronisation below is warp-wide), so a grid sized for a capacity costs little
  if (((long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / 4 >= nev) return;
  const bool active = gid < nev;
  const long ev = active ? (idx ? (long)idx[gid] : gid) : 0;
  r4<double> k[6];
  if (active) {
    load_event<6>(p, n, ev, k);
  } else {
    const double d[6][4] = {{1000, 0, 0, 1000},     {1000, 0, 0, -1000},     {600, 100, 200, 300},
                            {700, -150, -100, 200}, {400, 30, -80, -300}, {300, 20, -20, -200}};
#pragma unroll
    for (int l = 0; l < 6; ++l) k[l] = r4<double>{d[l][0], d[l][1], d[l][2], d[l][3]};
  }
  const TcColourB cb = tc_load_colour(kp.tab->C[PID]);
  const Kin<PID, float> K = prepare<PID, float>(k, kp.cp);
  const float g = (float)kp.cp.gs, mt = (float)kp.cp.mt;
  const r4<float>* q = K.q;
  const r4<float> kt = K.pl[2];
  const c4<float> v[2] = {spinor_v_of(K.wtb, -1), spinor_v_of(K.wtb, 1)};
  constexpr int LEG[4] = {0, 1, 4, 5};
  float acc = 0.0f;
  for (int b = 0; b < n_live_blocks<PID>(); ++b) {
    const int hb = live_block_hel<PID>(b);
    // 1. polarisation of gluon `lane`
    st_c4(cur, lane, polvec_of(K.wg[lane], hel_of(hb, LEG[lane]), LEG[lane] >= 2));
    __syncwarp();
    // 2. pair currents: slots 4 + lane and 8 + lane (< 10)
    for (int pp = lane; pp < 6; pp += 4) {
      const int x = pp < 3 ? 0 : (pp < 5 ? 1 : 2);
      const int y = pp < 3 ? pp + 1 : (pp < 5 ? pp - 1 : 3);
      st_c4(cur, 4 + pp, vvv(ld_c4(cur, x), ld_c4(cur, y), -q[x], -q[y], -g * K.ig[(1 << x) | (1 << y)]));
    }
    __syncwarp();
    // 3. triple currents
    for (int t = lane; t < 12; t += 4) {
      const int r = kJ3Rep[t], x = r & 15, y = (r >> 4) & 15, z = r >> 8;
      const int S = (1 << x) | (1 << y) | (1 << z);
      const c4<float> ex = ld_c4(cur, x), ey = ld_c4(cur, y), ez = ld_c4(cur, z);
      const float c3 = -g * K.ig[S];
      c4<float> J = vvv(ex, ld_j2(cur, y, z), -q[x], -(q[y] + q[z]), c3);
      vvv_acc(J, ld_j2(cur, x, y), ez, -(q[x] + q[y]), -q[z], c3);
      caxpy(J, g * g * K.ig[S], vvvv_ordered(ex, ey, ez));
      st_c4(cur, 10 + t, J);
    }
    __syncwarp();
    // 4. quadruple currents
    for (int t = lane; t < 12; t += 4) {
      const int r = kJ4Rep[t], w = r & 15, x = (r >> 4) & 15, y = (r >> 8) & 15, z = r >> 12;
      const c4<float> ew = ld_c4(cur, w), ez = ld_c4(cur, z);
      const c4<float> jwx = ld_j2(cur, w, x), jxy = ld_j2(cur, x, y), jyz = ld_j2(cur, y, z);
      const float c3 = -g * K.ig[15];
      c4<float> J = vvv(ew, ld_c4(cur, triple_slot(x, y, z)), -q[w], -(q[x] + q[y] + q[z]), c3);
      vvv_acc(J, jwx, jyz, -(q[w] + q[x]), -(q[y] + q[z]), c3);
      vvv_acc(J, ld_c4(cur, triple_slot(w, x, y)), ez, -(q[w] + q[x] + q[y]), -q[z], c3);
      c4<float> V = vvvv_ordered(ew, ld_c4(cur, x), jyz);
      cadd(V, vvvv_ordered(ew, jxy, ez));
      cadd(V, vvvv_ordered(jwx, ld_c4(cur, y), ez));
      caxpy(J, g * g * K.ig[15], V);
      st_c4(cur, 22 + t, J);
    }
    __syncwarp();
    // the quark lines only slash the 34 vectors against rows: convert them in place
    for (int sl = lane; sl < 34; sl += 4) slash_in_place(cur, sl);
    __syncwarp();
    // 5. quark line for the orderings starting with gluon w = lane
    const int w = lane;
    for (int ht = 0; ht < 2; ++ht) {
      const c4<float> ub = dbar(spinor_u_of(K.wt, ht ? 1 : -1));
      const int row0 = (wl & ~3) + 2 * ht;  // rows of (this event, ht, hv = 0 / 1)
      const c4<float> U1 = row_prop(row_slash(ub, ld_sl4(cur, w)), scaled_prop(kt + q[w], mt, -g * K.iq[1 << w]));
      // every lane runs the same 3 x 2 iterations (no lane idles on a skipped index):
      // x is the kx-th gluon other than w, y the ky-th other than w and x, in increasing
      // order, so f counts the orderings w x y z as the ordering tables do
      int f = 6 * w;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int x = kx + (kx >= w ? 1 : 0);
        c4<float> r2 = row_slash(ub, ld_sj2(cur, w, x));
        row_slash_acc(r2, U1, ld_sl4(cur, x));
        const c4<float> U2 = row_prop(r2, scaled_prop(kt + q[w] + q[x], mt, -g * K.iq[(1 << w) | (1 << x)]));
        const int lo = w < x ? w : x, hi = w < x ? x : w;
#pragma unroll
        for (int ky = 0; ky < 2; ++ky) {
          int y = ky;
          if (y >= lo) ++y;
          if (y >= hi) ++y;
          const int z = 6 - w - x - y;
          c4<float> r3 = row_slash(ub, ld_sl4(cur, triple_slot(w, x, y)));
          row_slash_acc(r3, U1, ld_sj2(cur, x, y));
          row_slash_acc(r3, U2, ld_sl4(cur, y));
          const c4<float> U3 =
              row_prop(r3, scaled_prop(kt + q[w] + q[x] + q[y], mt, -g * K.iq[(1 << w) | (1 << x) | (1 << y)]));
          const int s4 = kJ4OfOrdering[f];
          c4<float> R = row_slash(ub, ld_sl4(cur, 22 + (s4 > 0 ? s4 : -s4) - 1));
          if (s4 < 0) R = cneg(R);
          row_slash_acc(R, U1, ld_sl4(cur, triple_slot(x, y, z)));
          row_slash_acc(R, U2, ld_sj2(cur, y, z));
          row_slash_acc(R, U3, ld_sl4(cur, z));
#pragma unroll
          for (int hv = 0; hv < 2; ++hv) {
            const cx<float> a = times_i(spdot(R, v[hv])) * g;
            are[(row0 + hv) * TC4_ROW + f] = a.re;
            aim[(row0 + hv) * TC4_ROW + f] = a.im;
          }
          ++f;
        }
      }
    }
    __syncwarp();
    // 6. colour sum of row wl (this event, heavy-pair helicity lane) on the tensor cores
    cx<float> J[TC_NF];
#pragma unroll
    for (int fl = 0; fl < TC_NF; ++fl) J[fl] = cx<float>{are[wl * TC4_ROW + fl], aim[wl * TC4_ROW + fl]};
    const float sres = tc_colour_sum(J, cb, stage);
    if (active) acc += sres;
    __syncwarp();
  }
  const double tot = 2.0 * (double)group_sum<4>(acc, group_mask<4>());
  if (active && lane == 0) {
    const double w8 = wgt ? wgt[ev] : 1.0;
    bool pass = true;
    if (kp.cut.mask) {
      r4<double> kc[6];
      load_event<6>(p, n, ev, kc);
      pass = pass_cuts<P_GG_TTGG>(kc, kp.cut);
    }
    out[ev] = pass ? w8 * tot * kp.avg_inv * kp.nlo_factor : 0.0;
  }
}

// ---------------------------------------------------------------- FKS kinematics (double)
// Float64 throughout (the maps fix the counter-event kinematics that the subtraction
// compares with the real).  GB300 issues float64 at 1/64 of the float32 rate, and a
// float64 division or square root costs ~10 pipe instructions, so the maps use reciprocal
// square roots and shared reciprocals, and boost with the system momentum and mass.

// p (given in the rest frame of a system with momentum Q, mass M) in the frame where the
// system has momentum Q:  E' = (E Q0 + Q.p)/M,  p' = p + Q (E' + E)/(Q0 + M).
// sgn = -1 boosts the other way (from the frame of Q into its rest frame).
__device__ __forceinline__ r4<double> boost_by(const r4<double>& p, const r4<double>& Q, double inv_m, double m,
                                               double sgn) {
  const double qp = Q.x * p.x + Q.y * p.y + Q.z * p.z;
  const double e = (p.e * Q.e + sgn * qp) * inv_m;
  const double c = sgn * (e + p.e) / (Q.e + m);
  return r4<double>{e, p.x + c * Q.x, p.y + c * Q.y, p.z + c * Q.z};
}
// the same with 1 / (Q0 + M) given (several vectors boosted by one system)
__device__ __forceinline__ r4<double> boost_by_r(const r4<double>& p, const r4<double>& Q, double inv_m,
                                                 double inv_qm, double sgn) {
  const double qp = Q.x * p.x + Q.y * p.y + Q.z * p.z;
  const double e = (p.e * Q.e + sgn * qp) * inv_m;
  const double c = sgn * (e + p.e) * inv_qm;
  return r4<double>{e, p.x + c * Q.x, p.y + c * Q.y, p.z + c * Q.z};
}

__device__ __forceinline__ void unit3(const r4<double>& p, double& x, double& y, double& z) {
  const double a = rsqrt(p.x * p.x + p.y * p.y + p.z * p.z);
  x = p.x * a;
  y = p.y * a;
  z = p.z * a;
}

constexpr double PI = 3.14159265358979323846;
constexpr double CF_ = 4.0 / 3.0;
constexpr double CA_ = 3.0;

// Initial-state FKS sectors (i = gluon leg 4, j = beam 0 or 1) of 2 -> Q Qbar g.
struct IsrKin {
  double xi, iz, y[2], S[2], K, K0;  // iz = 1 / (1 - xi)
  r4<double> soft[4];     // soft Born: beams, heavy pair at sqrt(s) along n*
  // collinear Born of sector 1: beam 1 scaled by z = 1 - xi.  That of sector 2 (beam 2
  // scaled) is the same 2 -> 2 configuration boosted along the beam axis, and everything
  // evaluated there -- the unpolarised Born and the Born with a gluon polarised along the
  // transverse direction (0, cos phi, sin phi, 0) -- is invariant under that boost.
  r4<double> coll[4];
  double qdir[3];         // gluon direction
  double cphi, sphi;      // gluon azimuth
  // cuts (Algorithm 2) of the soft counter-event and of each sector's collinear one (its
  // beam scaled by z): the two collinear Borns differ by a boost along the beam, which
  // changes the heavy quarks' rapidities
  bool cut_s, cut_c[2];
};

__device__ __forceinline__ void isr_map(const r4<double>* k, double mass, IsrKin& o, const Cuts& cut) {
  const double rs = k[0].e + k[1].e, irs = 1.0 / rs, s = rs * rs, is = irs * irs;
  o.xi = 2.0 * k[4].e * irs;
  unit3(k[4], o.qdir[0], o.qdir[1], o.qdir[2]);
  double b0[3], b1[3];
  unit3(k[0], b0[0], b0[1], b0[2]);
  unit3(k[1], b1[0], b1[1], b1[2]);
  o.y[0] = o.qdir[0] * b0[0] + o.qdir[1] * b0[1] + o.qdir[2] * b0[2];
  o.y[1] = o.qdir[0] * b1[0] + o.qdir[1] * b1[1] + o.qdir[2] * b1[2];
  const double d0 = 1.0 - o.y[0], d1 = 1.0 - o.y[1];
  const double idd = 1.0 / (d0 + d1);
  o.S[0] = d1 * idd;
  o.S[1] = d0 * idd;
  const double pt2 = o.qdir[0] * o.qdir[0] + o.qdir[1] * o.qdir[1];
  const double ipt = pt2 > 0.0 ? rsqrt(pt2) : 0.0;
  o.cphi = pt2 > 0.0 ? o.qdir[0] * ipt : 1.0;
  o.sphi = pt2 > 0.0 ? o.qdir[1] * ipt : 0.0;
  // heavy-pair rest-frame direction of the quark
  const r4<double> Q = k[0] + k[1] - k[4];
  const double Q2 = mdot(Q, Q), iMQ = rsqrt(Q2);
  const r4<double> ks = boost_by(k[2], Q, iMQ, Q2 * iMQ, -1.0);
  double n[3];
  unit3(ks, n[0], n[1], n[2]);
  const double m4 = 4.0 * mass * mass;
  const double b2 = 1.0 - m4 * is, ibeta = rsqrt(b2), beta = b2 * ibeta;
  o.soft[0] = k[0];
  o.soft[1] = k[1];
  const double e = 0.5 * rs, pa = 0.5 * rs * beta;
  o.soft[2] = r4<double>{e, pa * n[0], pa * n[1], pa * n[2]};
  o.soft[3] = r4<double>{e, -pa * n[0], -pa * n[1], -pa * n[2]};
  const double z = 1.0 - o.xi;
  o.iz = 1.0 / z;
  const double sz = s * z, iM = rsqrt(sz), M = sz * iM;
  const double bQ = sqrt(fmax(0.0, 1.0 - m4 * is * o.iz));
  const double eQ = 0.5 * M, pQ = 0.5 * M * bQ;
  const r4<double> tr{eQ, pQ * n[0], pQ * n[1], pQ * n[2]};
  const r4<double> tbr{eQ, -pQ * n[0], -pQ * n[1], -pQ * n[2]};
  o.coll[0] = scale(z, k[0]);
  o.coll[1] = k[1];
  const r4<double> Qc = o.coll[0] + o.coll[1];
  const double Mc2 = mdot(Qc, Qc), iMc = rsqrt(Mc2), iqm = 1.0 / (Qc.e + Mc2 * iMc);
  o.coll[2] = boost_by_r(tr, Qc, iMc, iqm, 1.0);
  o.coll[3] = boost_by_r(tbr, Qc, iMc, iqm, 1.0);
  o.cut_s = o.cut_c[0] = o.cut_c[1] = true;
  if (cut.mask) {
    o.cut_s = heavy_pass(o.soft[2], cut) && heavy_pass(o.soft[3], cut);
    o.cut_c[0] = heavy_pass(o.coll[2], cut) && heavy_pass(o.coll[3], cut);
    const r4<double> Q1 = k[0] + scale(z, k[1]);
    const double M12 = mdot(Q1, Q1), iM1 = rsqrt(M12);
    o.cut_c[1] = heavy_pass(boost_by(tr, Q1, iM1, M12 * iM1, 1.0), cut) &&
                 heavy_pass(boost_by(tbr, Q1, iM1, M12 * iM1, 1.0), cut);
  }
  constexpr double i64pi3 = 1.0 / (64.0 * PI * PI * PI);
  o.K = s * bQ * i64pi3 * ibeta;
  o.K0 = s * i64pi3;
}

// Final-state FKS sectors (i = gluon leg 4, j = leg 2 or 3) of massless 2 -> 3.
struct FsrKin {
  double xi, y[2], S[2], K[2], K0, K1;
  r4<double> born[2][4];
  double qdir[3];
};

__device__ __forceinline__ void fsr_map(const r4<double>* k, FsrKin& o) {
  const double rs = k[0].e + k[1].e, s = rs * rs;
  o.xi = 2.0 * k[4].e / rs;
  unit3(k[4], o.qdir[0], o.qdir[1], o.qdir[2]);
  double nj[2][3];
  unit3(k[2], nj[0][0], nj[0][1], nj[0][2]);
  unit3(k[3], nj[1][0], nj[1][1], nj[1][2]);
  double c[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) c[j] = o.qdir[0] * nj[j][0] + o.qdir[1] * nj[j][1] + o.qdir[2] * nj[j][2];
  const double d0 = 1.0 - c[0], d1 = 1.0 - c[1];
  o.S[0] = d1 / (d0 + d1);
  o.S[1] = d0 / (d0 + d1);
  const double e = 0.5 * rs;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    o.y[j] = c[j];
    o.born[j][0] = k[0];
    o.born[j][1] = k[1];
    const r4<double> a{e, e * nj[j][0], e * nj[j][1], e * nj[j][2]};
    const r4<double> b{e, -e * nj[j][0], -e * nj[j][1], -e * nj[j][2]};
    o.born[j][2 + j] = a;
    o.born[j][3 - j] = b;
    const double den = 2.0 - o.xi * (1.0 - o.y[j]);
    o.K[j] = s * (1.0 - o.xi) / (16.0 * PI * PI * PI * den * den);
  }
  o.K0 = s / (64.0 * PI * PI * PI);
  o.K1 = s * (1.0 - o.xi) / (64.0 * PI * PI * PI);
}

__device__ __forceinline__ double eik(const r4<double>& a, const r4<double>& b, const double* q) {
  const r4<double> qq{1.0, q[0], q[1], q[2]};
  return mdot(a, b) / (mdot(a, qq) * mdot(b, qq));
}

// ---------------------------------------------------------------- real - counterterms
// One point of the subtracted real, summed over FKS sectors (ME units):
//   W_j = R S_j - [Th_s G(0,y) + Th_c G(xi,1) - Th_s Th_c G(0,1)] / (xi^2 (1-y) K),
// with the error scale of the stability test.  The LPE lanes of a group evaluate one
// point together and all return the same result.
//
// W is linear in its matrix-element ingredients -- the real's helicity blocks R_b
// (R = sum_b R_b) and the Born values of the counterterms (for initial-state sectors:
// the eikonal-weighted soft Born E, the soft Born B_s, the collinear Born B_c and, for
// g g, the two spin-correlated Borns B_p; for final-state sectors the Born B_j of each
// sector) -- with float64 coefficients fixed by the FKS maps:  W = sum_i a_i v_i.  The
// item rescue re-evaluates in float64 only the ingredients whose float32 error the
// point's tolerance cannot absorb, and recombines W from the coefficients.
template <int PID>
struct RealLayout {
  static constexpr int NB = n_live_blocks<PID>();                                   // real's blocks
  static constexpr int NBV = PID == P_EE_UUG ? 2 : (PID == P_GG_TTG ? 5 : 3);      // Born values
  static constexpr int NI = NB + NBV;
};
constexpr int MAX_ITEMS = 9;

struct RealSubOut {
  double W;     // subtracted real, summed over sectors
  double mag;   // error scale: |R S| + |CT_coll| + |CT_soft - CT_softcoll| per sector
  double magR;  // its real part, sum_j |R S_j|
  double y[2];  // y_j of both sectors (collinear resolution of the test)
  bool near;    // inside xi_thr / y_thr of an active counterterm
};

// Ingredients and coefficients of one point for the item rescue (group lane 0).
struct RealItems {
  double a[MAX_ITEMS];  // W = sum_i a_i v_i
  double v[MAX_ITEMS];  // bulk-precision values: R blocks, then the Born values
  double born_scale;    // error scale of the Born values together (as in RealSubOut::mag)
};

// Eikonal-weighted colour-correlation matrix of the soft counter-event (2x2, row-major):
// E = sum_{k,l} w_kl C^{kl}, w_kl = (p_k.p_l) / ((p_k.q)(p_l.q)), q = (1, gluon direction),
// over the four coloured legs of the 2 -> 2 Born (k = l included); four reciprocals.
template <int BPID>
__device__ __forceinline__ void isr_eikonal_matrix(const IsrKin& f, const KParams& kp, double* E) {
  const int ci = (BPID == P_GG_TT) ? 0 : 1;
  E[0] = E[1] = E[2] = E[3] = 0.0;
  const r4<double> qq{1.0, f.qdir[0], f.qdir[1], f.qdir[2]};
  double iaq[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) iaq[a] = 1.0 / mdot(f.soft[a], qq);
  int pr = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b, ++pr) {
      const double w = mdot(f.soft[a], f.soft[b]) * iaq[a] * iaq[b] * (a == b ? 1.0 : 2.0);
#pragma unroll
      for (int q = 0; q < 4; ++q) E[q] += w * kp.tab->Ccorr[ci][pr][q];
    }
}

// Born values of the soft counter-event kb: vE = E-weighted correlated Born (multiplies
// -4 g^2 / s in the soft limit), vS = plain Born.  Every sum ran over one helicity of
// each flipped pair (|M(h)|^2 = |M(-h)|^2), hence the factor 2.
template <int BPID, typename T, int LPE>
__device__ __forceinline__ void isr_soft_pair(const r4<double>* kb, const double* E, const KParams& kp, int lane,
                                              unsigned mask, double& vE, double& vS) {
  const T Et[4] = {(T)E[0], (T)E[1], (T)E[2], (T)E[3]};
  T aE = T(0), aS = T(0);
  const Kin<BPID, T> KB = prepare<BPID, T>(kb, kp.cp);
  for (int b = lane; b < n_live_blocks<BPID>(); b += LPE)
    amplitude_block<BPID, T>(KB, live_block_hel<BPID>(b), kp.cp, [&](int, const cx<T>* J) {
      aE += quad2(Et, J);
      aS += colour_sum<BPID, T>(kp.tab, J);
    });
  const double bav = 2.0 * kp.born_avg_inv;
  vE = (double)group_sum<LPE>(aE, mask) * bav;
  vS = (double)group_sum<LPE>(aS, mask) * bav;
}

// Born values of the collinear counter-event kb: v[0] = B_c (plain), and for g g the
// spin-correlated Borns v[1], v[2] with gluon 0 or 1 polarised along the transverse
// direction (0, cos phi, sin phi, 0) of the emission.
template <int BPID, typename T, int LPE>
__device__ __forceinline__ void isr_coll_set(const r4<double>* kb, double cphi, double sphi, const KParams& kp,
                                             int lane, unsigned mask, double* v, bool want0 = true,
                                             bool want1 = true) {
  c4<T> eperp;
  eperp.v[0] = cx<T>{T(0), T(0)};
  eperp.v[1] = cx<T>{(T)cphi, T(0)};
  eperp.v[2] = cx<T>{(T)sphi, T(0)};
  eperp.v[3] = cx<T>{T(0), T(0)};
  T aC = T(0), aP[2] = {T(0), T(0)};
  const Kin<BPID, T> KB = prepare<BPID, T>(kb, kp.cp);
  for (int b = lane; b < n_live_blocks<BPID>(); b += LPE)
    amplitude_block<BPID, T>(KB, live_block_hel<BPID>(b), kp.cp,
                             [&](int, const cx<T>* J) { aC += colour_sum<BPID, T>(kp.tab, J); });
  if constexpr (BPID == P_GG_TT) {
    // polarised gluon 0; gluon 1 fixed to +, the heavy pair free (the flip covers the rest)
    if (lane == 0 && want0)
      amplitude_block<BPID, T>(
          KB, 2, kp.cp, [&](int, const cx<T>* J) { aP[0] += colour_sum<BPID, T>(kp.tab, J); }, &eperp, 0);
    // polarised gluon 1, gluon 0 fixed to +: sector 2's spin-correlated Born, at the
    // same kinematics (invariant under the boost that relates the two sectors)
    if (lane == 1 % LPE && want1)
      amplitude_block<BPID, T>(
          KB, 1, kp.cp, [&](int, const cx<T>* J) { aP[1] += colour_sum<BPID, T>(kp.tab, J); }, &eperp, 1);
  }
  const double bav = 2.0 * kp.born_avg_inv;
  v[0] = (double)group_sum<LPE>(aC, mask) * bav;
  if constexpr (BPID == P_GG_TT) {
    v[1] = (double)group_sum<LPE>(aP[0], mask) * bav;
    v[2] = (double)group_sum<LPE>(aP[1], mask) * bav;
  }
}

// Born values of the initial-state counterterms: v[0] = E (eikonal-weighted soft Born),
// v[1] = B_s (soft Born), v[2] = B_c (collinear Born), v[3], v[4] = B_p (spin-correlated
// Borns, g g only).
template <int PID, typename T, int LPE>
__device__ __forceinline__ void isr_born_values(const IsrKin& f, const KParams& kp, int lane, unsigned mask,
                                                double* v) {
  constexpr int BPID = PID == P_GG_TTG ? P_GG_TT : P_UU_TT;
  double E[4];
  isr_eikonal_matrix<BPID>(f, kp, E);
  isr_soft_pair<BPID, T, LPE>(f.soft, E, kp, lane, mask, v[0], v[1]);
  // sector j's spin-correlated Born enters only where its collinear term is active (one
  // sector at most for delta <= 1); where that is sector 2 alone, the beams are swapped
  // (Bose symmetry of g g -> t tbar) so that every lane evaluates the gluon-0 block
  const bool w0 = BPID == P_GG_TT && f.y[0] > 1.0 - kp.delta && f.cut_c[0];
  const bool w1 = BPID == P_GG_TT && f.y[1] > 1.0 - kp.delta && f.cut_c[1];
  const bool sw = w1 && !w0;
  const r4<double> cb[4] = {sw ? f.coll[1] : f.coll[0], sw ? f.coll[0] : f.coll[1], f.coll[2], f.coll[3]};
  isr_coll_set<BPID, T, LPE>(cb, f.cphi, f.sphi, kp, lane, mask, v + 2, w0 || sw, w1 && !sw);
  if constexpr (BPID == P_GG_TT) {
    if (sw) {
      v[4] = v[3];
      v[3] = 0.0;
    }
  }
}

// The Born |M|^2 of e+e- -> u ubar at kb (a final-state counterterm's Born).
template <typename T, int LPE>
__device__ __forceinline__ double fsr_born_one(const r4<double>* kb, const KParams& kp, int lane, unsigned mask) {
  T aB = T(0);
  const Kin<P_EE_UU, T> KB = prepare<P_EE_UU, T>(kb, kp.cp);
  for (int b = lane; b < n_live_blocks<P_EE_UU>(); b += LPE)
    amplitude_block<P_EE_UU, T>(KB, live_block_hel<P_EE_UU>(b), kp.cp,
                                [&](int, const cx<T>* J) { aB += colour_sum<P_EE_UU, T>(kp.tab, J); });
  return 2.0 * (double)group_sum<LPE>(aB, mask) * kp.born_avg_inv;
}

// Born values of the final-state counterterms: v[j] = the Born at sector j's kinematics.
template <typename T, int LPE>
__device__ __forceinline__ void fsr_born_values(const FsrKin& f, const KParams& kp, int lane, unsigned mask,
                                                double* v) {
#pragma unroll
  for (int j = 0; j < 2; ++j) v[j] = fsr_born_one<T, LPE>(f.born[j], kp, lane, mask);
}

// One helicity block b of the real matrix element, colour-summed and averaged:
// R = sum over the live blocks.
template <int PID, typename T>
__device__ __forceinline__ double real_block_value(const Kin<PID, T>& K, int b, const KParams& kp) {
  T acc = T(0);
  amplitude_block<PID, T>(K, live_block_hel<PID>(b), kp.cp, [&](int, const cx<T>* J) { acc += colour_sum<PID, T>(kp.tab, J); });
  return 2.0 * (double)acc * kp.avg_inv;
}

// `items` (optional): filled with the coefficients and ingredient values on group lane 0
// (every lane of the group must pass it or none).
template <int PID, typename T, int LPE>
__device__ __forceinline__ RealSubOut real_sub_event(const double* __restrict__ p, long n, long ev, const KParams& kp,
                                                     int lane, unsigned mask, RealItems* items = nullptr) {
  constexpr int NEXT = Proc<PID>::NEXT;
  constexpr int NB = RealLayout<PID>::NB;
  constexpr int NBL = (NB + LPE - 1) / LPE;  // real blocks per lane
  r4<double> k[NEXT];
  load_event<NEXT>(p, n, ev, k);
  const double rs = k[0].e + k[1].e, s = rs * rs;
  const double g2 = kp.cp.gs * kp.cp.gs;
  // Algorithm 2's cut of the real term, at the real point
  const double cR = (!kp.cut.mask || pass_cuts<PID>(k, kp.cut)) ? 1.0 : 0.0;

  // real matrix element; lane l holds blocks l, l + LPE, ... (one copy of the block code:
  // the loop is not unrolled)
  double blk[NBL];
  double mine = 0.0;
  {
    const Kin<PID, T> K = prepare<PID, T>(k, kp.cp);
#pragma unroll 1
    for (int i = 0; i < NBL; ++i) {
      const int b = lane + i * LPE;
      const double v = b < NB ? real_block_value<PID, T>(K, b, kp) : 0.0;
      blk[i] = v;
      mine += v;
    }
  }
  const double R = group_sum<LPE>(mine, mask);

  double W = 0.0, mag = 0.0;
  double ysec[2] = {-1.0, -1.0};  // y_j of both sectors (collinear resolution of the flag)
  double xi_pt = 0.0;             // the emission's energy fraction
  bool near = false;
  double a_R = 0.0, ab[RealLayout<PID>::NBV] = {};  // coefficients of R and of the Born values
  double bv[RealLayout<PID>::NBV];
  if constexpr (PID == P_EE_UUG) {
    FsrKin f;
    fsr_map(k, f);
    ysec[0] = f.y[0];
    ysec[1] = f.y[1];
    xi_pt = f.xi;
    fsr_born_values<T, LPE>(f, kp, lane, mask, bv);
    const double* B = bv;
    // Algorithm 2's cuts: both counterterms of sector j at sector j's Born
    const bool cuts = kp.cut.mask != 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double cB = (!cuts || pass_cuts<P_EE_UU>(f.born[j], kp.cut)) ? 1.0 : 0.0;
      const double th_s = f.xi < kp.xi_cut ? cB : 0.0;
      // soft: sum_{kl} w_kl B_kl with B_23 = B_32 = -C_F B (massless diagonal terms vanish)
      const double cs = (1.0 - f.y[j]) * 0.5 * (1.0 + f.y[j]) * f.K0 * (-(4.0 * g2 / s) * 2.0 * eik(f.born[j][2], f.born[j][3], f.qdir) * (-CF_));
      const double cc = f.K1 * (2.0 / (s * (1.0 - f.xi))) * 2.0 * g2 * CF_ * (1.0 + (1.0 - f.xi) * (1.0 - f.xi));
      const double csc = f.K0 * (2.0 / s) * 2.0 * g2 * 2.0 * CF_;
      const double Gs = cs * B[j], Gc = cc * B[j], Gsc = csc * B[j];
      const double th_c = f.y[j] > 1.0 - kp.delta ? cB : 0.0;
      const double iden = 1.0 / (f.xi * f.xi * (1.0 - f.y[j]) * f.K[j]);
      const double ct = (th_s * Gs + th_c * Gc - th_s * th_c * Gsc) * iden;
      const double rsj = R * f.S[j] * cR;
      W += rsj - ct;
      // error scale: the real, the collinear term, and the soft pair (whose Borns are shared)
      mag += fabs(rsj) + fabs(th_c * Gc * iden) + fabs(th_s * (Gs - th_c * Gsc) * iden);
      near |= (th_s > 0.0 && f.xi < kp.xi_thr) || (th_c > 0.0 && 1.0 - f.y[j] < kp.y_thr);
      a_R += f.S[j] * cR;
      ab[j] = -(th_s * cs + th_c * cc - th_s * th_c * csc) * iden;
    }
  } else {
    constexpr int BPID = PID == P_GG_TTG ? P_GG_TT : P_UU_TT;
    IsrKin f;
    isr_map(k, kp.cp.mt, f, kp.cut);
    ysec[0] = f.y[0];
    ysec[1] = f.y[1];
    xi_pt = f.xi;
    isr_born_values<PID, T, LPE>(f, kp, lane, mask, bv);
    // Algorithm 2's cuts (isr_map): soft and soft-collinear terms at the soft
    // counter-event, the collinear term of sector j at sector j's collinear counter-event
    const double x2R = -(4.0 * g2 / s) * bv[0];
    const double Bs = bv[1], Bc = bv[2];
    const double Bp[2] = {BPID == P_GG_TT ? bv[3 % RealLayout<PID>::NBV] : 0.0,
                          BPID == P_GG_TT ? bv[4 % RealLayout<PID>::NBV] : 0.0};
    const double xi = f.xi, z = 1.0 - xi, iz = f.iz, is2 = 2.0 / s;
    const double th_s = xi < kp.xi_cut && f.cut_s ? 1.0 : 0.0;
    // 1 / (xi^2 (1 - y_j) K) of both sectors from one reciprocal
    const double den0 = xi * xi * (1.0 - f.y[0]) * f.K, den1 = xi * xi * (1.0 - f.y[1]) * f.K;
    const double rden = 1.0 / (den0 * den1);
    const double iden[2] = {den1 * rden, den0 * rden};
    // d xi P / d B_c, d xi P / d B_p, d xi P_0 / d B_s of the splitting kernels
    const double kc = BPID == P_GG_TT ? 2.0 * CA_ * (z + xi * xi * z) : CF_ * (1.0 + z * z);
    const double kp_ = BPID == P_GG_TT ? 2.0 * CA_ * 2.0 * (xi * xi * iz) : 0.0;
    const double ks = BPID == P_GG_TT ? 2.0 * CA_ : 2.0 * CF_;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double Gs = (1.0 - f.y[j]) * f.S[j] * f.K0 * x2R;
      const double xiP = kc * Bc + kp_ * Bp[j];
      const double xiP0 = ks * Bs;
      const double Gc = f.K * is2 * iz * 2.0 * g2 * xiP;
      const double Gsc = f.K0 * is2 * 2.0 * g2 * xiP0;
      const double th_c = f.y[j] > 1.0 - kp.delta ? 1.0 : 0.0;  // soft-collinear term's
      const double th_cc = f.cut_c[j] ? th_c : 0.0;             // collinear term's
      const double ct = (th_s * Gs + th_cc * Gc - th_s * th_c * Gsc) * iden[j];
      const double rsj = R * f.S[j] * cR;
      W += rsj - ct;
      // error scale: the real, the collinear term, and the soft pair (whose Borns are shared)
      mag += fabs(rsj) + fabs(th_cc * Gc * iden[j]) + fabs(th_s * (Gs - th_c * Gsc) * iden[j]);
      near |= (th_s > 0.0 && xi < kp.xi_thr) || ((th_cc > 0.0 || th_s * th_c > 0.0) && 1.0 - f.y[j] < kp.y_thr);
      a_R += f.S[j] * cR;
      const double gcj = th_cc * f.K * is2 * iz * 2.0 * g2 * iden[j];
      ab[0] -= th_s * (1.0 - f.y[j]) * f.S[j] * f.K0 * (-(4.0 * g2 / s)) * iden[j];
      ab[1] += th_s * th_c * f.K0 * is2 * 2.0 * g2 * ks * iden[j];
      ab[2] -= gcj * kc;
      if constexpr (BPID == P_GG_TT) ab[3 + j] = -gcj * kp_;
    }
  }
  // A point on the boundary of the FKS domain -- no emitted energy (xi = 0), all of it
  // (xi = 1), or the emission exactly along a sector's reference direction (y_j = 1) --
  // has measure zero and no defined subtracted weight (1 / (xi^2 (1 - y)) diverges):
  // weight 0, and it is not re-evaluated.  The comparisons are false for NaN.
  if (!(xi_pt > 0.0 && xi_pt < 1.0 && 1.0 - ysec[0] > 0.0 && 1.0 - ysec[1] > 0.0)) {
    W = 0.0;
    mag = 0.0;
    near = false;
  }
  if (items) {
    // every block value to lane 0 (block b lives on lane b % LPE, slot b / LPE)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double x = 0.0;
#pragma unroll
      for (int i = 0; i < NBL; ++i)
        if (i == b / LPE) x = blk[i];
      if constexpr (LPE > 1) x = __shfl_sync(mask, x, b % LPE, LPE);
      items->v[b] = x;
      items->a[b] = a_R;
    }
#pragma unroll
    for (int t = 0; t < RealLayout<PID>::NBV; ++t) {
      items->v[NB + t] = bv[t];
      items->a[NB + t] = ab[t];
    }
    items->born_scale = mag - fabs(R) * a_R;
  }
  const double magR = mag > 0.0 ? fabs(R) * a_R : 0.0;
  return RealSubOut{W, mag, magR, {ysec[0], ysec[1]}, near};
}

// Stability test of a bulk-precision result: the error of W is ~ me_eps x (error
// scale); the float32 error of the real's amplitudes per unit scale grows towards the
// collinear limit, as 1 + sqrt(rho_0 / rho) with rho = min_j (1 - y_j), rho_0 = 0.01.
// The counterterms' Born values are evaluated at regular 2 -> 2 kinematics, whose error
// does not grow there: error ~ me_eps x (growth x real part + Born part).
__device__ __forceinline__ double error_growth(const RealSubOut& r) {
  const float rho = fmaxf((float)fmin(1.0 - r.y[0], 1.0 - r.y[1]), 1e-30f);
  return 1.0 + (double)sqrtf(0.01f / rho);
}
__device__ __forceinline__ bool unstable_point(const RealSubOut& r, const KParams& kp) {
  const double g = error_growth(r);
  return r.near || !((r.magR * g + (r.mag - r.magR)) * kp.me_eps <= kp.tol * fabs(r.W));
}

// Items of a flagged point to re-evaluate in float64: bit b < NB for the real's block
// b, bit NB for the Born values together.  Largest error scale first, until the scale
// of the items left in float32, times the bulk-precision error per unit scale, is
// within kp.item_budget x tol |W|.  Points inside the thresholds take every item.
template <int PID>
__device__ __forceinline__ unsigned rescue_mask(const RealSubOut& r, const RealItems& it, const KParams& kp) {
  constexpr int NB = RealLayout<PID>::NB;
  constexpr unsigned all = (1u << (NB + 1)) - 1u;
  if (r.near) return all;
  double e[NB + 1];
  double rest = 0.0;
#pragma unroll
  for (int b = 0; b < NB; ++b) rest += (e[b] = fabs(it.a[b] * it.v[b]));
  const double grow = error_growth(r);
  rest += (e[NB] = fabs(it.born_scale) / grow);  // no growth for the Born part (see above)
  const double budget = kp.item_budget * kp.tol * fabs(r.W) / (grow * kp.me_eps);
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k <= NB; ++k) {
    if (!(rest > budget)) break;  // NaN or over budget: keep going
    int pick = -1;
    double best = -1.0;
#pragma unroll
    for (int b = 0; b <= NB; ++b)
      if (!(m >> b & 1u) && e[b] > best) {
        best = e[b];
        pick = b;
      }
    if (pick < 0) break;
    m |= 1u << pick;
    rest -= best;
  }
  return m ? m : all;
}

// Buffers of the item rescue (structure of arrays, capacity `cap` points):
// ev[slot], mask[slot], a[i * cap + slot], v[i * cap + slot]; the item lists hold
// slot * 4 + b (real blocks) and slot (Born values); count[0] = flagged points,
// count[2] = real-block items, count[3] = Born items (count[1] is the queued kernel's
// tile counter).
struct ItemBufs {
  int* ev;
  int* mask;
  double* a;
  double* v;
  int* list_r;
  int* list_b;
  long cap;
};

// out[i] = wgt[i] * W(p_i).  In the bulk precision with kp.flag_unstable set, the
// points failing the stability test are appended to resc_list; the float64 launch over
// that list (idx, count) re-evaluates them.  With kp.item_rescue set as well, each
// flagged point gets a record (coefficients, bulk-precision values, item mask) and its
// float64 items are appended to the item lists instead (warp-aggregated appends).
template <int PID, typename T, int LPE>
__global__ void __launch_bounds__(128, ME_MINB) k_real_sub(const double* __restrict__ p, const double* __restrict__ wgt,
                                                  long n, double* __restrict__ out, KParams kp,
                                                  const int* __restrict__ idx, const int* __restrict__ count,
                                                  int* __restrict__ resc_list, int* __restrict__ resc_count,
                                                  ItemBufs ib) {
  constexpr int NB = RealLayout<PID>::NB, NI = RealLayout<PID>::NI;
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) / LPE;
  const int lane = threadIdx.x % LPE;
  const long nev = count ? (long)*count : n;
  if (gid >= nev) return;
  const long ev = idx ? (long)idx[gid] : gid;
  RealItems it;
  const bool want = kp.flag_unstable && kp.item_rescue;
  const RealSubOut r = real_sub_event<PID, T, LPE>(p, n, ev, kp, lane, group_mask<LPE>(), want ? &it : nullptr);
  if (lane == 0) {
    out[ev] = (wgt ? wgt[ev] : 1.0) * r.W;
    if (kp.flag_unstable && unstable_point(r, kp)) {
      if (!kp.item_rescue) {
        const int slot = atomicAdd(resc_count, 1);
        resc_list[slot] = (int)ev;
      } else {
        const unsigned m = rescue_mask<PID>(r, it, kp);
        // warp-aggregated appends over the flagged group leaders of this warp
        const unsigned am = __activemask();
        const int wl = threadIdx.x & 31, leader = __ffs(am) - 1;
        const unsigned lt = (1u << wl) - 1u;
        int base = 0;
        if (wl == leader) base = atomicAdd(resc_count, __popc(am));
        const int slot = __shfl_sync(am, base, leader) + __popc(am & lt);
        ib.ev[slot] = (int)ev;
        ib.mask[slot] = (int)m;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          ib.a[i * ib.cap + slot] = it.a[i];
          ib.v[i * ib.cap + slot] = it.v[i];
        }
        // real-block items, ordered by block then lane within the warp
        unsigned bal[NB];
        int tot = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) tot += __popc(bal[b] = __ballot_sync(am, m >> b & 1u));
        int rbase = 0;
        if (wl == leader) rbase = atomicAdd(resc_count + 2, tot);
        rbase = __shfl_sync(am, rbase, leader);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (m >> b & 1u) ib.list_r[rbase + __popc(bal[b] & lt)] = slot * 4 + b;
          rbase += __popc(bal[b]);
        }
        const unsigned bb = __ballot_sync(am, m >> NB & 1u);
        int bbase = 0;
        if (wl == leader) bbase = atomicAdd(resc_count + 3, __popc(bb));
        bbase = __shfl_sync(am, bbase, leader);
        if (m >> NB & 1u) ib.list_b[bbase + __popc(bb & lt)] = slot;
      }
    }
  }
}

// Float64 evaluation of the rescue items (grid-stride over the item lists, counts read
// on the device): blockIdx.y = 0 takes real blocks, 1 takes the Born values.  Every
// item writes its value into its point's record.
template <int PID>
__global__ void __launch_bounds__(128, ME_MINB) k_rescue_items(const double* __restrict__ p, long n, KParams kp,
                                                               const int* __restrict__ counts, ItemBufs ib) {
  constexpr int NEXT = Proc<PID>::NEXT, NB = RealLayout<PID>::NB;
  const long stride = (long)gridDim.x * blockDim.x;
  if (blockIdx.y == 0) {
    const long nit = counts[2];
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nit; t += stride) {
      const int item = ib.list_r[t], slot = item >> 2, b = item & 3;
      r4<double> k[NEXT];
      load_event<NEXT>(p, n, ib.ev[slot], k);
      const Kin<PID, double> K = prepare<PID, double>(k, kp.cp);
      ib.v[b * ib.cap + slot] = real_block_value<PID, double>(K, b, kp);
    }
  } else {
    const long nit = counts[3];
    const unsigned self = 1u << (threadIdx.x & 31u);
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nit; t += stride) {
      const int slot = ib.list_b[t];
      r4<double> k[NEXT];
      load_event<NEXT>(p, n, ib.ev[slot], k);
      double bv[RealLayout<PID>::NBV];
      if constexpr (PID == P_EE_UUG) {
        FsrKin f;
        fsr_map(k, f);
        fsr_born_values<double, 1>(f, kp, 0, self, bv);
      } else {
        IsrKin f;
        isr_map(k, kp.cp.mt, f, Cuts{});  // the cuts are in the coefficients already
        isr_born_values<PID, double, 1>(f, kp, 0, self, bv);
      }
#pragma unroll
      for (int i = 0; i < RealLayout<PID>::NBV; ++i) ib.v[(NB + i) * ib.cap + slot] = bv[i];
    }
  }
}

// W of every flagged point from its coefficients and values (float64 where re-evaluated).
template <int PID>
__global__ void k_rescue_combine(const double* __restrict__ wgt, double* __restrict__ out,
                                 const int* __restrict__ counts, ItemBufs ib) {
  constexpr int NI = RealLayout<PID>::NI;
  const long m = counts[0];
  for (long slot = (long)blockIdx.x * blockDim.x + threadIdx.x; slot < m; slot += (long)gridDim.x * blockDim.x) {
    double W = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) W += ib.a[i * ib.cap + slot] * ib.v[i * ib.cap + slot];
    const int ev = ib.ev[slot];
    out[ev] = (wgt ? wgt[ev] : 1.0) * W;
  }
}

// Mixed-precision subtracted real in one launch, with the float64 re-evaluation queued
// per block (the per-term queues of the event-parallel design, here for the unstable
// points).  A persistent grid takes tiles of QT points from a device counter.  Each
// point is evaluated in float32, one lane per point; a point that fails the stability
// test goes to a queue in shared memory.  Whenever the queue holds QT points the block
// re-evaluates them in float64, one lane per point with every lane busy, while the
// SM's other blocks run float32 tiles next to it.  The remainder is drained at the
// end.  A point's result depends only on the point, so the output does not depend on
// which block took which tile.  `count` (optional, device): number of points.
// `tiles` must be zero at launch; `resc_count` receives the number re-evaluated.
constexpr int QT = 128;

template <int PID>
__global__ void __launch_bounds__(QT, ME_MINB) k_real_sub_queued(const double* __restrict__ p,
                                                        const double* __restrict__ wgt, long n,
                                                        double* __restrict__ out, KParams kp,
                                                        const int* __restrict__ count, int* __restrict__ tiles,
                                                        int* __restrict__ resc_count) {
  __shared__ int q[2 * QT];
  __shared__ int qn, tile;
  const long nev = count ? (long)*count : n;
  const long ntile = (nev + QT - 1) / QT;
  const unsigned self = 1u << (threadIdx.x & 31u);
  if (threadIdx.x == 0) qn = 0;
  int done = 0;
  for (;;) {
    if (threadIdx.x == 0) tile = atomicAdd(tiles, 1);
    __syncthreads();
    const long t = tile;
    const bool last = t >= ntile;  // uniform over the block
    if (!last) {
      const long ev = t * QT + threadIdx.x;
      if (ev < nev) {
        const RealSubOut r = real_sub_event<PID, float, 1>(p, n, ev, kp, 0, self);
        out[ev] = (wgt ? wgt[ev] : 1.0) * r.W;
        if (unstable_point(r, kp)) q[atomicAdd(&qn, 1)] = (int)ev;
      }
    }
    __syncthreads();
    // a full queue, or the rest once the tiles are gone (then fewer than QT are left)
    const int qc = qn;  // uniform: qn is not written between this read and the barriers below
    if (qc >= QT || (last && qc > 0)) {
      const int take = qc < QT ? qc : QT;
      if ((int)threadIdx.x < take) {
        const int e = q[threadIdx.x];
        const RealSubOut r = real_sub_event<PID, double, 1>(p, n, e, kp, 0, self);
        out[e] = (wgt ? wgt[e] : 1.0) * r.W;
      }
      const int rest = qc - take;  // < QT: at most QT - 1 were left before this tile
      __syncthreads();
      if ((int)threadIdx.x < rest) q[threadIdx.x] = q[QT + threadIdx.x];
      done += take;
      __syncthreads();
      if (threadIdx.x == 0) qn = rest;  // ordered before any append by the next barrier
    }
    if (last) break;
  }
  if (threadIdx.x == 0 && done > 0) atomicAdd(resc_count, done);
}

// ---------------------------------------------------------------- per-term queues
// The variant of Algorithm 2 discussed after it (Sec. 4.3): rather than evaluating every
// term of every point and masking the ones whose cuts fail, a float64 pass (k_terms) maps
// each point, decides its cuts and counterterm regions, stores the coefficients of W =
// sum_i a_i v_i, and queues only the amplitudes the point needs -- the real's helicity
// blocks if the real passes its cuts, the soft Born set if the soft term is active and its
// counter-event passes, the collinear Born set likewise, each with its counter-event
// momenta.  k_term_items then evaluates every queued amplitude, one lane each, in one
// launch over all queues; k_terms_combine recombines W (and, in mixed precision, applies
// the stability test and queues the float64 items of the flagged points, which the same
// item kernel evaluates in float64; k_terms_final recombines those).
//
// Value layout per record: v[b], b < NB, the real's blocks; then the Born values: initial
// state v[NB] = E, v[NB+1] = B_s (set 0, soft counter-event), v[NB+2] = B_c, v[NB+3],
// v[NB+4] = B_p (set 1, collinear counter-event); final state v[NB+j] = B_j (set j).
struct TermBufs {
  int* ev;      // [cap] point of the record
  int* flags;   // [cap] bit 0: inside xi_thr / y_thr of an active counterterm
  float* grow;  // [cap] error growth factor of the stability test
  double* a;    // [MAX_ITEMS][cap] coefficients
  double* v;    // [MAX_ITEMS][cap] values
  double* m;    // [6][cap] error-scale coefficients of the Born values (term_born_scale)
  int* cfg;     // [2][cap] the record's Born configurations, -1 for none
  double* bp;   // [16][2 cap] configuration momenta, index (component * 4 + leg)
  double* bx;   // [4][2 cap] set 0 (initial state): eikonal correlator matrix; set 1: cos, sin phi
  int* bslot;   // [2 cap] record slot | set << 30
  int* q_real;  // [cap] records whose real is evaluated (every block in one lane; Born
                //   configurations are queued as they are stored: set 0 at 0 .. cnt[TC_QB] - 1,
                //   set 1 at cap .. cap + cnt[TC_QB1] - 1, so that a warp runs one kind)
  int* r_real;  // [4 cap] float64 rescue: real blocks, slot * 4 + b
  int* r_born;  // [2 cap] float64 rescue: Born configurations, set 0 from 0, set 1 from cap
  int* flagged; // [cap] records that failed the stability test
  int* cnt;     // [8]: records, q_real, set-0 configurations, flagged, r_real, r_born set 0,
                //   set-1 configurations, r_born set 1
  long cap;
};
enum : int { TC_REC = 0, TC_QR = 1, TC_QB = 2, TC_FLAG = 3, TC_RR = 4, TC_RB = 5, TC_QB1 = 6, TC_RB1 = 7 };

// Reserve `c` consecutive entries of counter `ctr` for each lane of a full warp (every
// lane calls it; c = 0 reserves nothing): one atomic per warp.  Returns the lane's base.
__device__ __forceinline__ int warp_reserve(int* ctr, int c) {
  const int lane = threadIdx.x & 31;
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(ctr, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - c;
}

// Error scale of the Born values of a record (as RealSubOut::mag without the real):
// initial state sum_j |m_2j E + m_2j+1 B_s| + |m_4+j B_c + cp_j B_p,j| with cp_j =
// -a[NB+3+j] (g g); final state sum_j m_j |B_j|.
template <int PID>
__device__ __forceinline__ double term_born_scale(const TermBufs& tb, long slot) {
  constexpr int NB = RealLayout<PID>::NB;
  const long c = tb.cap;
  const double* v = tb.v + NB * c + slot;
  const double* m = tb.m + slot;
  if constexpr (PID == P_EE_UUG) {
    return m[0] * fabs(v[0]) + m[c] * fabs(v[c]);
  } else {
    const double E = v[0], Bs = v[c], Bc = v[2 * c];
    double sc = fabs(m[0] * E + m[c] * Bs) + fabs(m[2 * c] * E + m[3 * c] * Bs);
    if constexpr (PID == P_GG_TTG) {
      const double* a = tb.a + NB * c + slot;
      sc += fabs(m[4 * c] * Bc - a[3 * c] * v[3 * c]) + fabs(m[5 * c] * Bc - a[4 * c] * v[4 * c]);
    } else {
      sc += fabs(m[4 * c] * Bc) + fabs(m[5 * c] * Bc);
    }
    return sc;
  }
}

// Float64 pass of the per-term queues: one thread per point (the counter-event maps,
// the cuts of every term, the coefficients, and the queues).  Points with nothing left
// to evaluate get weight 0 here.  `pc` (optional, device memory, same layout as p): the
// momenta are copied there, so that the item kernels read device memory when p is host
// memory read in place over the CPU-GPU link (p is then read once).
template <int PID>
__global__ void __launch_bounds__(128) k_terms(const double* __restrict__ p, long n, double* __restrict__ out,
                                               KParams kp, const int* __restrict__ count, TermBufs tb,
                                               double* __restrict__ pc) {
  constexpr int NEXT = Proc<PID>::NEXT, NB = RealLayout<PID>::NB, NBV = RealLayout<PID>::NBV;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nev = count ? (long)*count : n;
  const bool act = i < nev;
  r4<double> k[NEXT];
  if (act) {
    load_event<NEXT>(p, n, i, k);
    if (pc) {
#pragma unroll
      for (int l = 0; l < NEXT; ++l) {
        pc[(0L * NEXT + l) * n + i] = k[l].e;
        pc[(1L * NEXT + l) * n + i] = k[l].x;
        pc[(2L * NEXT + l) * n + i] = k[l].y;
        pc[(3L * NEXT + l) * n + i] = k[l].z;
      }
    }
  } else {
#pragma unroll
    for (int l = 0; l < NEXT; ++l) k[l] = r4<double>{1.0, 0.0, 0.0, 0.0};
  }
  const double rs = k[0].e + k[1].e, s = rs * rs;
  const double g2 = kp.cp.gs * kp.cp.gs;
  const double cR = (!kp.cut.mask || pass_cuts<PID>(k, kp.cut)) ? 1.0 : 0.0;
  double a_R = 0.0, ab[NBV] = {}, m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool need[2] = {false, false}, near = false;
  double xi, y0, y1;
  r4<double> kb[2][4];
  double bx[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  double E[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (PID == P_EE_UUG) {
    FsrKin f;
    fsr_map(k, f);
    xi = f.xi;
    y0 = f.y[0];
    y1 = f.y[1];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double cB = (!kp.cut.mask || pass_cuts<P_EE_UU>(f.born[j], kp.cut)) ? 1.0 : 0.0;
      const double th_s = f.xi < kp.xi_cut ? cB : 0.0;
      const double th_c = f.y[j] > 1.0 - kp.delta ? cB : 0.0;
      const double cs = (1.0 - f.y[j]) * 0.5 * (1.0 + f.y[j]) * f.K0 * (-(4.0 * g2 / s) * 2.0 * eik(f.born[j][2], f.born[j][3], f.qdir) * (-CF_));
      const double cc = f.K1 * (2.0 / (s * (1.0 - f.xi))) * 2.0 * g2 * CF_ * (1.0 + (1.0 - f.xi) * (1.0 - f.xi));
      const double csc = f.K0 * (2.0 / s) * 2.0 * g2 * 2.0 * CF_;
      const double iden = 1.0 / (f.xi * f.xi * (1.0 - f.y[j]) * f.K[j]);
      ab[j] = -(th_s * cs + th_c * cc - th_s * th_c * csc) * iden;
      m[j] = fabs(th_c * cc * iden) + fabs(th_s * (cs - th_c * csc) * iden);
      near |= (th_s > 0.0 && f.xi < kp.xi_thr) || (th_c > 0.0 && 1.0 - f.y[j] < kp.y_thr);
      a_R += f.S[j] * cR;
      need[j] = th_s > 0.0 || th_c > 0.0;
#pragma unroll
      for (int l = 0; l < 4; ++l) kb[j][l] = f.born[j][l];
    }
  } else {
    constexpr int BPID = PID == P_GG_TTG ? P_GG_TT : P_UU_TT;
    IsrKin f;
    isr_map(k, kp.cp.mt, f, kp.cut);
    xi = f.xi;
    y0 = f.y[0];
    y1 = f.y[1];
    const double z = 1.0 - xi, iz = f.iz, is2 = 2.0 / s;
    const double th_s = xi < kp.xi_cut && f.cut_s ? 1.0 : 0.0;
    const double den0 = xi * xi * (1.0 - f.y[0]) * f.K, den1 = xi * xi * (1.0 - f.y[1]) * f.K;
    const double rden = 1.0 / (den0 * den1);
    const double iden[2] = {den1 * rden, den0 * rden};
    const double kc = BPID == P_GG_TT ? 2.0 * CA_ * (z + xi * xi * z) : CF_ * (1.0 + z * z);
    const double kp_ = BPID == P_GG_TT ? 2.0 * CA_ * 2.0 * (xi * xi * iz) : 0.0;
    const double ks = BPID == P_GG_TT ? 2.0 * CA_ : 2.0 * CF_;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double th_c = f.y[j] > 1.0 - kp.delta ? 1.0 : 0.0;
      const double th_cc = f.cut_c[j] ? th_c : 0.0;
      a_R += f.S[j] * cR;
      const double sE = th_s * (1.0 - f.y[j]) * f.S[j] * f.K0 * (-(4.0 * g2 / s)) * iden[j];
      const double sB = -th_s * th_c * f.K0 * is2 * 2.0 * g2 * ks * iden[j];
      const double gcj = th_cc * f.K * is2 * iz * 2.0 * g2 * iden[j];
      ab[0] -= sE;
      ab[1] -= sB;
      ab[2] -= gcj * kc;
      if constexpr (BPID == P_GG_TT) ab[3 + j] = -gcj * kp_;
      m[2 * j] = sE;
      m[2 * j + 1] = sB;
      m[4 + j] = gcj * kc;
      near |= (th_s > 0.0 && xi < kp.xi_thr) || ((th_cc > 0.0 || th_s * th_c > 0.0) && 1.0 - f.y[j] < kp.y_thr);
      need[1] |= th_cc > 0.0;
    }
    need[0] = th_s > 0.0;
    if (need[0]) isr_eikonal_matrix<BPID>(f, kp, E);
    // spin-correlated Borns the collinear configuration needs (g g): sector j's has a
    // nonzero coefficient only where sector j's collinear term is active, which with
    // delta <= 1 is one sector at most.  If only sector 2's is needed, the beams are
    // stored swapped: by Bose symmetry the Born with gluon 1 polarised at (k0, k1, ..)
    // is the Born with gluon 0 polarised at (k1, k0, ..), and the plain Born is
    // symmetric, so every lane then evaluates gluon 0 polarised (one code path).
    const bool p0 = BPID == P_GG_TT && ab[3 % NBV] != 0.0, p1 = BPID == P_GG_TT && ab[4 % NBV] != 0.0;
    const bool swap = p1 && !p0;
#pragma unroll
    for (int l = 0; l < 4; ++l) kb[0][l] = f.soft[l];
    kb[1][0] = swap ? f.coll[1] : f.coll[0];
    kb[1][1] = swap ? f.coll[0] : f.coll[1];
    kb[1][2] = f.coll[2];
    kb[1][3] = f.coll[3];
    bx[1][0] = f.cphi;
    bx[1][1] = f.sphi;
    bx[1][2] = (double)((p0 ? 1 : 0) | (p1 ? 2 : 0) | (swap ? 4 : 0));
  }
  // the boundary of the FKS domain has measure zero and weight 0 (see real_sub_event)
  const bool inside = act && xi > 0.0 && xi < 1.0 && 1.0 - y0 > 0.0 && 1.0 - y1 > 0.0;
  const bool need_real = inside && cR > 0.0;
  need[0] = need[0] && inside;
  need[1] = need[1] && inside;
  const bool rec = need_real || need[0] || need[1];
  if (act && !rec) out[i] = 0.0;
  const int slot = warp_reserve(tb.cnt + TC_REC, rec ? 1 : 0);
  const int qr = warp_reserve(tb.cnt + TC_QR, need_real ? 1 : 0);
  const int qb0 = warp_reserve(tb.cnt + TC_QB, need[0] ? 1 : 0);
  const int qb1 = warp_reserve(tb.cnt + TC_QB1, need[1] ? 1 : 0);
  if (!rec) return;
  const long c = tb.cap, c2 = 2 * tb.cap;
  tb.ev[slot] = (int)i;
  tb.flags[slot] = near ? 1 : 0;
  const float rho = fmaxf((float)fmin(1.0 - y0, 1.0 - y1), 1e-30f);
  tb.grow[slot] = 1.0f + sqrtf(0.01f / rho);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    tb.a[b * c + slot] = need_real ? a_R : 0.0;
    tb.v[b * c + slot] = 0.0;
  }
#pragma unroll
  for (int t = 0; t < NBV; ++t) {
    tb.a[(NB + t) * c + slot] = ab[t];
    tb.v[(NB + t) * c + slot] = 0.0;
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) tb.m[r * c + slot] = m[r];
  if (need_real) tb.q_real[qr] = slot;
#pragma unroll
  for (int set = 0; set < 2; ++set) {
    const int ci = set == 0 ? qb0 : (int)c + qb1;
    tb.cfg[set * c + slot] = need[set] ? ci : -1;
    if (!need[set]) continue;
    tb.bslot[ci] = slot | (set << 30);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      tb.bp[(0 * 4 + l) * c2 + ci] = kb[set][l].e;
      tb.bp[(1 * 4 + l) * c2 + ci] = kb[set][l].x;
      tb.bp[(2 * 4 + l) * c2 + ci] = kb[set][l].y;
      tb.bp[(3 * 4 + l) * c2 + ci] = kb[set][l].z;
    }
    if constexpr (PID != P_EE_UUG) {
      if (set == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tb.bx[q * c2 + ci] = E[q];
      } else {
        tb.bx[0 * c2 + ci] = bx[1][0];
        tb.bx[1 * c2 + ci] = bx[1][1];
        tb.bx[2 * c2 + ci] = bx[1][2];
      }
    }
  }
}

// Every queued amplitude, one lane each, in precision T: reals (from the point's momenta;
// all helicity blocks of a point in one lane, or one block per lane in the rescue queue)
// and Born configurations (from the stored counter-event momenta), in one index space
// (reals first).  RESCUE selects the float64 rescue queues.  PART: 0 every queue, 1 the
// reals only, 2 the Born configurations only (the bulk launches the two kinds apart, so
// that each kernel's code is smaller and its instruction fetch misses less).
template <int PID, typename T, bool RESCUE, int PART = 0>
__global__ void __launch_bounds__(128, ME_MINB) k_term_items(const double* __restrict__ p, long n, KParams kp,
                                                             TermBufs tb) {
  constexpr bool rescue = RESCUE;
  constexpr int NEXT = Proc<PID>::NEXT, NB = RealLayout<PID>::NB;
  const int* qr = rescue ? tb.r_real : tb.q_real;
  const long nr = PART == 2 ? 0 : tb.cnt[rescue ? TC_RR : TC_QR];
  const long n0 = PART == 1 ? 0 : tb.cnt[rescue ? TC_RB : TC_QB];
  const long nt = nr + n0 + (PART == 1 ? 0 : tb.cnt[rescue ? TC_RB1 : TC_QB1]);
  const long c = tb.cap, c2 = 2 * tb.cap;
  const unsigned self = 1u << (threadIdx.x & 31u);
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (long)gridDim.x * blockDim.x) {
    if (PART != 2 && t < nr) {
      const int item = qr[t];
      const int slot = rescue ? item >> 2 : item;
      r4<double> k[NEXT];
      load_event<NEXT>(p, n, tb.ev[slot], k);
      const Kin<PID, T> K = prepare<PID, T>(k, kp.cp);
      if constexpr (RESCUE) {
        const int b = item & 3;
        tb.v[b * c + slot] = real_block_value<PID, T>(K, b, kp);
      } else {
#pragma unroll 1
        for (int b = 0; b < NB; ++b) tb.v[b * c + slot] = real_block_value<PID, T>(K, b, kp);
      }
    } else if constexpr (PART != 1) {
      // set-0 configurations, then set-1 ones (stored from index cap)
      const long u = t - nr < n0 ? t - nr : c + (t - nr - n0);
      const int ci = rescue ? tb.r_born[u] : (int)u;
      const int bs = tb.bslot[ci], slot = bs & 0x3fffffff, set = bs >> 30;
      r4<double> kb[4];
#pragma unroll
      for (int l = 0; l < 4; ++l)
        kb[l] = r4<double>{tb.bp[(0 * 4 + l) * c2 + ci], tb.bp[(1 * 4 + l) * c2 + ci], tb.bp[(2 * 4 + l) * c2 + ci],
                           tb.bp[(3 * 4 + l) * c2 + ci]};
      if constexpr (PID == P_EE_UUG) {
        tb.v[(NB + set) * c + slot] = fsr_born_one<T, 1>(kb, kp, 0, self);
      } else {
        constexpr int BPID = PID == P_GG_TTG ? P_GG_TT : P_UU_TT;
        if (set == 0) {
          const double E[4] = {tb.bx[0 * c2 + ci], tb.bx[1 * c2 + ci], tb.bx[2 * c2 + ci], tb.bx[3 * c2 + ci]};
          double vE, vS;
          isr_soft_pair<BPID, T, 1>(kb, E, kp, 0, self, vE, vS);
          tb.v[NB * c + slot] = vE;
          tb.v[(NB + 1) * c + slot] = vS;
        } else {
          double vc[3];
          // only the spin-correlated Borns with a nonzero coefficient (flags from k_terms:
          // 1 sector 1's, 2 sector 2's, 4 beams swapped so that sector 2's is gluon 0's)
          const int fl = (int)tb.bx[2 * c2 + ci];
          const bool sw = fl & 4;
          isr_coll_set<BPID, T, 1>(kb, tb.bx[0 * c2 + ci], tb.bx[1 * c2 + ci], kp, 0, self, vc,
                                   (fl & 1) || sw, (fl & 2) && !sw);
          tb.v[(NB + 2) * c + slot] = vc[0];
          if constexpr (BPID == P_GG_TT) {
            if (fl & 1) tb.v[(NB + 3) * c + slot] = vc[1];
            if (fl & 2) tb.v[(NB + 4) * c + slot] = sw ? vc[1] : vc[2];
          }
        }
      }
    }
  }
}

// W of every record; in mixed precision (kp.flag_unstable) the stability test of
// real_sub_event and the item selection of rescue_mask, with the flagged records' float64
// items queued (whole warps iterate together for the aggregated appends).
template <int PID>
__global__ void __launch_bounds__(128) k_terms_combine(const double* __restrict__ wgt, double* __restrict__ out,
                                                       KParams kp, TermBufs tb) {
  constexpr int NB = RealLayout<PID>::NB, NI = RealLayout<PID>::NI;
  const long nrec = tb.cnt[TC_REC];
  const long c = tb.cap;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t0 = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < nrec; t0 += stride) {
    const long slot = t0 + lane;
    const bool act = slot < nrec;
    double W = 0.0;
    bool flag = false;
    unsigned msk = 0;
    int ev = 0;
    if (act) {
#pragma unroll
      for (int q = 0; q < NI; ++q) W += tb.a[q * c + slot] * tb.v[q * c + slot];
      ev = tb.ev[slot];
      if (kp.flag_unstable) {
        double R = 0.0;
#pragma unroll
        for (int b = 0; b < NB; ++b) R += tb.v[b * c + slot];
        const double grow = (double)tb.grow[slot];
        // the growth of the float32 error towards the collinear limit is the real's; the
        // Born part enters unscaled (unstable_point)
        const double bsc = term_born_scale<PID>(tb, slot) / grow;
        const double mag = fabs(tb.a[slot] * R) + bsc;
        const bool near = tb.flags[slot] & 1;
        flag = near || !(mag * grow * kp.me_eps <= kp.tol * fabs(W));
        if (flag) {
          constexpr unsigned all = (1u << (NB + 1)) - 1u;
          if (near) {
            msk = all;
          } else {
            double e[NB + 1];
            double rest = 0.0;
#pragma unroll
            for (int b = 0; b < NB; ++b) rest += (e[b] = fabs(tb.a[b * c + slot] * tb.v[b * c + slot]));
            rest += (e[NB] = bsc);
            const double budget = kp.item_budget * kp.tol * fabs(W) / (grow * kp.me_eps);
#pragma unroll
            for (int kk = 0; kk <= NB; ++kk) {
              if (!(rest > budget)) break;
              int pick = -1;
              double best = -1.0;
#pragma unroll
              for (int b = 0; b <= NB; ++b)
                if (!(msk >> b & 1u) && e[b] > best) {
                  best = e[b];
                  pick = b;
                }
              if (pick < 0) break;
              msk |= 1u << pick;
              rest -= best;
            }
            if (!msk) msk = all;
          }
          // real blocks with a zero coefficient (the real failed its cuts) stay as they are
          if (tb.a[slot] == 0.0) msk &= ~((1u << NB) - 1u);
        }
      }
      if (!flag) out[ev] = (wgt ? wgt[ev] : 1.0) * W;
    }
    // queue the flagged records' float64 items (every lane of the warp takes part)
    const int nbl = __popc(msk & ((1u << NB) - 1u));
    const bool born = msk >> NB & 1u;
    const int ci0 = born ? tb.cfg[slot] : -1, ci1 = born ? tb.cfg[c + slot] : -1;
    const int fb = warp_reserve(tb.cnt + TC_FLAG, flag ? 1 : 0);
    const int rb = warp_reserve(tb.cnt + TC_RR, nbl);
    const int cb0 = warp_reserve(tb.cnt + TC_RB, ci0 >= 0 ? 1 : 0);
    const int cb1 = warp_reserve(tb.cnt + TC_RB1, ci1 >= 0 ? 1 : 0);
    if (flag) {
      tb.flagged[fb] = (int)slot;
      int r = rb;
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (msk >> b & 1u) tb.r_real[r++] = (int)slot * 4 + b;
      if (ci0 >= 0) tb.r_born[cb0] = ci0;
      if (ci1 >= 0) tb.r_born[c + cb1] = ci1;
    }
  }
}

// W of the flagged records after their float64 items; thread 0 of block 0 copies the
// rescue counts to `counts` ([0] flagged points, [2] real blocks, [3] Born configurations,
// [4] / [5] those of set 0 / set 1: the layout me_last_rescue_work and
// me_last_rescue_configs read).
template <int PID>
__global__ void k_terms_final(const double* __restrict__ wgt, double* __restrict__ out, TermBufs tb,
                              int* __restrict__ counts) {
  constexpr int NI = RealLayout<PID>::NI;
  const long nf = tb.cnt[TC_FLAG];
  const long c = tb.cap;
  if (blockIdx.x == 0 && threadIdx.x == 0 && counts) {
    counts[0] = tb.cnt[TC_FLAG];
    counts[2] = tb.cnt[TC_RR];
    counts[3] = tb.cnt[TC_RB] + tb.cnt[TC_RB1];
    counts[4] = tb.cnt[TC_RB];
    counts[5] = tb.cnt[TC_RB1];
  }
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (long)gridDim.x * blockDim.x) {
    const long slot = tb.flagged[t];
    double W = 0.0;
#pragma unroll
    for (int q = 0; q < NI; ++q) W += tb.a[q * c + slot] * tb.v[q * c + slot];
    const int ev = tb.ev[slot];
    out[ev] = (wgt ? wgt[ev] : 1.0) * W;
  }
}

// Tree-level entries with per-term queues: the points that pass the cuts are listed
// (list, *listed); the others get weight 0.
template <int PID>
__global__ void __launch_bounds__(128) k_cut_list(const double* __restrict__ p, long n, const int* __restrict__ count,
                                                  double* __restrict__ out, KParams kp, int* __restrict__ list,
                                                  int* __restrict__ listed) {
  constexpr int NEXT = Proc<PID>::NEXT;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nev = count ? (long)*count : n;
  bool pass = false;
  if (i < nev) {
    r4<double> k[NEXT];
    load_event<NEXT>(p, n, i, k);
    pass = pass_cuts<PID>(k, kp.cut);
    if (!pass) out[i] = 0.0;
  }
  const int at = warp_reserve(listed, pass ? 1 : 0);
  if (pass) list[at] = (int)i;
}

// ---------------------------------------------------------------- weight accumulation
// Deterministic two-pass reduction: per-block partial (sum w, sum w^2) in a fixed tree
// order, then one block adds the partials in block order.  No floating atomics.
// `cnt` (optional, device): the number of points, read on the device (at most n).
__global__ void k_partials(const double* __restrict__ w, long n, double* __restrict__ part, const int* __restrict__ cnt);
__global__ void k_finish(const double* __restrict__ part, int nblk, double* __restrict__ acc, long n,
                         const int* __restrict__ cnt);

// ---------------------------------------------------------------- launch registry
struct LaunchArgs {
  const double* p;
  const double* wgt;
  long n;
  double* out;
  KParams kp;
  const int* idx;    // optional event list (rescue), length *count on the device
  const int* count;  // optional number of events, read on the device (events 0..*count-1 without idx)
  int* resc_list;    // real kernel in bulk precision: unstable points are appended here
  int* resc_count;   // [0] flagged points, [1] queued kernel's tiles, [2] / [3] real-block / Born items
  ItemBufs items;    // item rescue records and lists
  long groups;       // number of event groups to launch (n, or the list capacity)
  int* tiles;        // queued kernel: tile counter, zero at launch
  double* p_copy;    // per-term queues: device copy of p made by k_terms (p in host memory), or null
};
enum KernelKind : int { K_TREE = 0, K_REAL = 1 };

template <int PID, typename T, int LPE>
cudaError_t launch_one(int kind, const LaunchArgs& a, cudaStream_t st) {
  (void)cudaGetLastError();  // the launch status below must not report an earlier call's error
  const int threads = 128;
  const long total = a.groups * LPE;
  const long blocks = (total + threads - 1) / threads;
  if (blocks <= 0) return cudaSuccess;
  if (kind == K_TREE) {
    if constexpr (PID == P_GG_TTGG && std::is_same<T, float>::value) {
      if constexpr (LPE != 4) {
        return cudaErrorInvalidValue;
      } else {
        static bool attr_set[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !attr_set[dev]) {
          cudaFuncSetAttribute(k_tree_tc4<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC4_SMEM);
          attr_set[dev] = true;
        }
        const long tb = (total + TC4_THREADS - 1) / TC4_THREADS;
        k_tree_tc4<4><<<(unsigned)tb, TC4_THREADS, TC4_SMEM, st>>>(a.p, a.wgt, a.n, a.out, a.kp, a.idx, a.count);
      }
    } else {
      k_tree<PID, T, LPE><<<(unsigned)blocks, threads, 0, st>>>(a.p, a.wgt, a.n, a.out, a.kp, a.idx, a.count);
    }
  } else {
    if constexpr (PID == P_EE_UUG || PID == P_GG_TTG || PID == P_UU_TTG)
      k_real_sub<PID, T, LPE><<<(unsigned)blocks, threads, 0, st>>>(a.p, a.wgt, a.n, a.out, a.kp, a.idx, a.count,
                                                                       a.resc_list, a.resc_count, a.items);
    else
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The item rescue after a bulk-precision launch with kp.item_rescue: float64 items,
// then the recombination.  Persistent grids (resident blocks x SMs, found once per
// device) walk the lists, whose lengths are read on the device.
template <int PID>
cudaError_t launch_items_one(const LaunchArgs& a, cudaStream_t st) {
  (void)cudaGetLastError();
  static std::atomic<int> resident[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int g = resident[dev].load(std::memory_order_relaxed);
  if (g == 0) {
    int per = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rescue_items<PID>, 128, 0);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
    resident[dev].store(g, std::memory_order_relaxed);
  }
  const long cap_blocks = (a.items.cap * 4 + 127) / 128;
  const unsigned gx = (unsigned)std::max(1L, std::min<long>(g, cap_blocks));
  k_rescue_items<PID><<<dim3(gx, 2), 128, 0, st>>>(a.p, a.n, a.kp, a.resc_count, a.items);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned gc = (unsigned)std::max(1L, std::min<long>(4 * g, (a.items.cap + 255) / 256));
  k_rescue_combine<PID><<<gc, 256, 0, st>>>(a.wgt, a.out, a.resc_count, a.items);
  return cudaGetLastError();
}

// per-process launchers (one translation unit each); lpe in {1, 2, 4, 8, 16}
cudaError_t launch_ee(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_gg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_ggg(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_ggg64(int kind, int lpe, const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_uu(int pid, int kind, bool fp64, int lpe, const LaunchArgs& a, cudaStream_t st);
// float64 items and recombination of the item rescue (one per process family)
cudaError_t launch_items_ee(const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_items_gg(const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_items_uu(const LaunchArgs& a, cudaStream_t st);
// mixed-precision subtracted real with the queued float64 re-evaluation (k_real_sub_queued)
cudaError_t launch_queued(int pid, const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_queued_gg(const LaunchArgs& a, cudaStream_t st);

// One persistent launch of k_real_sub_queued: as many blocks as are resident at once
// (occupancy x SMs, found once per device), at most one per tile.
template <int PID>
cudaError_t launch_queued_one(const LaunchArgs& a, cudaStream_t st) {
  (void)cudaGetLastError();  // the launch status below must not report an earlier call's error
  static std::atomic<int> resident[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int g = resident[dev].load(std::memory_order_relaxed);
  if (g == 0) {
    int per = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_real_sub_queued<PID>, QT, 0);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
    resident[dev].store(g, std::memory_order_relaxed);
  }
  const long ntile = (a.groups + QT - 1) / QT;
  if (ntile <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)(ntile < g ? ntile : g);
  k_real_sub_queued<PID><<<blocks, QT, 0, st>>>(a.p, a.wgt, a.n, a.out, a.kp, a.count, a.tiles, a.resc_count);
  return cudaGetLastError();
}

// Per-term queues (k_terms ... k_terms_final): phase 0 enqueues the float64 pass, the
// bulk-precision items and the recombination (with the stability test in mixed
// precision); phase 1 the float64 rescue items and the flagged points' recombination
// (mixed precision only), and copies the rescue counts to `counts`.
template <int PID>
cudaError_t launch_terms_one(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts,
                             cudaStream_t st) {
  (void)cudaGetLastError();
  static std::atomic<int> resident[2][64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const bool f64 = phase == 1 || !mixed;
  int g = resident[f64][dev].load(std::memory_order_relaxed);
  if (g == 0) {
    int per = 0, sms = 0;
    e = f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_term_items<PID, double, true>, 128, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_term_items<PID, float, false, 1>, 128, 0);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
    resident[f64][dev].store(g, std::memory_order_relaxed);
  }
  const long items_cap = (RealLayout<PID>::NB + 2) * tb.cap;
  const unsigned gi = (unsigned)std::max(1L, std::min<long>(g, (items_cap + 127) / 128));
  const unsigned gc = (unsigned)std::max(1L, std::min<long>(4 * g, (tb.cap + 127) / 128));
  if (phase == 0) {
    if ((e = cudaMemsetAsync(tb.cnt, 0, 8 * sizeof(int), st)) != cudaSuccess) return e;
    const long blocks = (a.groups + 127) / 128;
    if (blocks <= 0) return cudaSuccess;
    k_terms<PID><<<(unsigned)blocks, 128, 0, st>>>(a.p, a.n, a.out, a.kp, a.count, tb, a.p_copy);
    const double* pi = a.p_copy ? a.p_copy : a.p;
    if (mixed) {
      k_term_items<PID, float, false, 1><<<gi, 128, 0, st>>>(pi, a.n, a.kp, tb);
      k_term_items<PID, float, false, 2><<<gi, 128, 0, st>>>(pi, a.n, a.kp, tb);
    } else {
      k_term_items<PID, double, false><<<gi, 128, 0, st>>>(pi, a.n, a.kp, tb);
    }
    k_terms_combine<PID><<<gc, 128, 0, st>>>(a.wgt, a.out, a.kp, tb);
  } else {
    k_term_items<PID, double, true><<<gi, 128, 0, st>>>(a.p_copy ? a.p_copy : a.p, a.n, a.kp, tb);
    k_terms_final<PID><<<gc, 128, 0, st>>>(a.wgt, a.out, tb, counts);
  }
  return cudaGetLastError();
}
cudaError_t launch_terms_ee(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts, cudaStream_t st);
cudaError_t launch_terms_gg(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts, cudaStream_t st);
cudaError_t launch_terms_uu(int phase, bool mixed, const LaunchArgs& a, const TermBufs& tb, int* counts, cudaStream_t st);
// tree entries with per-term queues: list the points that pass the cuts (k_cut_list)
cudaError_t launch_cut_list(int pid, const LaunchArgs& a, int* list, int* listed, cudaStream_t st);

}  // namespace me

#define ME_LPE_SWITCH(PID, T)                                            \
  switch (lpe) {                                                         \
    case 1: return me::launch_one<PID, T, 1>(kind, a, st);               \
    case 2: return me::launch_one<PID, T, 2>(kind, a, st);               \
    case 4: return me::launch_one<PID, T, 4>(kind, a, st);               \
    case 8: return me::launch_one<PID, T, 8>(kind, a, st);               \
    case 16: return me::launch_one<PID, T, 16>(kind, a, st);             \
    default: return cudaErrorInvalidValue;                               \
  }
// g g -> t tbar g g runs at most 8 lanes per event (it has 8 helicity blocks)
#define ME_LPE_SWITCH8(PID, T)                                           \
  switch (lpe) {                                                         \
    case 1: return me::launch_one<PID, T, 1>(kind, a, st);               \
    case 2: return me::launch_one<PID, T, 2>(kind, a, st);               \
    case 4: return me::launch_one<PID, T, 4>(kind, a, st);               \
    case 8: return me::launch_one<PID, T, 8>(kind, a, st);               \
    default: return cudaErrorInvalidValue;                               \
  }
#define ME_PREC_SWITCH(PID)                      \
  if (fp64) {                                    \
    ME_LPE_SWITCH(PID, double)                   \
  } else {                                       \
    ME_LPE_SWITCH(PID, float)                    \
  }
