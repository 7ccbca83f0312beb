// Algorithmic operation count of the amplitude code (host program).
//
// The same templated amplitude routines that the kernels run are instantiated with a
// counting scalar type: every floating-point +, -, *, / and sqrt on the amplitude's
// arithmetic type counts as one operation (a fused multiply-add therefore counts two),
// sign flips and comparisons count zero.  Momentum sums and propagator denominators,
// which the kernels keep in float64, are not counted.  The colour sums are counted
// from their loop structure.  Per event, one helicity of each flipped pair (h, -h) is
// evaluated, as in the kernels, in helicity blocks.  Output: one JSON object with
// operations per helicity (per-event Born count over the helicities evaluated) and per
// event for every process and entry point.
#include <cmath>
#include <cstdio>

#include "me_procs.cuh"

static long g_ops = 0;
struct Flop {
  double v;
  Flop() = default;
  Flop(double x) : v(x) {}
};
inline Flop operator+(Flop a, Flop b) { ++g_ops; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { ++g_ops; return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { ++g_ops; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++g_ops; return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop& operator+=(Flop& a, Flop b) { ++g_ops; a.v += b.v; return a; }
inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
inline bool operator>=(Flop a, Flop b) { return a.v >= b.v; }
inline bool operator==(Flop a, Flop b) { return a.v == b.v; }
inline Flop msqrt(Flop a) { ++g_ops; return Flop(std::sqrt(a.v)); }  // found by argument lookup

using namespace me;

// J^dagger C J per helicity as the kernels evaluate it (me_kernels.cuh: colour_sum): for up
// to 6 flows the triangular form over the doubled upper triangle, 2 NF^2 + 4 NF flops;
// beyond, the full matrix, 4 NF^2 + 4 NF
static double colour_flops(int nf) { return nf <= 6 ? 2.0 * nf * nf + 4.0 * nf : 4.0 * nf * nf + 4.0 * nf; }

// one helicity block (me_procs.cuh): amplitudes of four helicities plus their colour sums
template <int PID>
static double block_ops(const r4<double>* p, int hb = 1, const c4<Flop>* ov = nullptr, int ov_leg = -1) {
  const Couplings cp{1.2, 0.3, 173.0};
  const Kin<PID, Flop> K = prepare<PID, Flop>(p, cp);
  g_ops = 0;
  int calls = 0;
  amplitude_block<PID, Flop>(K, hb, cp, [&](int, const cx<Flop>*) { ++calls; }, ov, ov_leg);
  return (double)g_ops + calls * colour_flops(Proc<PID>::NFLOW);
}

// per-event preparation (reciprocal denominators etc. in the amplitude's type)
template <int PID>
static double prep_ops(const r4<double>* p) {
  const Couplings cp{1.2, 0.3, 173.0};
  g_ops = 0;
  const Kin<PID, Flop> K = prepare<PID, Flop>(p, cp);
  (void)K;
  return (double)g_ops;
}

// Born |M|^2 of one event: every block of the half helicity set, plus the preparation
template <int PID>
static double born_ops(const r4<double>* p) {
  double t = prep_ops<PID>(p);
  for (int b = 0; b < n_live_blocks<PID>(); ++b) t += block_ops<PID>(p, live_block_hel<PID>(b));
  return t;
}

int main() {
  // a generic massive 2 -> 4 configuration is enough: the count does not depend on values
  r4<double> p[6] = {{1000, 0, 0, 1000},     {1000, 0, 0, -1000}, {600, 100, 200, 300},
                     {700, -150, -100, 200}, {400, 30, -80, -300}, {300, 20, -20, -200}};
  c4<Flop> e;
  for (int i = 0; i < 4; ++i) e.v[i] = cx<Flop>{Flop(0.5), Flop(0.0)};
  const double quad2 = 10.0;  // J^dagger E J for the 2x2 eikonal-weighted correlator matrix
  // subtracted real: real blocks + Born tasks (soft with the eikonal form, collinear,
  // spin-correlated for g g: both polarised gluons at the one collinear kinematics)
  const double real_ee = born_ops<P_EE_UUG>(p) + 2 * born_ops<P_EE_UU>(p);
  const double real_gg = born_ops<P_GG_TTG>(p) + born_ops<P_GG_TT>(p) + 8 * quad2 + born_ops<P_GG_TT>(p) +
                         block_ops<P_GG_TT>(p, 2, &e, 0) + block_ops<P_GG_TT>(p, 1, &e, 1);
  const double real_uu = born_ops<P_UU_TTG>(p) + born_ops<P_UU_TT>(p) + 8 * quad2 + born_ops<P_UU_TT>(p);
  const double b[7] = {born_ops<P_EE_UU>(p),  born_ops<P_EE_UUG>(p), born_ops<P_GG_TT>(p), born_ops<P_GG_TTG>(p),
                       born_ops<P_GG_TTGG>(p), born_ops<P_UU_TT>(p), born_ops<P_UU_TTG>(p)};
  const int nh[7] = {16, 32, 16, 32, 64, 16, 32};
  std::printf("{\"per_helicity\": {\"ee_uu\": %.0f, \"ee_uug\": %.0f, \"gg_tt\": %.0f, \"gg_ttg\": %.0f, "
              "\"gg_ttgg\": %.0f, \"uu_tt\": %.0f, \"uu_ttg\": %.0f},\n",
              2 * b[0] / nh[0], 2 * b[1] / nh[1], 2 * b[2] / nh[2], 2 * b[3] / nh[3], 2 * b[4] / nh[4],
              2 * b[5] / nh[5], 2 * b[6] / nh[6]);
  std::printf(" \"born_per_event\": {\"ee_uu\": %.0f, \"ee_uug\": %.0f, \"gg_tt\": %.0f, \"gg_ttg\": %.0f, "
              "\"gg_ttgg\": %.0f, \"uu_tt\": %.0f, \"uu_ttg\": %.0f},\n",
              b[0], b[1], b[2], b[3], b[4], b[5], b[6]);
  std::printf(" \"real_subtracted_per_event\": {\"ee_uug\": %.0f, \"gg_ttg\": %.0f, \"uu_ttg\": %.0f},\n", real_ee,
              real_gg, real_uu);
  // per-term queues: one Born configuration per lane -- soft (Born with the eikonal
  // form), collinear (Born plus, for g g, the spin-correlated block of the one sector
  // whose collinear term is active, delta <= 1), or a final-state sector's Born
  const double soft_gg = born_ops<P_GG_TT>(p) + 8 * quad2,
               coll_gg = born_ops<P_GG_TT>(p) + block_ops<P_GG_TT>(p, 2, &e, 0);
  const double soft_uu = born_ops<P_UU_TT>(p) + 8 * quad2, coll_uu = born_ops<P_UU_TT>(p);
  std::printf(" \"term_config_per_event\": {\"ee_uug\": [%.0f, %.0f], \"gg_ttg\": [%.0f, %.0f], "
              "\"uu_ttg\": [%.0f, %.0f]},\n", b[0], b[0], soft_gg, coll_gg, soft_uu, coll_uu);
  std::printf(" \"colour_sum_per_event\": {\"gg_ttgg\": %.0f}}\n", 32 * (4.0 * 24 * 24 + 4.0 * 24));
  return 0;
}
