// Algorithmic operation count of the amplitude code (host program).
//
// The same templated amplitude routines that the kernels run are instantiated with a
// counting scalar type: every floating-point +, -, *, / and sqrt on the amplitude's
// arithmetic type counts as one operation (a fused multiply-add therefore counts two),
// sign flips and comparisons count zero.  Momentum sums and propagator denominators,
// which the kernels keep in float64, are not counted.  The colour sums are counted
// from their loop structure.  Per event, one helicity of each flipped pair (h, -h) is
// evaluated, as in the kernels.  Output: one JSON object with operations per helicity
// and per event for every process and entry point.
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

template <int PID>
static double amp_ops(const r4<double>* p, const c4<Flop>* ov = nullptr, int ov_leg = -1, int hel = 5) {
  cx<Flop> J[24];
  const Couplings cp{1.2, 0.3, 173.0};
  const Kin<PID, Flop> K = prepare<PID, Flop>(p, cp);
  g_ops = 0;
  amplitude<PID, Flop>(K, hel, cp, J, ov, ov_leg);
  return (double)g_ops;
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

static double csum_ops(int nf) { return 4.0 * nf * nf + 4.0 * nf; }

int main() {
  // a generic massive 2 -> 4 configuration is enough: the count does not depend on values
  r4<double> p[6] = {{1000, 0, 0, 1000},     {1000, 0, 0, -1000}, {600, 100, 200, 300},
                     {700, -150, -100, 200}, {400, 30, -80, -300}, {300, 20, -20, -200}};
  const double ee = amp_ops<P_EE_UU>(p), eeg = amp_ops<P_EE_UUG>(p);
  const double gg = amp_ops<P_GG_TT>(p), ggg = amp_ops<P_GG_TTG>(p), gggg = amp_ops<P_GG_TTGG>(p);
  const double uu = amp_ops<P_UU_TT>(p), uug = amp_ops<P_UU_TTG>(p);
  c4<Flop> e;
  for (int i = 0; i < 4; ++i) e.v[i] = cx<Flop>{Flop(0.5), Flop(0.0)};
  const double gg_ov = amp_ops<P_GG_TT>(p, &e, 0);
  // per-helicity cost = amplitude + colour sum
  const double h_ee = ee + csum_ops(1), h_eeg = eeg + csum_ops(1);
  const double h_gg = gg + csum_ops(2), h_ggg = ggg + csum_ops(6), h_gggg = gggg + csum_ops(24);
  const double h_uu = uu + csum_ops(2), h_uug = uug + csum_ops(4);
  // subtracted real: real helicities + Born tasks (soft with eikonal form, collinear, spin-correlated)
  const double quad2 = 10.0;
  const double pr_ee = prep_ops<P_EE_UU>(p), pr_eeg = prep_ops<P_EE_UUG>(p);
  const double pr_gg = prep_ops<P_GG_TT>(p), pr_ggg = prep_ops<P_GG_TTG>(p);
  const double pr_uu = prep_ops<P_UU_TT>(p), pr_uug = prep_ops<P_UU_TTG>(p);
  // one helicity of each flipped pair is evaluated (the sums are doubled)
  const double real_ee = 16 * h_eeg + pr_eeg + 16 * h_ee + 2 * pr_ee;
  const double real_gg = 16 * h_ggg + pr_ggg + 8 * (h_gg + quad2) + 8 * h_gg + 8 * (gg_ov + csum_ops(2)) + 3 * pr_gg;
  const double real_uu = 16 * h_uug + pr_uug + 8 * (h_uu + quad2) + 8 * h_uu + 2 * pr_uu;
  std::printf(
      "{\"per_helicity\": {\"ee_uu\": %.0f, \"ee_uug\": %.0f, \"gg_tt\": %.0f, \"gg_ttg\": %.0f, "
      "\"gg_ttgg\": %.0f, \"uu_tt\": %.0f, \"uu_ttg\": %.0f},\n"
      " \"born_per_event\": {\"ee_uu\": %.0f, \"ee_uug\": %.0f, \"gg_tt\": %.0f, \"gg_ttg\": %.0f, "
      "\"gg_ttgg\": %.0f, \"uu_tt\": %.0f, \"uu_ttg\": %.0f},\n"
      " \"real_subtracted_per_event\": {\"ee_uug\": %.0f, \"gg_ttg\": %.0f, \"uu_ttg\": %.0f},\n"
      " \"colour_sum_per_event\": {\"gg_ttgg\": %.0f}}\n",
      h_ee, h_eeg, h_gg, h_ggg, h_gggg, h_uu, h_uug, 8 * h_ee + pr_ee, 16 * h_eeg + pr_eeg, 8 * h_gg + pr_gg,
      16 * h_ggg + pr_ggg, 32 * h_gggg + prep_ops<P_GG_TTGG>(p), 8 * h_uu + pr_uu, 16 * h_uug + pr_uug, real_ee,
      real_gg, real_uu, 32 * csum_ops(24));
  return 0;
}
