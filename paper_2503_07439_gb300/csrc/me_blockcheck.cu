// Host check of the helicity-block amplitude routines (test program, built by the CPU
// test suite; no GPU needed).  For every point read from stdin it evaluates the
// colour-summed |M|^2 twice with the same templates the kernels use: over every
// helicity one at a time, and over the blocks of one member of each flipped pair
// (doubled), in float64 and in float32.  It prints one line per point:
//   <block fp64> <single fp64> <block fp32> <single fp32>
// Input: "<pid> <n> <n_ext>" then the momenta [4][n_ext][n] (float64, SoA).
#include <cmath>
#include <cstdio>
#include <vector>

#include "me_internal.h"
#include "me_kernels.cuh"

using namespace me;

template <int PID, typename T>
static double csum(const ColourTables& tab, const cx<T>* J) {
  constexpr int NF = Proc<PID>::NFLOW;
  const double* C = tab.C[PID];
  double t = 0;
  for (int a = 0; a < NF; ++a)
    for (int b = 0; b < NF; ++b)
      t += C[a * NF + b] * ((double)J[a].re * (double)J[b].re + (double)J[a].im * (double)J[b].im);
  return t;
}

template <int PID, typename T>
static void eval(const ColourTables& tab, const r4<double>* k, const Couplings& cp, double* blk, double* single) {
  constexpr int NH = Proc<PID>::NHEL, NF = Proc<PID>::NFLOW;
  const Kin<PID, T> K = prepare<PID, T>(k, cp);
  double s = 0;
  for (int h = 0; h < NH; ++h) {
    cx<T> J[NF];
    amplitude<PID, T>(K, h, cp, J);
    s += csum<PID, T>(tab, J);
  }
  double b = 0;
  for (int i = 0; i < n_live_blocks<PID>(); ++i)
    amplitude_block<PID, T>(K, live_block_hel<PID>(i), cp, [&](int, const cx<T>* A) { b += csum<PID, T>(tab, A); });
  *blk = 2.0 * b;
  *single = s;
}

template <int PID>
static void run(const ColourTables& tab, const std::vector<double>& p, int n, int next) {
  const Couplings cp{std::sqrt(4 * M_PI * 0.118), std::sqrt(4 * M_PI / 132.507), 173.0};
  for (int i = 0; i < n; ++i) {
    r4<double> k[6];
    for (int l = 0; l < next; ++l)
      k[l] = {p[(0 * next + l) * n + i], p[(1 * next + l) * n + i], p[(2 * next + l) * n + i], p[(3 * next + l) * n + i]};
    double b64, s64, b32, s32;
    eval<PID, double>(tab, k, cp, &b64, &s64);
    eval<PID, float>(tab, k, cp, &b32, &s32);
    std::printf("%.17g %.17g %.17g %.17g\n", b64, s64, b32, s32);
  }
}

int main() {
  static ColourTables tab;
  if (me_internal_build_tables(&tab) != ME_OK) return 1;
  int pid, n, next;
  while (std::scanf("%d %d %d", &pid, &n, &next) == 3) {
    std::vector<double> p((size_t)4 * next * n);
    for (auto& x : p)
      if (std::scanf("%lf", &x) != 1) return 1;
    switch (pid) {
      case P_EE_UU: run<P_EE_UU>(tab, p, n, next); break;
      case P_EE_UUG: run<P_EE_UUG>(tab, p, n, next); break;
      case P_GG_TT: run<P_GG_TT>(tab, p, n, next); break;
      case P_GG_TTG: run<P_GG_TTG>(tab, p, n, next); break;
      case P_GG_TTGG: run<P_GG_TTGG>(tab, p, n, next); break;
      case P_UU_TT: run<P_UU_TT>(tab, p, n, next); break;
      case P_UU_TTG: run<P_UU_TTG>(tab, p, n, next); break;
      default: return 2;
    }
  }
  return 0;
}
