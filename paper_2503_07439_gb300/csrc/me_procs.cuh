// Per-process colour-decomposed helicity amplitudes (device).
//
// Each routine returns, for one helicity configuration, the partial amplitudes
// J_c of the process in its colour-flow basis, so that the colour-summed squared
// amplitude is J^dagger C J (Sec. 2.1, Eq. (born): |sum of diagrams|^2; Sec. 4.2:
// Born, real and counterterms are all tree-level amplitudes).
//
//  * t tbar + n gluons (gg->tt, gg->ttg, gg->ttgg): colour-ordered Berends-Giele
//    recursion.  Full amplitude M = sum_sigma (T^{a_s1} ... T^{a_sn})_{i_t j_tbar} A(sigma);
//    colour-ordered rules derived from the Feynman rules with [T^a,T^b] = i f^abc T^c:
//      gluon current  J(LR)  = -(g/Q^2) V3(J_L, J_R; -Q_L, -Q_R)
//                     J(LMR) = +(g^2/Q^2) [2(J_L.J_R) J_M - (J_L.J_M) J_R - (J_M.J_R) J_L]
//      quark line     U(s_1..s_k) = sum_j U(s_1..s_j) (i g Jslash(s_{j+1}..s_k)) i(Qslash+m)/(Q^2-m^2)
//      amplitude      A(s) = sum_j U(s_1..s_j) (i g Jslash(s_{j+1}..s_n)) v(tbar).
//  * e+e- -> u ubar (g): photon current from the leptons inserted on the quark line.
//  * u ubar -> t tbar (g): explicit diagrams, colour by Fierz onto a 2- (4-) element basis.
// Momenta: all-outgoing (q = -p for incoming legs).  Everything that does not depend
// on the helicities -- momenta in T and the reciprocal propagator denominators, whose
// invariants are formed in float64 to avoid cancellation -- is prepared once per event
// (prepare<PID,T>) and shared by all helicities; spinors and currents are in T.
#pragma once
#include "me_math.cuh"

namespace me {

enum ProcId : int {
  P_EE_UU = 0,
  P_EE_UUG = 1,
  P_GG_TT = 2,
  P_GG_TTG = 3,
  P_GG_TTGG = 4,
  P_UU_TT = 5,
  P_UU_TTG = 6,
  P_COUNT = 7
};

template <int PID> struct Proc;
template <> struct Proc<P_EE_UU> { static constexpr int NEXT = 4, NHEL = 16, NFLOW = 1; };
template <> struct Proc<P_EE_UUG> { static constexpr int NEXT = 5, NHEL = 32, NFLOW = 1; };
template <> struct Proc<P_GG_TT> { static constexpr int NEXT = 4, NHEL = 16, NFLOW = 2, NG = 2; };
template <> struct Proc<P_GG_TTG> { static constexpr int NEXT = 5, NHEL = 32, NFLOW = 6, NG = 3; };
template <> struct Proc<P_GG_TTGG> { static constexpr int NEXT = 6, NHEL = 64, NFLOW = 24, NG = 4; };
template <> struct Proc<P_UU_TT> { static constexpr int NEXT = 4, NHEL = 16, NFLOW = 2; };
template <> struct Proc<P_UU_TTG> { static constexpr int NEXT = 5, NHEL = 32, NFLOW = 4; };

struct Couplings {
  double gs;   // strong coupling g_s
  double ee;   // electromagnetic coupling e
  double mt;   // top mass
};

__host__ __device__ constexpr int factorial(int n) { return n <= 1 ? 1 : n * factorial(n - 1); }

// permutation number `idx` (lexicographic) of {0..n-1}
ME_HD void nth_perm(int n, int idx, int* out) {
  int pool[4] = {0, 1, 2, 3};
  int m = n;
  for (int i = 0; i < n; ++i) {
    int f = factorial(m - 1);
    int k = idx / f;
    idx -= k * f;
    out[i] = pool[k];
    for (int j = k; j < m - 1; ++j) pool[j] = pool[j + 1];
    --m;
  }
}

ME_HD int hel_of(int hel, int leg) { return ((hel >> leg) & 1) ? 1 : -1; }

// ----------------------------------------------------------------------------
// Per-event kinematics of t tbar + NG gluons.  Gluon g (0..NG-1) is leg 0, 1, 4, 5.
// ig[S] = 1/Q_S^2 for a gluon subset S (bit mask, |S| >= 2), iq[S] = 1/((p_t+Q_S)^2-m^2).
template <typename T, int NG>
struct KinTT {
  r4<T> pl[6];          // physical external momenta (wavefunctions)
  r4<T> q[NG];          // outgoing gluon momenta
  T ig[1 << NG];
  T iq[1 << NG];
  wf_v<T> wg[NG];       // polarisation ingredients of the gluons (legs 0, 1, 4, 5)
  wf_f<T> wt, wtb;      // spinor ingredients of the top and the antitop
};

template <typename T, int NG>
ME_HD KinTT<T, NG> prep_tt(const r4<double>* p, const Couplings& cp) {
  KinTT<T, NG> K;
  const int NEXT = NG + 2;
  for (int l = 0; l < NEXT; ++l) K.pl[l] = cast4<T>(p[l]);
  r4<double> q[NG];
  for (int i = 0; i < NG; ++i) {
    const int l = i < 2 ? i : i + 2;
    q[i] = l < 2 ? -p[l] : p[l];
    K.q[i] = l < 2 ? -K.pl[l] : K.pl[l];
    K.wg[i] = wf_vector(K.pl[l]);
  }
  K.wt = wf_fermion(K.pl[2], (T)cp.mt);
  K.wtb = wf_fermion(K.pl[3], (T)cp.mt);
  // The gluons are massless and the top on shell, so every subset invariant is a sum of
  // pairwise products (float64):  Q_S^2 = 2 sum_{i<j in S} q_i.q_j,
  // (p_t + Q_S)^2 - m^2 = 2 sum_{i in S} p_t.q_i + Q_S^2.
  double qq[NG][NG], tq[NG];
  for (int i = 0; i < NG; ++i) {
    tq[i] = mdot(p[2], q[i]);
    for (int j = i + 1; j < NG; ++j) qq[i][j] = mdot(q[i], q[j]);
  }
  for (int S = 1; S < (1 << NG); ++S) {
    double s2 = 0.0, st = 0.0;
    int cnt = 0;
    for (int i = 0; i < NG; ++i)
      if (S >> i & 1) {
        st += tq[i];
        ++cnt;
        for (int j = i + 1; j < NG; ++j)
          if (S >> j & 1) s2 += qq[i][j];
      }
    K.ig[S] = cnt >= 2 ? T(1) / (T)(2.0 * s2) : T(0);
    K.iq[S] = cnt <= NG - 1 ? T(1) / (T)(2.0 * (st + s2)) : T(0);
  }
  K.ig[0] = K.iq[0] = T(0);
  return K;
}

// Generic colour-ordered recursion (used for 4 gluons): for every ordering, contiguous
// gluon currents J[i][j] and the top line U[k]; denominators from the per-event table.
template <typename T, int NG>
ME_HD void amp_ttng(const KinTT<T, NG>& K, int hel, const Couplings& cp, cx<T>* A) {
  constexpr int NF = factorial(NG);
  const T g = (T)cp.gs;
  const T mt = (T)cp.mt;
  c4<T> eps[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) {
    const int l = i < 2 ? i : i + 2;
    eps[i] = polvec(K.pl[l], hel_of(hel, l), l >= 2);
  }
  const c4<T> ub = dbar(spinor_u(K.pl[2], mt, hel_of(hel, 2)));
  const c4<T> vb = spinor_v(K.pl[3], mt, hel_of(hel, 3));
  for (int f = 0; f < NF; ++f) {
    int s[NG];
    nth_perm(NG, f, s);
    c4<T> J[NG][NG];
    r4<T> Q[NG][NG];
    int M[NG][NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      J[i][i] = eps[s[i]];
      Q[i][i] = K.q[s[i]];
      M[i][i] = 1 << s[i];
    }
#pragma unroll
    for (int len = 2; len <= NG; ++len) {
#pragma unroll
      for (int i = 0; i + len - 1 < NG; ++i) {
        const int j = i + len - 1;
        Q[i][j] = Q[i][j - 1] + K.q[s[j]];
        M[i][j] = M[i][j - 1] | (1 << s[j]);
        const T inv = K.ig[M[i][j]];
        c4<T> acc = czero<T>();
#pragma unroll
        for (int k = i; k < j; ++k) cadd(acc, vvv(J[i][k], J[k + 1][j], -Q[i][k], -Q[k + 1][j]));
        cscale(acc, -g * inv);
        if (len >= 3) {
          c4<T> acc4 = czero<T>();
#pragma unroll
          for (int k = i; k < j - 1; ++k)
#pragma unroll
            for (int l = k + 1; l < j; ++l) cadd(acc4, vvvv_ordered(J[i][k], J[k + 1][l], J[l + 1][j]));
          caxpy(acc, cx<T>{g * g * inv, T(0)}, acc4);
        }
        J[i][j] = acc;
      }
    }
    c4<T> U[NG];
    U[0] = ub;
    r4<T> Qu = K.pl[2];
#pragma unroll
    for (int k = 1; k < NG; ++k) {
      Qu = Qu + K.q[s[k - 1]];
      c4<T> acc = czero<T>();
#pragma unroll
      for (int j = 0; j < k; ++j) cadd(acc, row_slash(U[j], J[j][k - 1]));
      c4<T> pr = row_prop(acc, Qu, mt);
      cscale(pr, -g * K.iq[M[0][k - 1]]);
      U[k] = pr;
    }
    cx<T> a = cx<T>{T(0), T(0)};
#pragma unroll
    for (int j = 0; j < NG; ++j) a = a + spdot(row_slash(U[j], J[j][NG - 1]), vb);
    A[f] = times_i(a) * g;
  }
}

// t tbar + 2 or 3 gluons with every sub-current computed once per helicity.
// Colour-ordered currents obey the reflection identity J(s reversed) = (-1)^(k+1) J(s)
// for k gluons (V3 is antisymmetric in its two legs, the ordered V4 symmetric in its
// outer legs), so J(yx) = -J(xy) and J(zyx) = J(xyz); the quark currents U(x), U(xy)
// and the amplitudes of all orderings then reuse them.  Orderings are numbered
// lexicographically as in amp_ttng, so the colour basis is the same.
template <typename T>
ME_HD void amp_tt2_fast(const KinTT<T, 2>& K, int hel, const Couplings& cp, const c4<T>* ov, int ov_leg, cx<T>* A) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  const r4<T> k0 = K.q[0], k1 = K.q[1], kt = K.pl[2];
  const c4<T> e0 = (ov != nullptr && ov_leg == 0) ? *ov : polvec(K.pl[0], hel_of(hel, 0), false);
  const c4<T> e1 = (ov != nullptr && ov_leg == 1) ? *ov : polvec(K.pl[1], hel_of(hel, 1), false);
  const c4<T> ub = dbar(spinor_u(kt, mt, hel_of(hel, 2)));
  const c4<T> vb = spinor_v(K.pl[3], mt, hel_of(hel, 3));
  c4<T> J01 = vvv(e0, e1, -k0, -k1);
  cscale(J01, -g * K.ig[3]);
  const cx<T> s01 = spdot(row_slash(ub, J01), vb);
  c4<T> U0 = row_prop(row_slash(ub, e0), kt + k0, mt);
  cscale(U0, -g * K.iq[1]);
  c4<T> U1 = row_prop(row_slash(ub, e1), kt + k1, mt);
  cscale(U1, -g * K.iq[2]);
  // A(01) = ig[ub J01 v + U0 e1 v],  A(10) = ig[-ub J01 v + U1 e0 v]
  A[0] = times_i(s01 + spdot(row_slash(U0, e1), vb)) * g;
  A[1] = times_i(spdot(row_slash(U1, e0), vb) - s01) * g;
}

template <typename T>
ME_HD void amp_tt3_fast(const KinTT<T, 3>& K, int hel, const Couplings& cp, cx<T>* A) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  const r4<T> k0 = K.q[0], k1 = K.q[1], k2 = K.q[2], kt = K.pl[2];
  const c4<T> e0 = polvec(K.pl[0], hel_of(hel, 0), false);
  const c4<T> e1 = polvec(K.pl[1], hel_of(hel, 1), false);
  const c4<T> e2 = polvec(K.pl[4], hel_of(hel, 4), true);
  const c4<T> ub = dbar(spinor_u(kt, mt, hel_of(hel, 2)));
  const c4<T> vb = spinor_v(K.pl[3], mt, hel_of(hel, 3));
  // pair currents J(xy), x<y; J(yx) = -J(xy)
  c4<T> J01 = vvv(e0, e1, -k0, -k1);
  cscale(J01, -g * K.ig[3]);
  c4<T> J02 = vvv(e0, e2, -k0, -k2);
  cscale(J02, -g * K.ig[5]);
  c4<T> J12 = vvv(e1, e2, -k1, -k2);
  cscale(J12, -g * K.ig[6]);
  // three-gluon currents F(abc) = F(cba): -(g/Q^2)[V3(a, bc) + V3(ab, c)] + (g^2/Q^2) V4(a,b,c)
  const T c3 = -g * K.ig[7], c4g = g * g * K.ig[7];
  cx<T> a[6];
  {
    c4<T> F = vvv(e0, J12, -k0, -(k1 + k2));
    cadd(F, vvv(J01, e2, -(k0 + k1), -k2));
    cscale(F, c3);
    caxpy(F, cx<T>{c4g, T(0)}, vvvv_ordered(e0, e1, e2));
    a[0] = a[5] = spdot(row_slash(ub, F), vb);  // 012, 210
  }
  {
    c4<T> mJ12 = J12;
    cscale(mJ12, T(-1));
    c4<T> F = vvv(e0, mJ12, -k0, -(k1 + k2));
    cadd(F, vvv(J02, e1, -(k0 + k2), -k1));
    cscale(F, c3);
    caxpy(F, cx<T>{c4g, T(0)}, vvvv_ordered(e0, e2, e1));
    a[1] = a[3] = spdot(row_slash(ub, F), vb);  // 021, 120
  }
  {
    c4<T> mJ01 = J01;
    cscale(mJ01, T(-1));
    c4<T> F = vvv(e1, J02, -k1, -(k0 + k2));
    cadd(F, vvv(mJ01, e2, -(k0 + k1), -k2));
    cscale(F, c3);
    caxpy(F, cx<T>{c4g, T(0)}, vvvv_ordered(e1, e0, e2));
    a[2] = a[4] = spdot(row_slash(ub, F), vb);  // 102, 201
  }
  // orderings grouped by the gluon next to the top: U(x), then U(x y) = U(x) e_y + ubar J(xy)
  {  // x = 0: orderings 012 (a0), 021 (a1)
    c4<T> U = row_prop(row_slash(ub, e0), kt + k0, mt);
    cscale(U, -g * K.iq[1]);
    const cx<T> t = spdot(row_slash(U, J12), vb);
    a[0] = a[0] + t;
    a[1] = a[1] - t;
    c4<T> r = row_slash(U, e1);
    cadd(r, row_slash(ub, J01));
    c4<T> W = row_prop(r, kt + k0 + k1, mt);
    cscale(W, -g * K.iq[3]);
    a[0] = a[0] + spdot(row_slash(W, e2), vb);
    r = row_slash(U, e2);
    cadd(r, row_slash(ub, J02));
    W = row_prop(r, kt + k0 + k2, mt);
    cscale(W, -g * K.iq[5]);
    a[1] = a[1] + spdot(row_slash(W, e1), vb);
  }
  {  // x = 1: orderings 102 (a2), 120 (a3)
    c4<T> U = row_prop(row_slash(ub, e1), kt + k1, mt);
    cscale(U, -g * K.iq[2]);
    const cx<T> t = spdot(row_slash(U, J02), vb);
    a[2] = a[2] + t;
    a[3] = a[3] - t;
    c4<T> r = row_slash(U, e0);
    c4<T> b = row_slash(ub, J01);
    cscale(b, T(-1));
    cadd(r, b);
    c4<T> W = row_prop(r, kt + k0 + k1, mt);
    cscale(W, -g * K.iq[3]);
    a[2] = a[2] + spdot(row_slash(W, e2), vb);
    r = row_slash(U, e2);
    cadd(r, row_slash(ub, J12));
    W = row_prop(r, kt + k1 + k2, mt);
    cscale(W, -g * K.iq[6]);
    a[3] = a[3] + spdot(row_slash(W, e0), vb);
  }
  {  // x = 2: orderings 201 (a4), 210 (a5)
    c4<T> U = row_prop(row_slash(ub, e2), kt + k2, mt);
    cscale(U, -g * K.iq[4]);
    const cx<T> t = spdot(row_slash(U, J01), vb);
    a[4] = a[4] + t;
    a[5] = a[5] - t;
    c4<T> r = row_slash(U, e0);
    c4<T> b = row_slash(ub, J02);
    cscale(b, T(-1));
    cadd(r, b);
    c4<T> W = row_prop(r, kt + k0 + k2, mt);
    cscale(W, -g * K.iq[5]);
    a[4] = a[4] + spdot(row_slash(W, e1), vb);
    r = row_slash(U, e1);
    b = row_slash(ub, J12);
    cscale(b, T(-1));
    cadd(r, b);
    W = row_prop(r, kt + k1 + k2, mt);
    cscale(W, -g * K.iq[6]);
    a[5] = a[5] + spdot(row_slash(W, e0), vb);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) A[f] = times_i(a[f]) * g;
}

// ----------------------------------------------------------------------------
// Helicity blocks.  A block is one helicity configuration hb of every leg except the
// heavy pair (legs 2 and 3; their bits in hb are zero) together with the four (t, tbar)
// helicities hb | (r << 2), r = 0..3.  For t tbar + gluons the gluon currents depend on
// the gluon helicities only and the quark-line rows ubar(t) ... on the top helicity
// only, so a block builds the gluon currents once, the rows once per top helicity, and
// closes each row with both antitop spinors: the partial amplitudes of the four
// single-helicity evaluations, with the shared pieces computed once.
// consume(r, A) receives the partial amplitudes of helicity hb | (r << 2).

// g g -> t tbar.  A(01) = ig ubar [J01 + U0 e1] v,  A(10) = ig ubar [-J01 + U1 e0] v.
template <typename T, class F>
ME_HD void amp_tt2_block(const KinTT<T, 2>& K, int hb, const Couplings& cp, const c4<T>* ov, int ov_leg,
                         F&& consume) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  const r4<T> k0 = K.q[0], k1 = K.q[1], kt = K.pl[2];
  const c4<T> e0 = (ov != nullptr && ov_leg == 0) ? *ov : polvec_of(K.wg[0], hel_of(hb, 0), false);
  const c4<T> e1 = (ov != nullptr && ov_leg == 1) ? *ov : polvec_of(K.wg[1], hel_of(hb, 1), false);
  const c4<T> J01 = vvv(e0, e1, -k0, -k1, -g * K.ig[3]);
  const sl4<T> s0 = slashed(e0), s1 = slashed(e1), s01 = slashed(J01);
  const prop4<T> P0 = scaled_prop(kt + k0, mt, -g * K.iq[1]), P1 = scaled_prop(kt + k1, mt, -g * K.iq[2]);
  const c4<T> v[2] = {spinor_v_of(K.wtb, -1), spinor_v_of(K.wtb, 1)};
#pragma unroll
  for (int ht = 0; ht < 2; ++ht) {
    const c4<T> ub = dbar(spinor_u_of(K.wt, ht ? 1 : -1));
    const c4<T> S = row_slash(ub, s01);
    const c4<T> U0 = row_prop(row_slash(ub, s0), P0);
    const c4<T> U1 = row_prop(row_slash(ub, s1), P1);
    c4<T> R0 = S;
    row_slash_acc(R0, U0, s1);
    c4<T> R1 = cneg(S);
    row_slash_acc(R1, U1, s0);
#pragma unroll
    for (int hv = 0; hv < 2; ++hv) {
      cx<T> A[2] = {times_i(spdot(R0, v[hv])) * g, times_i(spdot(R1, v[hv])) * g};
      consume(ht | (hv << 1), A);
    }
  }
}

// g g -> t tbar g: the three-gluon currents F(012) = F(210), F(021) = F(120),
// F(102) = F(201) and the pair currents J(xy) are built once per block; per top
// helicity the row R_s of ordering s collects ubar F(s), U(x) J(yz) and W(xy) e_z.
template <typename T, class F>
ME_HD void amp_tt3_block(const KinTT<T, 3>& K, int hb, const Couplings& cp, F&& consume) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  const r4<T> k0 = K.q[0], k1 = K.q[1], k2 = K.q[2], kt = K.pl[2];
  const c4<T> e0 = polvec_of(K.wg[0], hel_of(hb, 0), false);
  const c4<T> e1 = polvec_of(K.wg[1], hel_of(hb, 1), false);
  const c4<T> e2 = polvec_of(K.wg[2], hel_of(hb, 4), true);
  const c4<T> J01 = vvv(e0, e1, -k0, -k1, -g * K.ig[3]);
  const c4<T> J02 = vvv(e0, e2, -k0, -k2, -g * K.ig[5]);
  const c4<T> J12 = vvv(e1, e2, -k1, -k2, -g * K.ig[6]);
  const T c3 = -g * K.ig[7], c4g = g * g * K.ig[7];
  c4<T> F0 = vvv(e0, J12, -k0, -(k1 + k2), c3);
  vvv_acc(F0, J01, e2, -(k0 + k1), -k2, c3);
  caxpy(F0, c4g, vvvv_ordered(e0, e1, e2));
  c4<T> F1 = vvv(J12, e0, -(k1 + k2), -k0, c3);  // = vvv(e0, -J12, ...) by antisymmetry
  vvv_acc(F1, J02, e1, -(k0 + k2), -k1, c3);
  caxpy(F1, c4g, vvvv_ordered(e0, e2, e1));
  c4<T> F2 = vvv(e1, J02, -k1, -(k0 + k2), c3);
  vvv_acc(F2, e2, J01, -k2, -(k0 + k1), c3);  // = vvv(-J01, e2, ...)
  caxpy(F2, c4g, vvvv_ordered(e1, e0, e2));
  const sl4<T> se0 = slashed(e0), se1 = slashed(e1), se2 = slashed(e2);
  const sl4<T> sJ01 = slashed(J01), sJ02 = slashed(J02), sJ12 = slashed(J12);
  const sl4<T> sF0 = slashed(F0), sF1 = slashed(F1), sF2 = slashed(F2);
  const c4<T> v[2] = {spinor_v_of(K.wtb, -1), spinor_v_of(K.wtb, 1)};
  const r4<T> Q0 = kt + k0, Q1 = kt + k1, Q2 = kt + k2;
  const prop4<T> P0 = scaled_prop(Q0, mt, -g * K.iq[1]), P1 = scaled_prop(Q1, mt, -g * K.iq[2]),
                 P2 = scaled_prop(Q2, mt, -g * K.iq[4]);
  const prop4<T> P01 = scaled_prop(Q0 + k1, mt, -g * K.iq[3]), P02 = scaled_prop(Q0 + k2, mt, -g * K.iq[5]),
                 P12 = scaled_prop(Q1 + k2, mt, -g * K.iq[6]);
#pragma unroll
  for (int ht = 0; ht < 2; ++ht) {
    const c4<T> ub = dbar(spinor_u_of(K.wt, ht ? 1 : -1));
    c4<T> R[6];
    R[0] = row_slash(ub, sF0);  // orderings 012, 021, 102, 120, 201, 210
    R[1] = row_slash(ub, sF1);
    R[2] = row_slash(ub, sF2);
    R[3] = R[1];
    R[4] = R[2];
    R[5] = R[0];
    const c4<T> S01 = row_slash(ub, sJ01), S02 = row_slash(ub, sJ02), S12 = row_slash(ub, sJ12);
    {  // first gluon 0: orderings 012, 021
      const c4<T> U = row_prop(row_slash(ub, se0), P0);
      const c4<T> t = row_slash(U, sJ12);
      cadd(R[0], t);
      csub(R[1], t);
      c4<T> r = S01;
      row_slash_acc(r, U, se1);
      row_slash_acc(R[0], row_prop(r, P01), se2);
      r = S02;
      row_slash_acc(r, U, se2);
      row_slash_acc(R[1], row_prop(r, P02), se1);
    }
    {  // first gluon 1: orderings 102, 120
      const c4<T> U = row_prop(row_slash(ub, se1), P1);
      const c4<T> t = row_slash(U, sJ02);
      cadd(R[2], t);
      csub(R[3], t);
      c4<T> r = cneg(S01);
      row_slash_acc(r, U, se0);
      row_slash_acc(R[2], row_prop(r, P01), se2);
      r = S12;
      row_slash_acc(r, U, se2);
      row_slash_acc(R[3], row_prop(r, P12), se0);
    }
    {  // first gluon 2: orderings 201, 210
      const c4<T> U = row_prop(row_slash(ub, se2), P2);
      const c4<T> t = row_slash(U, sJ01);
      cadd(R[4], t);
      csub(R[5], t);
      c4<T> r = cneg(S02);
      row_slash_acc(r, U, se0);
      row_slash_acc(R[4], row_prop(r, P02), se1);
      r = cneg(S12);
      row_slash_acc(r, U, se1);
      row_slash_acc(R[5], row_prop(r, P12), se0);
    }
#pragma unroll
    for (int hv = 0; hv < 2; ++hv) {
      cx<T> A[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) A[f] = times_i(spdot(R[f], v[hv])) * g;
      consume(ht | (hv << 1), A);
    }
  }
}

// ----------------------------------------------------------------------------
// e+(0) e-(1) -> u(2) ubar(3) [g(4)].  Photon exchange; charges Q_e = -1, Q_u = 2/3.
template <typename T>
struct KinEE {
  r4<T> pl[5];
  T is;      // 1/s of the photon
  T i1, i2;  // 1/(p_u+k)^2, 1/(p_ubar+k)^2 (real emission)
};

template <typename T, int NEXT>
ME_HD KinEE<T> prep_ee(const r4<double>* p) {
  KinEE<T> K;
  for (int l = 0; l < NEXT; ++l) K.pl[l] = cast4<T>(p[l]);
  const r4<double> Q = p[0] + p[1];
  K.is = T(1) / (T)mdot(Q, Q);
  K.i1 = K.i2 = T(0);
  if (NEXT == 5) {
    const r4<double> Q1 = p[2] + p[4], Q2 = p[3] + p[4];
    K.i1 = T(1) / (T)mdot(Q1, Q1);
    K.i2 = T(1) / (T)mdot(Q2, Q2);
  }
  return K;
}

template <typename T>
ME_HD c4<T> lepton_current(const KinEE<T>& K, int hel, const Couplings& cp) {
  // vbar(e+) gamma^mu u(e-) with the photon propagator: (e Q_e / s) vbar gamma u
  c4<T> vb = dbar(spinor_v(K.pl[0], T(0), hel_of(hel, 0)));
  c4<T> u = spinor_u(K.pl[1], T(0), hel_of(hel, 1));
  c4<T> L = vcurrent(vb, u);
  cscale(L, -(T)cp.ee * K.is);
  return L;
}

template <typename T>
ME_HD void amp_ee_uu(const KinEE<T>& K, int hel, const Couplings& cp, cx<T>* A) {
  c4<T> L = lepton_current<T>(K, hel, cp);
  c4<T> ub = dbar(spinor_u(K.pl[2], T(0), hel_of(hel, 2)));
  c4<T> v = spinor_v(K.pl[3], T(0), hel_of(hel, 3));
  const T equ = (T)(cp.ee * (2.0 / 3.0));
  A[0] = times_i(spdot(row_slash(ub, L), v)) * equ;
}

template <typename T>
ME_HD void amp_ee_uug(const KinEE<T>& K, int hel, const Couplings& cp, cx<T>* A) {
  c4<T> L = lepton_current<T>(K, hel, cp);
  c4<T> ub = dbar(spinor_u(K.pl[2], T(0), hel_of(hel, 2)));
  c4<T> v = spinor_v(K.pl[3], T(0), hel_of(hel, 3));
  c4<T> eps = polvec(K.pl[4], hel_of(hel, 4), true);
  const T g = (T)cp.gs;
  const T equ = (T)(cp.ee * (2.0 / 3.0));
  // gluon on the quark side: ubar (i g eps) i(Q1slash)/Q1^2, Q1 = p_u + p_g
  c4<T> u1 = row_prop(row_slash(ub, eps), K.pl[2] + K.pl[4], T(0));
  cscale(u1, -g * K.i1);
  // gluon on the antiquark side: i(-Q2slash)/Q2^2 (i g eps) v, Q2 = p_ubar + p_g
  c4<T> v1 = col_prop(K.pl[3] + K.pl[4], T(0), slash_col(eps, v));
  cscale(v1, -g * K.i2);
  cx<T> a = spdot(row_slash(u1, L), v) + spdot(row_slash(ub, L), v1);
  A[0] = times_i(a) * equ;
}

// ----------------------------------------------------------------------------
// u(0) ubar(1) -> t(2) tbar(3) [g(4)].  Colour basis (i=t, j=tbar, k=u, l=ubar):
//   Born: e1 = d_ik d_lj, e2 = d_ij d_lk;  (T^b)_ij (T^b)_lk = (e1 - e2/N)/2.
//   Real: e1 = T^a_ik d_lj, e2 = d_ik T^a_lj, e3 = T^a_ij d_lk, e4 = d_ij T^a_lk.
template <typename T>
struct KinUU {
  r4<T> pl[5];
  r4<T> q[5];  // outgoing momenta
  T is;        // 1/(q0+q1)^2
  T ia, ib;    // top / antitop propagators with the gluon
  T ic, id;    // light-quark propagators with the gluon
  T is3, it;   // 1/(q0+q1+q4)^2, 1/(q2+q3)^2
};

template <typename T, int NEXT>
ME_HD KinUU<T> prep_uu(const r4<double>* p, const Couplings& cp) {
  KinUU<T> K;
  r4<double> q[5];
  for (int l = 0; l < NEXT; ++l) {
    K.pl[l] = cast4<T>(p[l]);
    q[l] = l < 2 ? -p[l] : p[l];
    K.q[l] = l < 2 ? -K.pl[l] : K.pl[l];
  }
  const double m2 = cp.mt * cp.mt;
  const r4<double> s01 = q[0] + q[1];
  K.is = T(1) / (T)mdot(s01, s01);
  K.ia = K.ib = K.ic = K.id = K.is3 = K.it = T(0);
  if (NEXT == 5) {
    const r4<double> a = q[2] + q[4], b = q[3] + q[4], c = q[1] + q[4], d = q[0] + q[4];
    const r4<double> s3 = s01 + q[4], t = q[2] + q[3];
    K.ia = T(1) / (T)(mdot(a, a) - m2);
    K.ib = T(1) / (T)(mdot(b, b) - m2);
    K.ic = T(1) / (T)mdot(c, c);
    K.id = T(1) / (T)mdot(d, d);
    K.is3 = T(1) / (T)mdot(s3, s3);
    K.it = T(1) / (T)mdot(t, t);
  }
  return K;
}

template <typename T>
ME_HD c4<T> light_current(const c4<T>& vbar_ub, const c4<T>& u_u, T inv, T g) {
  // (g/Q^2) vbar gamma u  (vertex i g gamma, propagator -i/Q^2)
  c4<T> J = vcurrent(vbar_ub, u_u);
  cscale(J, g * inv);
  return J;
}

template <typename T>
ME_HD void amp_uu_tt(const KinUU<T>& K, int hel, const Couplings& cp, cx<T>* A) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  c4<T> uu = spinor_u(K.pl[0], T(0), hel_of(hel, 0));
  c4<T> vbu = dbar(spinor_v(K.pl[1], T(0), hel_of(hel, 1)));
  c4<T> ub = dbar(spinor_u(K.pl[2], mt, hel_of(hel, 2)));
  c4<T> vt = spinor_v(K.pl[3], mt, hel_of(hel, 3));
  c4<T> Ju = light_current(vbu, uu, K.is, g);
  cx<T> d = times_i(spdot(row_slash(ub, Ju), vt)) * g;
  A[0] = d * T(0.5);
  A[1] = d * (T)(-1.0 / 6.0);
}

template <typename T>
ME_HD void amp_uu_ttg(const KinUU<T>& K, int hel, const Couplings& cp, cx<T>* A) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  c4<T> uu = spinor_u(K.pl[0], T(0), hel_of(hel, 0));
  c4<T> vbu = dbar(spinor_v(K.pl[1], T(0), hel_of(hel, 1)));
  c4<T> ub = dbar(spinor_u(K.pl[2], mt, hel_of(hel, 2)));
  c4<T> vt = spinor_v(K.pl[3], mt, hel_of(hel, 3));
  c4<T> eps = polvec(K.pl[4], hel_of(hel, 4), true);
  const r4<T>* q = K.q;
  // u-line current without emission
  c4<T> Ju = light_current(vbu, uu, K.is, g);
  // D1: gluon off the top: ubar (ig eps) S_F(q2+q4) (ig Ju) v
  c4<T> r1 = row_prop(row_slash(ub, eps), q[2] + q[4], mt);
  cscale(r1, -g * K.ia);
  cx<T> D1 = times_i(spdot(row_slash(r1, Ju), vt)) * g;
  // D2: gluon off the antitop: ubar (ig Ju) S_F(-(q3+q4)) (ig eps) v
  c4<T> c1 = col_prop(q[3] + q[4], mt, slash_col(eps, vt));
  cscale(c1, -g * K.ib);
  cx<T> D2 = times_i(spdot(row_slash(ub, Ju), c1)) * g;
  // D3: gluon off the incoming antiquark (row side of the light line)
  c4<T> r3 = row_prop(row_slash(vbu, eps), q[1] + q[4], T(0));
  cscale(r3, -g * K.ic);
  c4<T> J3 = light_current(r3, uu, K.is3, g);
  cx<T> D3 = times_i(spdot(row_slash(ub, J3), vt)) * g;
  // D4: gluon off the incoming quark (column side)
  c4<T> c4u = col_prop(q[0] + q[4], T(0), slash_col(eps, uu));
  cscale(c4u, -g * K.id);
  c4<T> J4 = light_current(vbu, c4u, K.is3, g);
  cx<T> D4 = times_i(spdot(row_slash(ub, J4), vt)) * g;
  // D5: three-gluon vertex joining the light current, the heavy current and the gluon
  c4<T> Jt = vcurrent(ub, vt);
  cscale(Jt, g * K.it);
  c4<T> W = vvv(Ju, Jt, -(q[0] + q[1]), -(q[2] + q[3]));
  cx<T> D5 = cdot(W, eps) * g;
  const T h = T(0.5), hn = (T)(-1.0 / 6.0);
  cx<T> iD5 = times_i(D5);
  A[0] = (D1 + D4) * h - iD5 * h;
  A[1] = (D2 + D3) * h + iD5 * h;
  A[2] = (D1 + D2) * hn;
  A[3] = (D3 + D4) * hn;
}

// ----------------------------------------------------------------------------
template <int PID, typename T> struct KinOf;
template <typename T> struct KinOf<P_EE_UU, T> { using type = KinEE<T>; };
template <typename T> struct KinOf<P_EE_UUG, T> { using type = KinEE<T>; };
template <typename T> struct KinOf<P_GG_TT, T> { using type = KinTT<T, 2>; };
template <typename T> struct KinOf<P_GG_TTG, T> { using type = KinTT<T, 3>; };
template <typename T> struct KinOf<P_GG_TTGG, T> { using type = KinTT<T, 4>; };
template <typename T> struct KinOf<P_UU_TT, T> { using type = KinUU<T>; };
template <typename T> struct KinOf<P_UU_TTG, T> { using type = KinUU<T>; };
template <int PID, typename T> using Kin = typename KinOf<PID, T>::type;

// helicity-independent per-event kinematics
template <int PID, typename T>
ME_HD Kin<PID, T> prepare(const r4<double>* p, const Couplings& cp) {
  if constexpr (PID == P_EE_UU) return prep_ee<T, 4>(p);
  else if constexpr (PID == P_EE_UUG) return prep_ee<T, 5>(p);
  else if constexpr (PID == P_GG_TT) return prep_tt<T, 2>(p, cp);
  else if constexpr (PID == P_GG_TTG) return prep_tt<T, 3>(p, cp);
  else if constexpr (PID == P_GG_TTGG) return prep_tt<T, 4>(p, cp);
  else if constexpr (PID == P_UU_TT) return prep_uu<T, 4>(p, cp);
  else return prep_uu<T, 5>(p, cp);
}

// partial amplitudes of one helicity; `eps_override` replaces the polarisation of gluon
// leg `ov_leg` (g g -> t tbar only: the spin-correlated Born)
template <int PID, typename T>
ME_HD void amplitude(const Kin<PID, T>& K, int hel, const Couplings& cp, cx<T>* A,
                     const c4<T>* eps_override = nullptr, int ov_leg = -1) {
  if constexpr (PID == P_EE_UU) amp_ee_uu<T>(K, hel, cp, A);
  else if constexpr (PID == P_EE_UUG) amp_ee_uug<T>(K, hel, cp, A);
  else if constexpr (PID == P_GG_TT) amp_tt2_fast<T>(K, hel, cp, eps_override, ov_leg, A);
  else if constexpr (PID == P_GG_TTG) amp_tt3_fast<T>(K, hel, cp, A);
  else if constexpr (PID == P_GG_TTGG) amp_ttng<T, 4>(K, hel, cp, A);
  else if constexpr (PID == P_UU_TT) amp_uu_tt<T>(K, hel, cp, A);
  else amp_uu_ttg<T>(K, hel, cp, A);
}

// g g -> t tbar g g.  The ordered gluon currents are built once per block with the
// reflection identities: 6 pairs J(xy), x < y; 12 triples J(xyz) (one of each
// reversed pair); 12 quadruples J(wxyz) with w < z.  Per top helicity, the quark line
// is extended ordering by ordering, U(w) -> U(wx) -> U(wxy), and the row of ordering
// wxyz is ubar J(wxyz) + U(w) J(xyz) + U(wx) J(yz) + U(wxy) e_z.  Orderings are
// numbered lexicographically, as in amp_ttng.
template <typename T, class F>
ME_HD void amp_tt4_block(const KinTT<T, 4>& K, int hb, const Couplings& cp, F&& consume) {
  const T g = (T)cp.gs, mt = (T)cp.mt;
  constexpr int LEG[4] = {0, 1, 4, 5};
  c4<T> e[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) e[i] = polvec_of(K.wg[i], hel_of(hb, LEG[i]), LEG[i] >= 2);
  const r4<T>* q = K.q;
  // pair currents, index pidx(x, y) for x < y
  c4<T> J2[6];
  auto pidx = [](int x, int y) { return x == 0 ? y - 1 : (x == 1 ? y + 1 : 5); };
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = x + 1; y < 4; ++y) {
      J2[pidx(x, y)] = vvv(e[x], e[y], -q[x], -q[y], -g * K.ig[(1 << x) | (1 << y)]);
    }
  auto j2 = [&](int x, int y) {  // ordered pair current, J(yx) = -J(xy)
    c4<T> J = J2[x < y ? pidx(x, y) : pidx(y, x)];
    if (x > y) cscale(J, T(-1));
    return J;
  };
  // triple currents J(xyz) for x < z (J(zyx) = J(xyz)); index tidx = 3 * (missing gluon) + (middle slot)
  c4<T> J3[12];
  auto tidx = [](int x, int y, int z) {
    const int miss = 6 - x - y - z;
    // the three gluons of the triple in increasing order a < b < c; middle y in {a, b, c}
    const int a = miss == 0 ? 1 : 0;
    const int c = miss == 3 ? 2 : 3;
    return 3 * miss + (y == a ? 0 : (y == c ? 2 : 1));
  };
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int z = x + 1; z < 4; ++z) {
        if (y == x || y == z) continue;
        const int S = (1 << x) | (1 << y) | (1 << z);
        const T c3 = -g * K.ig[S], c4g = g * g * K.ig[S];
        c4<T> J = vvv(e[x], j2(y, z), -q[x], -(q[y] + q[z]), c3);
        vvv_acc(J, j2(x, y), e[z], -(q[x] + q[y]), -q[z], c3);
        caxpy(J, c4g, vvvv_ordered(e[x], e[y], e[z]));
        J3[tidx(x, y, z)] = J;
      }
  auto j3 = [&](int x, int y, int z) { return J3[tidx(x, y, z)]; };
  // quadruple currents J(wxyz) for w < z (J(zyxw) = -J(wxyz)); index by ordering rank
  c4<T> J4[12];
  int n4 = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        if (x == w || y == w || y == x) continue;
        const int z = 6 - w - x - y;
        if (z < w) continue;
        const T c3 = -g * K.ig[15], c4g = g * g * K.ig[15];
        c4<T> J = vvv(e[w], j3(x, y, z), -q[w], -(q[x] + q[y] + q[z]), c3);
        vvv_acc(J, j2(w, x), j2(y, z), -(q[w] + q[x]), -(q[y] + q[z]), c3);
        vvv_acc(J, j3(w, x, y), e[z], -(q[w] + q[x] + q[y]), -q[z], c3);
        c4<T> V = vvvv_ordered(e[w], e[x], j2(y, z));
        cadd(V, vvvv_ordered(e[w], j2(x, y), e[z]));
        cadd(V, vvvv_ordered(j2(w, x), e[y], e[z]));
        caxpy(J, c4g, V);
        J4[n4++] = J;
      }
  // rank of the quadruple current of ordering wxyz among those with first < last
  auto q4 = [](int w, int x, int y) {
    // enumeration order above: w ascending, then x, then y, keeping z > w
    int r = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int c = 0; c < 4; ++c) {
          if (b == a || c == a || c == b) continue;
          const int d = 6 - a - b - c;
          if (d < a) continue;
          if (a == w && b == x && c == y) return r;
          ++r;
        }
    return -1;
  };
  const c4<T> v[2] = {spinor_v_of(K.wtb, -1), spinor_v_of(K.wtb, 1)};
  const r4<T> kt = K.pl[2];
#pragma unroll 1
  for (int ht = 0; ht < 2; ++ht) {
    const c4<T> ub = dbar(spinor_u_of(K.wt, ht ? 1 : -1));
    cx<T> A[2][24];
    int f = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const c4<T> U1 = row_prop(row_slash(ub, e[w]), scaled_prop(kt + q[w], mt, -g * K.iq[1 << w]));
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        if (x == w) continue;
        c4<T> r2 = row_slash(ub, j2(w, x));
        row_slash_acc(r2, U1, e[x]);
        const c4<T> U2 = row_prop(r2, scaled_prop(kt + q[w] + q[x], mt, -g * K.iq[(1 << w) | (1 << x)]));
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          if (y == w || y == x) continue;
          const int z = 6 - w - x - y;
          c4<T> r3 = row_slash(ub, j3(w, x, y));
          row_slash_acc(r3, U1, j2(x, y));
          row_slash_acc(r3, U2, e[y]);
          const c4<T> U3 =
              row_prop(r3, scaled_prop(kt + q[w] + q[x] + q[y], mt, -g * K.iq[(1 << w) | (1 << x) | (1 << y)]));
          c4<T> J = z > w ? J4[q4(w, x, y)] : J4[q4(z, y, x)];
          if (z < w) cscale(J, T(-1));
          c4<T> R = row_slash(ub, J);
          row_slash_acc(R, U1, j3(x, y, z));
          row_slash_acc(R, U2, j2(y, z));
          row_slash_acc(R, U3, e[z]);
#pragma unroll
          for (int hv = 0; hv < 2; ++hv) A[hv][f] = times_i(spdot(R, v[hv])) * g;
          ++f;
        }
      }
    }
#pragma unroll
    for (int hv = 0; hv < 2; ++hv) consume(ht | (hv << 1), A[hv]);
  }
}

// Helicity blocks of one member of each flipped pair (leg 0 at +): NHEL / 8 blocks;
// block b sets legs 1, 4, 5 from the bits of b.
template <int PID> __host__ __device__ constexpr int n_blocks() { return Proc<PID>::NHEL / 8; }
ME_HD int block_hel(int b) { return 1 | ((b & 1) << 1) | ((b >> 1) << 4); }

// A massless fermion pair coupled through a vector current has opposite helicities
// (chirality is conserved at the vertex; the wrong-chirality spinor components are
// exactly zero): with legs 0, 1 such a pair (e+e-, u ubar), the blocks with leg 1 at +
// vanish identically and are skipped, and for e+e- -> u ubar (g) the heavy-pair slots
// (legs 2, 3 = u, ubar) with equal helicities vanish too.
template <int PID> __host__ __device__ constexpr bool massless_initial_pair() {
  return PID == P_EE_UU || PID == P_EE_UUG || PID == P_UU_TT || PID == P_UU_TTG;
}
template <int PID> __host__ __device__ constexpr int n_live_blocks() {
  return massless_initial_pair<PID>() ? n_blocks<PID>() / 2 : n_blocks<PID>();
}
template <int PID> ME_HD int live_block_hel(int i) { return block_hel(massless_initial_pair<PID>() ? 2 * i : i); }

// partial amplitudes of the four helicities hb | (r << 2) (see amp_tt2_block); processes
// without a block routine evaluate them one at a time
template <int PID, typename T, class F>
ME_HD void amplitude_block(const Kin<PID, T>& K, int hb, const Couplings& cp, F&& consume,
                           const c4<T>* eps_override = nullptr, int ov_leg = -1) {
  if constexpr (PID == P_GG_TT) {
    amp_tt2_block<T>(K, hb, cp, eps_override, ov_leg, consume);
  } else if constexpr (PID == P_GG_TTG) {
    amp_tt3_block<T>(K, hb, cp, consume);
  } else if constexpr (PID == P_GG_TTGG) {
    amp_tt4_block<T>(K, hb, cp, consume);
  } else {
    for (int r = 0; r < 4; ++r) {
      if constexpr (PID == P_EE_UU || PID == P_EE_UUG) {
        if (r == 0 || r == 3) continue;  // u, ubar with equal helicities: zero
      }
      cx<T> A[Proc<PID>::NFLOW];
      amplitude<PID, T>(K, hb | (r << 2), cp, A, eps_override, ov_leg);
      consume(r, A);
    }
  }
}

}  // namespace me
