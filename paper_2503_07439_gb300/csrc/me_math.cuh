// Device arithmetic for helicity amplitudes: complex numbers, four-vectors,
// Dirac spinors in the chiral representation, colour-stripped vertex routines.
//
// Conventions (standard QFT; the paper fixes none): metric (+,-,-,-); chiral
// gamma matrices gamma^0 = [[0,1],[1,0]], gamma^k = [[0,s^k],[-s^k,0]], so that
//   Vslash = [[0, V0 - s.V], [V0 + s.V, 0]];
// helicity spinors u(p,l) = (w_{-l} chi_l, w_{+l} chi_l),
//   v(p,l) = (-l w_{+l} chi_{-l}, l w_{-l} chi_{-l}), w_+- = sqrt(E +- |p|);
// polarisation vectors eps(k,l) = (-l e1 - i e2)/sqrt(2).
// Everything is templated on the arithmetic type T (float for the bulk path,
// double for the FP64 path and the rescue of unstable points).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

// Amplitude arithmetic compiles for the device and, for operation counting with a
// counting scalar type, for the host.
#ifndef ME_HD
#define ME_HD __host__ __device__ __forceinline__
#endif

namespace me {

// square root for every arithmetic type used by the amplitude code
ME_HD float msqrt(float x) { return sqrtf(x); }
ME_HD double msqrt(double x) { return ::sqrt(x); }

template <typename T>
struct cx {
  T re, im;
};

template <typename T> ME_HD cx<T> mk(T r, T i) { return cx<T>{r, i}; }
template <typename T> ME_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> ME_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> ME_HD cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <typename T> ME_HD cx<T> operator*(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> ME_HD cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> ME_HD cx<T> operator*(cx<T> a, T s) { return {s * a.re, s * a.im}; }
template <typename T> ME_HD cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
template <typename T> ME_HD cx<T> times_i(cx<T> a) { return {-a.im, a.re}; }
template <typename T> ME_HD T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// complex four-component object: a Lorentz vector with upper index, or a Dirac spinor
template <typename T>
struct c4 {
  cx<T> v[4];
};

template <typename T>
struct r4 {  // real four-vector (E, px, py, pz)
  T e, x, y, z;
};

template <typename T> ME_HD r4<T> operator+(r4<T> a, r4<T> b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T> ME_HD r4<T> operator-(r4<T> a, r4<T> b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T> ME_HD r4<T> operator-(r4<T> a) { return {-a.e, -a.x, -a.y, -a.z}; }
template <typename T> ME_HD r4<T> scale(T s, r4<T> a) { return {s * a.e, s * a.x, s * a.y, s * a.z}; }
template <typename T> ME_HD T mdot(r4<T> a, r4<T> b) { return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z; }
template <typename U, typename T> ME_HD r4<U> cast4(r4<T> a) { return {(U)a.e, (U)a.x, (U)a.y, (U)a.z}; }

// Sums of complex products are written as one left-to-right chain of real products, so
// that the compiler fuses every product after the first into the running sum (one
// fused multiply-add per real product).  Written as sums of complex temporaries, each
// complex product would end in a separate add: on GB300 float64 runs at 1/64 of the
// float32 rate, so the float64 path pays for every such add.
template <typename T> ME_HD cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {  // acc + a b
  return {acc.re + a.re * b.re - a.im * b.im, acc.im + a.re * b.im + a.im * b.re};
}
template <typename T> ME_HD cx<T> cmsb(cx<T> acc, cx<T> a, cx<T> b) {  // acc - a b
  return {acc.re - a.re * b.re + a.im * b.im, acc.im - a.re * b.im - a.im * b.re};
}

// complex-vector . complex-vector (Minkowski, no conjugation)
template <typename T>
ME_HD cx<T> cdot(const c4<T>& a, const c4<T>& b) {
  return cmsb(cmsb(cmsb(a.v[0] * b.v[0], a.v[1], b.v[1]), a.v[2], b.v[2]), a.v[3], b.v[3]);
}
// real-vector . complex-vector
template <typename T>
ME_HD cx<T> rdot(const r4<T>& a, const c4<T>& b) {
  return a.e * b.v[0] - a.x * b.v[1] - a.y * b.v[2] - a.z * b.v[3];
}
template <typename T>
ME_HD void cadd(c4<T>& acc, const c4<T>& x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.v[i] = acc.v[i] + x.v[i];
}
template <typename T>
ME_HD void csub(c4<T>& acc, const c4<T>& x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.v[i] = acc.v[i] - x.v[i];
}
template <typename T>
ME_HD void caxpy(c4<T>& acc, cx<T> a, const c4<T>& x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.v[i] = cmac(acc.v[i], a, x.v[i]);
}
// acc + s x, s real
template <typename T>
ME_HD void caxpy(c4<T>& acc, T s, const c4<T>& x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.v[i] = cx<T>{acc.v[i].re + s * x.v[i].re, acc.v[i].im + s * x.v[i].im};
}
template <typename T>
ME_HD c4<T> cneg(const c4<T>& x) {
  c4<T> o;
#pragma unroll
  for (int i = 0; i < 4; ++i) o.v[i] = -x.v[i];
  return o;
}
template <typename T>
ME_HD void cscale(c4<T>& x, cx<T> a) {
#pragma unroll
  for (int i = 0; i < 4; ++i) x.v[i] = a * x.v[i];
}
template <typename T>
ME_HD void cscale(c4<T>& x, T a) {
#pragma unroll
  for (int i = 0; i < 4; ++i) x.v[i] = a * x.v[i];
}
template <typename T>
ME_HD c4<T> czero() {
  c4<T> z;
#pragma unroll
  for (int i = 0; i < 4; ++i) z.v[i] = cx<T>{T(0), T(0)};
  return z;
}

// ---------------------------------------------------------------- wavefunctions
// two-component helicity eigenstate chi_lam along p/|p|; |p|+pz is formed without
// cancellation as pt^2/(|p|-pz) when pz < 0.
template <typename T>
ME_HD void chi(const r4<T>& p, int lam, cx<T>& c0, cx<T>& c1) {
  T pt2 = p.x * p.x + p.y * p.y;
  T pa = msqrt(pt2 + p.z * p.z);
  T s = (p.z >= T(0)) ? pa + p.z : pt2 / (pa - p.z);
  if (s > T(0)) {
    T rden = T(1) / msqrt(T(2) * pa * s);
    if (lam > 0) {
      c0 = cx<T>{s * rden, T(0)};
      c1 = cx<T>{p.x * rden, p.y * rden};
    } else {
      c0 = cx<T>{-p.x * rden, p.y * rden};
      c1 = cx<T>{s * rden, T(0)};
    }
  } else {  // exactly along -z
    if (lam > 0) {
      c0 = cx<T>{T(0), T(0)};
      c1 = cx<T>{T(1), T(0)};
    } else {
      c0 = cx<T>{T(-1), T(0)};
      c1 = cx<T>{T(0), T(0)};
    }
  }
}

template <typename T>
ME_HD void omegas(const r4<T>& p, T m, T& wp, T& wm) {
  T pa = msqrt(p.x * p.x + p.y * p.y + p.z * p.z);
  wp = msqrt(p.e + pa);
  wm = (m == T(0)) ? T(0) : m / wp;
}

template <typename T>
ME_HD c4<T> spinor_u(const r4<T>& p, T m, int lam) {
  T wp, wm;
  omegas(p, m, wp, wm);
  cx<T> a, b;
  chi(p, lam, a, b);
  T top = lam > 0 ? wm : wp, bot = lam > 0 ? wp : wm;
  return c4<T>{{top * a, top * b, bot * a, bot * b}};
}

template <typename T>
ME_HD c4<T> spinor_v(const r4<T>& p, T m, int lam) {
  T wp, wm;
  omegas(p, m, wp, wm);
  cx<T> a, b;
  chi(p, -lam, a, b);
  T top = lam > 0 ? -wp : wm;   // -lam * w_{+lam}
  T bot = lam > 0 ? wm : -wp;   //  lam * w_{-lam}
  return c4<T>{{top * a, top * b, bot * a, bot * b}};
}

// Dirac adjoint psi^dagger gamma^0 (chiral rep: swap blocks, conjugate)
template <typename T>
ME_HD c4<T> dbar(const c4<T>& s) {
  return c4<T>{{conj(s.v[2]), conj(s.v[3]), conj(s.v[0]), conj(s.v[1])}};
}

template <typename T>
ME_HD c4<T> polvec(const r4<T>& k, int lam, bool outgoing) {
  T pt2 = k.x * k.x + k.y * k.y;
  T pt = msqrt(pt2);
  T ka = msqrt(pt2 + k.z * k.z);
  T ct = k.z / ka, st = pt / ka;
  T cp = T(1), sp = T(0);
  if (pt > T(0)) {
    cp = k.x / pt;
    sp = k.y / pt;
  }
  const T r2 = T(0.70710678118654752440);
  // eps = (-lam e1 - i e2)/sqrt(2), e1 = (0, ct cp, ct sp, -st), e2 = (0, -sp, cp, 0)
  T l = (T)lam;
  c4<T> e;
  e.v[0] = cx<T>{T(0), T(0)};
  e.v[1] = cx<T>{-l * ct * cp * r2, sp * r2};
  e.v[2] = cx<T>{-l * ct * sp * r2, -cp * r2};
  e.v[3] = cx<T>{l * st * r2, T(0)};
  if (outgoing) {
#pragma unroll
    for (int i = 1; i < 4; ++i) e.v[i] = conj(e.v[i]);
  }
  return e;
}

// Helicity-independent ingredients of the wavefunctions, computed once per event and
// shared by all helicities (the same operations, in the same order, as the routines above).
// Fermion: omega_+, omega_- and the two-spinor chi_+ = (a, bx + i by), chi_- = (-bx + i by, a).
template <typename T>
struct wf_f {
  T wp, wm, a, bx, by;
};
template <typename T>
ME_HD wf_f<T> wf_fermion(const r4<T>& p, T m) {
  wf_f<T> w;
  omegas(p, m, w.wp, w.wm);
  T pt2 = p.x * p.x + p.y * p.y;
  T pa = msqrt(pt2 + p.z * p.z);
  T s = (p.z >= T(0)) ? pa + p.z : pt2 / (pa - p.z);
  if (s > T(0)) {
    T rden = T(1) / msqrt(T(2) * pa * s);
    w.a = s * rden;
    w.bx = p.x * rden;
    w.by = p.y * rden;
  } else {  // exactly along -z
    w.a = T(0);
    w.bx = T(1);
    w.by = T(0);
  }
  return w;
}
template <typename T>
ME_HD void chi_of(const wf_f<T>& w, int lam, cx<T>& c0, cx<T>& c1) {
  if (lam > 0) {
    c0 = cx<T>{w.a, T(0)};
    c1 = cx<T>{w.bx, w.by};
  } else {
    c0 = cx<T>{-w.bx, w.by};
    c1 = cx<T>{w.a, T(0)};
  }
}
template <typename T>
ME_HD c4<T> spinor_u_of(const wf_f<T>& w, int lam) {
  cx<T> a, b;
  chi_of(w, lam, a, b);
  T top = lam > 0 ? w.wm : w.wp, bot = lam > 0 ? w.wp : w.wm;
  return c4<T>{{top * a, top * b, bot * a, bot * b}};
}
template <typename T>
ME_HD c4<T> spinor_v_of(const wf_f<T>& w, int lam) {
  cx<T> a, b;
  chi_of(w, -lam, a, b);
  T top = lam > 0 ? -w.wp : w.wm;
  T bot = lam > 0 ? w.wm : -w.wp;
  return c4<T>{{top * a, top * b, bot * a, bot * b}};
}
// Vector: (ct cp, ct sp, st, sp, cp) / sqrt(2) of the momentum direction.
template <typename T>
struct wf_v {
  T ccp, csp, st, sp, cp;
};
template <typename T>
ME_HD wf_v<T> wf_vector(const r4<T>& k) {
  T pt2 = k.x * k.x + k.y * k.y;
  T pt = msqrt(pt2);
  T ka = msqrt(pt2 + k.z * k.z);
  T ct = k.z / ka, st = pt / ka;
  T cp = T(1), sp = T(0);
  if (pt > T(0)) {
    cp = k.x / pt;
    sp = k.y / pt;
  }
  const T r2 = T(0.70710678118654752440);
  return wf_v<T>{ct * cp * r2, ct * sp * r2, st * r2, sp * r2, cp * r2};
}
template <typename T>
ME_HD c4<T> polvec_of(const wf_v<T>& w, int lam, bool outgoing) {
  // eps = (-lam e1 - i e2)/sqrt(2), as polvec
  c4<T> e;
  e.v[0] = cx<T>{T(0), T(0)};
  e.v[1] = cx<T>{lam > 0 ? -w.ccp : w.ccp, w.sp};
  e.v[2] = cx<T>{lam > 0 ? -w.csp : w.csp, -w.cp};
  e.v[3] = cx<T>{lam > 0 ? w.st : -w.st, T(0)};
  if (outgoing) {
#pragma unroll
    for (int i = 1; i < 4; ++i) e.v[i] = conj(e.v[i]);
  }
  return e;
}

// ---------------------------------------------------------------- Dirac algebra
// row spinor times Vslash (V complex, upper index)
template <typename T>
ME_HD c4<T> row_slash(const c4<T>& r, const c4<T>& V) {
  cx<T> a = V.v[0] - V.v[3], b = V.v[0] + V.v[3];
  cx<T> c = V.v[1] - times_i(V.v[2]);  // V1 - i V2
  cx<T> d = V.v[1] + times_i(V.v[2]);  // V1 + i V2
  c4<T> o;
  o.v[0] = cmac(r.v[2] * b, r.v[3], d);
  o.v[1] = cmac(r.v[2] * c, r.v[3], a);
  o.v[2] = cmsb(r.v[0] * a, r.v[1], d);
  o.v[3] = cmsb(r.v[1] * b, r.v[0], c);
  return o;
}
// Vslash in the chiral representation is fixed by four combinations of V: a = V0 - V3,
// b = V0 + V3, c = V1 - i V2, d = V1 + i V2.  A vector that is slashed against many rows
// is converted once.
template <typename T>
struct sl4 {
  cx<T> a, b, c, d;
};
template <typename T>
ME_HD sl4<T> slashed(const c4<T>& V) {
  return sl4<T>{V.v[0] - V.v[3], V.v[0] + V.v[3], V.v[1] - times_i(V.v[2]), V.v[1] + times_i(V.v[2])};
}
template <typename T>
ME_HD c4<T> row_slash(const c4<T>& r, const sl4<T>& S) {
  c4<T> o;
  o.v[0] = cmac(r.v[2] * S.b, r.v[3], S.d);
  o.v[1] = cmac(r.v[2] * S.c, r.v[3], S.a);
  o.v[2] = cmsb(r.v[0] * S.a, r.v[1], S.d);
  o.v[3] = cmsb(r.v[1] * S.b, r.v[0], S.c);
  return o;
}
// acc + r Sslash, accumulated in place
template <typename T>
ME_HD void row_slash_acc(c4<T>& acc, const c4<T>& r, const sl4<T>& S) {
  acc.v[0] = cmac(cmac(acc.v[0], r.v[2], S.b), r.v[3], S.d);
  acc.v[1] = cmac(cmac(acc.v[1], r.v[2], S.c), r.v[3], S.a);
  acc.v[2] = cmsb(cmac(acc.v[2], r.v[0], S.a), r.v[1], S.d);
  acc.v[3] = cmac(cmsb(acc.v[3], r.v[0], S.c), r.v[1], S.b);
}
template <typename T>
ME_HD void row_slash_acc(c4<T>& acc, const c4<T>& r, const c4<T>& V) {
  row_slash_acc(acc, r, slashed(V));
}
// Vslash times column spinor
template <typename T>
ME_HD c4<T> slash_col(const c4<T>& V, const c4<T>& s) {
  cx<T> a = V.v[0] - V.v[3], b = V.v[0] + V.v[3];
  cx<T> c = V.v[1] - times_i(V.v[2]);
  cx<T> d = V.v[1] + times_i(V.v[2]);
  c4<T> o;
  o.v[0] = cmsb(a * s.v[2], c, s.v[3]);
  o.v[1] = cmsb(b * s.v[3], d, s.v[2]);
  o.v[2] = cmac(b * s.v[0], c, s.v[1]);
  o.v[3] = cmac(d * s.v[0], a, s.v[1]);
  return o;
}
// row spinor times (Qslash + m), Q real
template <typename T>
ME_HD c4<T> row_prop(const c4<T>& r, const r4<T>& Q, T m) {
  T a = Q.e - Q.z, b = Q.e + Q.z;
  cx<T> c = cx<T>{Q.x, -Q.y}, d = cx<T>{Q.x, Q.y};
  c4<T> o;
  o.v[0] = cmac(b * r.v[2] + m * r.v[0], r.v[3], d);
  o.v[1] = cmac(a * r.v[3] + m * r.v[1], r.v[2], c);
  o.v[2] = cmsb(a * r.v[0] + m * r.v[2], r.v[1], d);
  o.v[3] = cmsb(b * r.v[1] + m * r.v[3], r.v[0], c);
  return o;
}
// s (Qslash + m) for rows, Q real: the combinations row_prop uses, formed once for a
// propagator that closes several rows (the scale s, a coupling times the reciprocal
// denominator, is folded in here instead of into every row)
template <typename T>
struct prop4 {
  T a, b, m;
  cx<T> c, d;
};
template <typename T>
ME_HD prop4<T> scaled_prop(const r4<T>& Q, T m, T s) {
  const T sx = s * Q.x, sy = s * Q.y;
  return prop4<T>{s * (Q.e - Q.z), s * (Q.e + Q.z), s * m, cx<T>{sx, -sy}, cx<T>{sx, sy}};
}
template <typename T>
ME_HD c4<T> row_prop(const c4<T>& r, const prop4<T>& P) {
  c4<T> o;
  o.v[0] = cmac(P.b * r.v[2] + P.m * r.v[0], r.v[3], P.d);
  o.v[1] = cmac(P.a * r.v[3] + P.m * r.v[1], r.v[2], P.c);
  o.v[2] = cmsb(P.a * r.v[0] + P.m * r.v[2], r.v[1], P.d);
  o.v[3] = cmsb(P.b * r.v[1] + P.m * r.v[3], r.v[0], P.c);
  return o;
}
// (-Qslash + m) times column spinor, Q real
template <typename T>
ME_HD c4<T> col_prop(const r4<T>& Q, T m, const c4<T>& s) {
  T a = Q.e - Q.z, b = Q.e + Q.z;
  cx<T> c = cx<T>{Q.x, -Q.y}, d = cx<T>{Q.x, Q.y};
  c4<T> o;
  o.v[0] = cmac(m * s.v[0] - a * s.v[2], c, s.v[3]);
  o.v[1] = cmac(m * s.v[1] - b * s.v[3], d, s.v[2]);
  o.v[2] = cmsb(m * s.v[2] - b * s.v[0], c, s.v[1]);
  o.v[3] = cmsb(m * s.v[3] - a * s.v[1], d, s.v[0]);
  return o;
}
// vector current J^mu = r gamma^mu s
template <typename T>
ME_HD c4<T> vcurrent(const c4<T>& r, const c4<T>& s) {
  c4<T> J;
  J.v[0] = cmac(cmac(cmac(r.v[0] * s.v[2], r.v[1], s.v[3]), r.v[2], s.v[0]), r.v[3], s.v[1]);
  J.v[1] = cmsb(cmsb(cmac(r.v[0] * s.v[3], r.v[1], s.v[2]), r.v[2], s.v[1]), r.v[3], s.v[0]);
  J.v[2] = times_i(cmac(cmsb(cmsb(r.v[1] * s.v[2], r.v[0], s.v[3]), r.v[3], s.v[0]), r.v[2], s.v[1]));
  J.v[3] = cmac(cmsb(cmsb(r.v[0] * s.v[2], r.v[1], s.v[3]), r.v[2], s.v[0]), r.v[3], s.v[1]);
  return J;
}
template <typename T>
ME_HD cx<T> spdot(const c4<T>& r, const c4<T>& s) {
  return cmac(cmac(cmac(r.v[0] * s.v[0], r.v[1], s.v[1]), r.v[2], s.v[2]), r.v[3], s.v[3]);
}

// ---------------------------------------------------------------- gluon vertices
// three-gluon Lorentz structure contracted with J1_mu J2_nu, momenta k1,k2,k3 incoming:
// W^rho = (J1.J2)(k1-k2)^rho + J2^rho (k2-k3).J1 + J1^rho (k3-k1).J2
template <typename T>
ME_HD c4<T> vvv(const c4<T>& J1, const c4<T>& J2, const r4<T>& k1, const r4<T>& k2) {
  r4<T> k3 = -(k1 + k2);
  cx<T> j12 = cdot(J1, J2);
  cx<T> a = rdot(k2 - k3, J1);
  cx<T> b = rdot(k3 - k1, J2);
  r4<T> d = k1 - k2;
  c4<T> W;
  W.v[0] = cmac(cmac(d.e * j12, a, J2.v[0]), b, J1.v[0]);
  W.v[1] = cmac(cmac(d.x * j12, a, J2.v[1]), b, J1.v[1]);
  W.v[2] = cmac(cmac(d.y * j12, a, J2.v[2]), b, J1.v[2]);
  W.v[3] = cmac(cmac(d.z * j12, a, J2.v[3]), b, J1.v[3]);
  return W;
}
// s W(J1, J2), and acc + s W(J1, J2): the scale goes into the three scalar coefficients
template <typename T>
ME_HD c4<T> vvv(const c4<T>& J1, const c4<T>& J2, const r4<T>& k1, const r4<T>& k2, T s) {
  r4<T> k3 = -(k1 + k2);
  const cx<T> j12 = s * cdot(J1, J2);
  const cx<T> a = s * rdot(k2 - k3, J1);
  const cx<T> b = s * rdot(k3 - k1, J2);
  r4<T> d = k1 - k2;
  c4<T> W;
  W.v[0] = cmac(cmac(d.e * j12, a, J2.v[0]), b, J1.v[0]);
  W.v[1] = cmac(cmac(d.x * j12, a, J2.v[1]), b, J1.v[1]);
  W.v[2] = cmac(cmac(d.y * j12, a, J2.v[2]), b, J1.v[2]);
  W.v[3] = cmac(cmac(d.z * j12, a, J2.v[3]), b, J1.v[3]);
  return W;
}
template <typename T>
ME_HD void vvv_acc(c4<T>& acc, const c4<T>& J1, const c4<T>& J2, const r4<T>& k1, const r4<T>& k2, T s) {
  r4<T> k3 = -(k1 + k2);
  const cx<T> j12 = s * cdot(J1, J2);
  const cx<T> a = s * rdot(k2 - k3, J1);
  const cx<T> b = s * rdot(k3 - k1, J2);
  r4<T> d = k1 - k2;
  const T dd[4] = {d.e, d.x, d.y, d.z};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const cx<T> t{acc.v[i].re + dd[i] * j12.re, acc.v[i].im + dd[i] * j12.im};
    acc.v[i] = cmac(cmac(t, a, J2.v[i]), b, J1.v[i]);
  }
}
// colour-ordered four-gluon structure: 2(L.R) M - (L.M) R - (M.R) L
template <typename T>
ME_HD c4<T> vvvv_ordered(const c4<T>& L, const c4<T>& M, const c4<T>& R) {
  cx<T> lr = cdot(L, R), lm = cdot(L, M), mr = cdot(M, R);
  cx<T> two_lr = lr + lr;
  c4<T> o;
#pragma unroll
  for (int i = 0; i < 4; ++i) o.v[i] = cmsb(cmsb(two_lr * M.v[i], lm, R.v[i]), mr, L.v[i]);
  return o;
}

}  // namespace me
