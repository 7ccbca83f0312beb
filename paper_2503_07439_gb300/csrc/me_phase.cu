// Flat phase-space points generated on the device: the multi-event input (Sec. 4.4,
// step 1) produced where the matrix elements consume it, instead of on the host.
//
//  * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
//    random numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
//    Counter (point index lo, point index hi, stream, block), key (seed lo, seed hi).
//    Block b of point i gives the uniforms 2b and 2b+1 as 53-bit doubles in (0, 1):
//    ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) 2^-53 from the word pairs (w0, w1), (w2, w3).
//  * RAMBO (Kleiss, Stirling and Ellis, Comput. Phys. Commun. 40 (1986) 359): massless
//    momenta from isotropic directions with energies -log(u u'), boosted and scaled to the
//    centre-of-mass energy; constant weight (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2)/((n-1)!(n-2)!).
//    For massive particles the published rescaling k = (sqrt(m^2 + x^2 |p|^2), x p), x from
//    energy conservation by Newton iteration, with the weight factor
//    (sum |k| / sqrt s)^(2n-3) prod(|k|/E) sqrt(s) / sum(|k|^2/E).
// The two incoming beams are massless along +z and -z.  One thread per point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/me.h"
#include "me_internal.h"

namespace {

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    philox_round(c, k0, k1);
  }
}

__device__ __forceinline__ double u01(uint32_t w0, uint32_t w1) {
  return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

struct Masses {
  double m[4];
};

// RAMBO point from 4 NOUT uniforms: final momenta k[j][0..3] and the weight.
template <int NOUT>
__device__ __forceinline__ void rambo_point(const double* u, double rs, const double* masses, double w_massless,
                                            double k[][4], double& w_out) {
  // massless momenta
  double q[NOUT][4], Q[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < NOUT; ++j) {
    const double c = 2.0 * u[4 * j] - 1.0;
    const double s = sqrt(1.0 - c * c);
    const double f = 2.0 * M_PI * u[4 * j + 1];
    const double q0 = -log(u[4 * j + 2] * u[4 * j + 3]);
    double sf, cf;
    sincos(f, &sf, &cf);
    q[j][0] = q0;
    q[j][1] = q0 * s * cf;
    q[j][2] = q0 * s * sf;
    q[j][3] = q0 * c;
#pragma unroll
    for (int a = 0; a < 4; ++a) Q[a] += q[j][a];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double x = rs / M, g = Q[0] / M, a = 1.0 / (1.0 + g);
#pragma unroll
  for (int j = 0; j < NOUT; ++j) {
    const double bq = b[0] * q[j][1] + b[1] * q[j][2] + b[2] * q[j][3];
    k[j][0] = x * (g * q[j][0] + bq);
#pragma unroll
    for (int d = 0; d < 3; ++d) k[j][1 + d] = x * (q[j][1 + d] + b[d] * q[j][0] + a * bq * b[d]);
  }
  // massive rescaling
  double w = w_massless, msum = 0.0;
  bool massive = false;
#pragma unroll
  for (int j = 0; j < NOUT; ++j) {
    msum += masses[j];
    massive |= masses[j] != 0.0;
  }
  if (massive) {
    double pabs[NOUT];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) pabs[j] = k[j][0];
    double xs = sqrt(fmax(0.0, 1.0 - (msum / rs) * (msum / rs)));
    for (int it = 0; it < 60; ++it) {
      double fs = -rs, df = 0.0;
#pragma unroll
      for (int j = 0; j < NOUT; ++j) {
        const double e = sqrt(masses[j] * masses[j] + (xs * pabs[j]) * (xs * pabs[j]));
        fs += e;
        df += xs * pabs[j] * pabs[j] / e;
      }
      const double dx = fs / df;
      xs -= dx;
      // Newton converges quadratically: a step below 1e-15 of xs leaves xs exact to
      // rounding (an absolute 1e-16 would sit below the rounding of xs ~ 1 and run
      // all 60 steps)
      if (fabs(dx) <= 1e-15 * xs) break;
    }
    double sk = 0.0, prod = 1.0, sk2e = 0.0;
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      const double ka = xs * pabs[j];
      const double e = sqrt(masses[j] * masses[j] + ka * ka);
      k[j][0] = e;
#pragma unroll
      for (int d = 1; d < 4; ++d) k[j][d] *= xs;
      sk += ka;
      prod *= ka / e;
      sk2e += ka * ka / e;
    }
    double pw = 1.0;  // (sum |k| / sqrt s)^(2n-3)
#pragma unroll
    for (int e = 0; e < 2 * NOUT - 3; ++e) pw *= sk / rs;
    w *= pw * prod * rs / sk2e;
  }
  w_out = w;
}

template <int NOUT>
__global__ void k_rambo(uint64_t seed, uint32_t stream, long long first, double rs, Masses ms, double w_massless, long n,
                        double* __restrict__ p, double* __restrict__ wgt) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NEXT = NOUT + 2;
  const unsigned long long idx = (unsigned long long)(first + i);
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  double u[4 * NOUT];
#pragma unroll
  for (int b = 0; b < 2 * NOUT; ++b) {
    uint32_t c[4] = {(uint32_t)(idx & 0xFFFFFFFFull), (uint32_t)(idx >> 32), stream, (uint32_t)b};
    philox4x32_10(c, k0, k1);
    u[2 * b] = u01(c[0], c[1]);
    u[2 * b + 1] = u01(c[2], c[3]);
  }
  double k[NOUT][4], w;
  rambo_point<NOUT>(u, rs, ms.m, w_massless, k, w);
  // beams, then the outgoing momenta: p[comp][leg][n]
  const double hb = 0.5 * rs;
  const double beams[2][4] = {{hb, 0.0, 0.0, hb}, {hb, 0.0, 0.0, -hb}};
#pragma unroll
  for (int comp = 0; comp < 4; ++comp) {
    p[(comp * NEXT + 0) * n + i] = beams[0][comp];
    p[(comp * NEXT + 1) * n + i] = beams[1][comp];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) p[(comp * NEXT + 2 + j) * n + i] = k[j][comp];
  }
  if (wgt) wgt[i] = w;
}

// ---------------------------------------------------------------- points in FKS variables
// Real-emission points from a multichannel density whose channels are the variables of the
// two FKS sectors plus flat phase space (RAMBO).  u0 picks the channel: flat with share
// kAlphaFlat, else one sector (equal shares).  A sector channel is flat in the emitted
// gluon's energy fraction xi (flat three-body phase space has density ~ xi there) and
// samples its cosine to the sector's reference direction as y_j = 1 - 2 v^2, v uniform in
// (v_min, 1), 2 v_min^2 = kYCut (density g(y) = 1 / (4 v (1 - v_min)) ~ 1/sqrt(1 - y)),
// azimuth and Born direction uniform.  The weight is the phase-space measure over the sum
// of all channel densities at the point, 1 / (a_flat / w_RAMBO + sum_j a_j h_j): bounded
// by w_RAMBO / a_flat where the sector channels are thin, and no sector channel comes
// closer than kYCut to a collinear limit (the flat channel covers that region).
// Uniforms: u0..u17 of point i from Philox blocks 0..8 at counter (i lo, i hi, stream,
// block); the flat channel's RAMBO takes u6..u17.
constexpr double kAlphaFlat = 0.25;
constexpr double kYCut = 1e-6;

__device__ __forceinline__ double coll_density(double y) {
  const double vmin = sqrt(0.5 * kYCut);
  const double omy = 1.0 - y;
  if (!(omy >= kYCut)) return 0.0;
  return 1.0 / (4.0 * sqrt(0.5 * omy) * (1.0 - vmin));
}

__device__ __forceinline__ void boost_vel(const double p[4], const double b[3], double out[4]) {
  const double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double g = 1.0 / sqrt(1.0 - b2);
  const double bp = b[0] * p[1] + b[1] * p[2] + b[2] * p[3];
  const double g2 = b2 > 0.0 ? (g - 1.0) / b2 : 0.0;
  out[0] = g * (p[0] + bp);
#pragma unroll
  for (int d = 0; d < 3; ++d) out[1 + d] = p[1 + d] + (g2 * bp + g * p[0]) * b[d];
}

// Initial-state sectors of 2 -> Q Qbar g (beams j = 0 along +z, 1 along -z, Q mass
// `mass`): xi = xi_max u1, v from u2, phi = 2 pi u3, the pair's rest-frame direction
// (2 u4 - 1, 2 pi u5); the pair recoils against the gluon with mass^2 s (1 - xi).
// dPhi_3 = dPhi_2(s) xi K dxi dy dphi, K = s beta(s(1-xi)) / (64 pi^3 beta(s)):
// channel density h_j = 4 g(y_j) / (xi_max beta(s) xi K).
// Final-state sectors of massless 2 -> 3 (partner leg 2 or 3, along (2 u1 - 1, 2 pi u2)):
// xi = u3, v from u4, phi = 2 pi u5 about the partner; the partner's energy
// sqrt(s)(1-xi)/(2 - xi(1-y_j)) leaves the third parton massless; channel density
// h_j = 4 g(y_j) / (xi K_j), K_j = s (1 - xi) / (16 pi^3 (2 - xi (1 - y_j))^2).
template <bool ISR>
__global__ void k_fks_points(uint64_t seed, uint32_t stream, long long first, double rs, double mass, double w3_massless,
                             long n, double* __restrict__ p, double* __restrict__ wgt) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long idx = (unsigned long long)(first + i);
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  double u[18];
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    uint32_t c[4] = {(uint32_t)(idx & 0xFFFFFFFFull), (uint32_t)(idx >> 32), stream, (uint32_t)b};
    philox4x32_10(c, k0, k1);
    u[2 * b] = u01(c[0], c[1]);
    u[2 * b + 1] = u01(c[2], c[3]);
  }
  const double s = rs * rs;
  const double a_f = kAlphaFlat, a_s = 0.5 * (1.0 - kAlphaFlat);
  const bool flat = u[0] < a_f;
  const int sec = u[0] < a_f + a_s ? 0 : 1;
  const double vmin = sqrt(0.5 * kYCut);
  const double masses[3] = {ISR ? mass : 0.0, ISR ? mass : 0.0, 0.0};
  double q[5][4];  // legs: beams, then 2, 3, 4 (gluon)
  const double hb = 0.5 * rs;
  q[0][0] = hb; q[0][1] = 0.0; q[0][2] = 0.0; q[0][3] = hb;
  q[1][0] = hb; q[1][1] = 0.0; q[1][2] = 0.0; q[1][3] = -hb;
  if (flat) {
    double k[3][4], wr;
    rambo_point<3>(u + 6, rs, masses, w3_massless, k, wr);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) q[2 + j][c] = k[j][c];
  } else if (ISR) {
    const double ximax = 1.0 - 4.0 * mass * mass / s;
    const double xi = ximax * u[1];
    const double v = vmin + (1.0 - vmin) * u[2];
    const double yj = 1.0 - 2.0 * v * v;
    const double y = sec == 0 ? yj : -yj;
    double sf, cf, sp2, cp2;
    sincos(2.0 * M_PI * u[3], &sf, &cf);
    const double ek = 0.5 * rs * xi;
    const double st = sqrt(fmax(0.0, (1.0 - y) * (1.0 + y)));
    q[4][0] = ek;
    q[4][1] = ek * st * cf;
    q[4][2] = ek * st * sf;
    q[4][3] = ek * y;
    const double Q0 = rs - ek, M2 = Q0 * Q0 - ek * ek, M = sqrt(M2);
    const double pstar = sqrt(fmax(0.0, 0.25 * M2 - mass * mass));
    const double cp = 2.0 * u[4] - 1.0;
    const double sp = sqrt(fmax(0.0, (1.0 - cp) * (1.0 + cp)));
    sincos(2.0 * M_PI * u[5], &sp2, &cp2);
    const double nv[3] = {sp * cp2, sp * sp2, cp};
    const double e = 0.5 * M;
    const double p3[4] = {e, pstar * nv[0], pstar * nv[1], pstar * nv[2]};
    const double p4[4] = {e, -pstar * nv[0], -pstar * nv[1], -pstar * nv[2]};
    const double bvec[3] = {-q[4][1] / Q0, -q[4][2] / Q0, -q[4][3] / Q0};
    boost_vel(p3, bvec, q[2]);
    boost_vel(p4, bvec, q[3]);
  } else {
    const int partner = 2 + sec, other = 5 - partner;
    const double cdir = 2.0 * u[1] - 1.0, xi = u[3];
    const double v = vmin + (1.0 - vmin) * u[4];
    const double yj = 1.0 - 2.0 * v * v;
    double spd, cpd, sf, cf;
    sincos(2.0 * M_PI * u[2], &spd, &cpd);
    sincos(2.0 * M_PI * u[5], &sf, &cf);
    const double sd = sqrt(fmax(0.0, (1.0 - cdir) * (1.0 + cdir)));
    const double nj[3] = {sd * cpd, sd * spd, cdir};
    double ea[3] = {-cdir * nj[0], -cdir * nj[1], 1.0 - cdir * nj[2]};  // z - (z.nj) nj
    const double ia = 1.0 / sqrt(ea[0] * ea[0] + ea[1] * ea[1] + ea[2] * ea[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) ea[d] *= ia;
    const double eb[3] = {nj[1] * ea[2] - nj[2] * ea[1], nj[2] * ea[0] - nj[0] * ea[2], nj[0] * ea[1] - nj[1] * ea[0]};
    const double sr = sqrt(fmax(0.0, (1.0 - yj) * (1.0 + yj)));
    double ni[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ni[d] = yj * nj[d] + sr * (cf * ea[d] + sf * eb[d]);
    const double ei = 0.5 * rs * xi, ej = rs * (1.0 - xi) / (2.0 - xi * (1.0 - yj));
    q[partner][0] = ej;
    q[4][0] = ei;
    q[other][0] = rs - ej - ei;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      q[partner][1 + d] = ej * nj[d];
      q[4][1 + d] = ei * ni[d];
      q[other][1 + d] = -(ej * nj[d] + ei * ni[d]);
    }
  }
  // every channel's density at this point, from its momenta
  double h;
  {
    double kabs[3], sk = 0.0, prod = 1.0, sk2e = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      kabs[j] = sqrt(q[2 + j][1] * q[2 + j][1] + q[2 + j][2] * q[2 + j][2] + q[2 + j][3] * q[2 + j][3]);
      sk += kabs[j];
      prod *= kabs[j] / q[2 + j][0];
      sk2e += kabs[j] * kabs[j] / q[2 + j][0];
    }
    const double wr = ISR ? w3_massless * (sk / rs) * (sk / rs) * (sk / rs) * prod * rs / sk2e : w3_massless;
    h = a_f / wr;
  }
  const double ig = 1.0 / sqrt(q[4][1] * q[4][1] + q[4][2] * q[4][2] + q[4][3] * q[4][3]);
  const double xi_pt = 2.0 * q[4][0] / rs;
  if (ISR) {
    const double ximax = 1.0 - 4.0 * mass * mass / s, beta = sqrt(1.0 - 4.0 * mass * mass / s);
    const double K = s * sqrt(fmax(0.0, 1.0 - 4.0 * mass * mass / (s * (1.0 - xi_pt)))) / (64.0 * M_PI * M_PI * M_PI * beta);
    const double cz = q[4][3] * ig;
    h += a_s * 4.0 * (coll_density(cz) + coll_density(-cz)) / (ximax * beta * xi_pt * K);
  } else {
#pragma unroll
    for (int j = 2; j <= 3; ++j) {
      const double kn = sqrt(q[j][1] * q[j][1] + q[j][2] * q[j][2] + q[j][3] * q[j][3]);
      const double y = (q[4][1] * q[j][1] + q[4][2] * q[j][2] + q[4][3] * q[j][3]) * ig / kn;
      const double d = 2.0 - xi_pt * (1.0 - y);
      const double K = s * (1.0 - xi_pt) / (16.0 * M_PI * M_PI * M_PI * d * d);
      h += a_s * 4.0 * coll_density(y) / (xi_pt * K);
    }
  }
#pragma unroll
  for (int comp = 0; comp < 4; ++comp)
#pragma unroll
    for (int l = 0; l < 5; ++l) p[(comp * 5 + l) * n + i] = q[l][comp];
  if (wgt) wgt[i] = 1.0 / h;
}

// ---------------------------------------------------------------- unweighting
// Hit-or-miss unweighting of signed weights: point i is kept iff u_i w_max < |w_i|, with
// u_i the first uniform of Philox4x32-10 at counter (point lo, point hi, stream, 0);
// a kept point carries sign(w_i) max(w_max, |w_i|), so that the expected event weight
// is w_i.  The kept indices are written in increasing order: per-block counts, one
// exclusive scan, then a scatter that recomputes the same decisions.
constexpr int UW_THREADS = 256;

struct UwArgs {
  const double* w;
  long n;
  double wmax;                         // used when wmax_bits is null
  const unsigned long long* wmax_bits; // device: bit pattern of the batch maximum of |w|
  uint64_t seed;
  uint32_t stream;
  long long first;
};

__device__ __forceinline__ double uw_uniform(const UwArgs& a, long i) {
  const unsigned long long idx = (unsigned long long)(a.first + i);
  uint32_t c[4] = {(uint32_t)(idx & 0xFFFFFFFFull), (uint32_t)(idx >> 32), a.stream, 0u};
  philox4x32_10(c, (uint32_t)(a.seed & 0xFFFFFFFFull), (uint32_t)(a.seed >> 32));
  return u01(c[0], c[1]);
}
__device__ __forceinline__ double uw_wmax(const UwArgs& a) {
  return a.wmax_bits ? __longlong_as_double((long long)*a.wmax_bits) : a.wmax;
}

// maximum of |w| (NaN skipped): the bit patterns of non-negative doubles order like the
// numbers, so an integer maximum gives it, in any order of the blocks
__global__ void k_uw_absmax(const double* __restrict__ w, long n, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long sm[UW_THREADS / 32];
  unsigned long long m = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double x = fabs(w[i]);
    if (x == x) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(x);
      m = b > m ? b : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < UW_THREADS / 32 ? sm[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
      m = y > m ? y : m;
    }
    if (threadIdx.x == 0) atomicMax(out, m);
  }
}

__global__ void __launch_bounds__(UW_THREADS) k_uw_count(UwArgs a, int* __restrict__ counts,
                                                          unsigned long long* __restrict__ n_over) {
  const long i = (long)blockIdx.x * UW_THREADS + threadIdx.x;
  const double wmax = uw_wmax(a);
  bool keep = false, over = false;
  if (i < a.n) {
    const double aw = fabs(a.w[i]);
    keep = uw_uniform(a, i) * wmax < aw;
    over = aw > wmax;
  }
  const int c = __syncthreads_count(keep);
  const int o = __syncthreads_count(over);
  if (threadIdx.x == 0) {
    counts[blockIdx.x] = c;
    if (o) atomicAdd(n_over, (unsigned long long)o);
  }
}

// exclusive scan of the per-block counts (one block of 1024 threads), total to *total
__global__ void __launch_bounds__(1024) k_uw_scan(int* __restrict__ counts, long nb, unsigned long long* __restrict__ total) {
  __shared__ int warp_sum[32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long base = 0; base < nb; base += 1024) {
    const long i = base + threadIdx.x;
    const int v = i < nb ? counts[i] : 0;
    int x = v;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int s = warp_sum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sum[lane] = s;  // inclusive over the warps
    }
    __syncthreads();
    const int before = warp ? warp_sum[warp - 1] : 0;
    if (i < nb) counts[i] = (int)(carry + before + x - v);
    const int chunk = warp_sum[31];
    __syncthreads();
    if (threadIdx.x == 0) carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = (unsigned long long)carry;
}

__global__ void __launch_bounds__(UW_THREADS) k_uw_scatter(UwArgs a, const int* __restrict__ offsets,
                                                            int* __restrict__ kept, double* __restrict__ kept_w) {
  __shared__ int warp_cnt[UW_THREADS / 32];
  const long i = (long)blockIdx.x * UW_THREADS + threadIdx.x;
  const double wmax = uw_wmax(a);
  bool keep = false;
  double wi = 0.0;
  if (i < a.n) {
    wi = a.w[i];
    keep = uw_uniform(a, i) * wmax < fabs(wi);
  }
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[warp] = __popc(bal);
  __syncthreads();
  if (keep) {
    int pos = offsets[blockIdx.x] + __popc(bal & ((1u << lane) - 1u));
    for (int k = 0; k < warp; ++k) pos += warp_cnt[k];
    kept[pos] = (int)i;
    if (kept_w) kept_w[pos] = fabs(wi) > wmax ? wi : copysign(wmax, wi);
  }
}

bool on_device(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int me_generate_flat(me_handle* h, uint64_t seed, uint32_t stream, int64_t first_point, double sqrt_s,
                                int64_t n, double* momenta, double* ps_weights) {
  if (!h) return me_internal_fail(ME_ERR_ARG, "me_generate_flat: NULL handle");
  if (n < 0 || n > (int64_t)INT32_MAX || first_point < 0 || !(sqrt_s > 0.0))
    return me_internal_fail(ME_ERR_ARG, "me_generate_flat: bad n, first_point or sqrt_s");
  if (n == 0) return ME_OK;
  if (!momenta || !on_device(momenta) || (ps_weights && !on_device(ps_weights)))
    return me_internal_fail(ME_ERR_ARG, "me_generate_flat: momenta and ps_weights must be device memory");
  double masses[4];
  int nout = 0;
  cudaStream_t st = nullptr;
  const int rc = me_internal_final_masses(h, masses, &nout, &st);
  if (rc != ME_OK) return rc;
  double msum = 0.0;
  for (int j = 0; j < nout; ++j) msum += masses[j];
  if (!(msum < sqrt_s)) return me_internal_fail(ME_ERR_ARG, "me_generate_flat: sqrt_s below the final-state masses");
  // constant massless weight (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)
  const double s = sqrt_s * sqrt_s;
  double fact = 1.0;
  for (int j = 2; j <= nout - 1; ++j) fact *= j;
  double fact2 = 1.0;
  for (int j = 2; j <= nout - 2; ++j) fact2 *= j;
  const double w0 = std::pow(2.0 * M_PI, 4 - 3 * nout) * std::pow(0.5 * M_PI, nout - 1) * std::pow(s, nout - 2) /
                    (fact * fact2);
  Masses ms{};
  for (int j = 0; j < nout; ++j) ms.m[j] = masses[j];
  const int threads = 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  switch (nout) {
    case 2: k_rambo<2><<<blocks, threads, 0, st>>>(seed, stream, first_point, sqrt_s, ms, w0, n, momenta, ps_weights); break;
    case 3: k_rambo<3><<<blocks, threads, 0, st>>>(seed, stream, first_point, sqrt_s, ms, w0, n, momenta, ps_weights); break;
    case 4: k_rambo<4><<<blocks, threads, 0, st>>>(seed, stream, first_point, sqrt_s, ms, w0, n, momenta, ps_weights); break;
    default: return me_internal_fail(ME_ERR_PROCESS, "me_generate_flat: unsupported multiplicity");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return me_internal_fail(ME_ERR_CUDA, (std::string("me_generate_flat: ") + cudaGetErrorString(e)).c_str());
  return ME_OK;
}

extern "C" int me_generate_fks(me_handle* h, uint64_t seed, uint32_t stream, int64_t first_point, double sqrt_s,
                               int64_t n, double* momenta, double* ps_weights) {
  if (!h) return me_internal_fail(ME_ERR_ARG, "me_generate_fks: NULL handle");
  const int pid = me_internal_handle_process(h);
  const bool isr = pid == me_internal_process_id("gg_ttg") || pid == me_internal_process_id("uu_ttg");
  if (!isr && pid != me_internal_process_id("ee_uug"))
    return me_internal_fail(ME_ERR_PROCESS, "me_generate_fks: process has no FKS sectors");
  if (n < 0 || n > (int64_t)INT32_MAX || first_point < 0 || !(sqrt_s > 0.0))
    return me_internal_fail(ME_ERR_ARG, "me_generate_fks: bad n, first_point or sqrt_s");
  if (n == 0) return ME_OK;
  if (!momenta || !on_device(momenta) || (ps_weights && !on_device(ps_weights)))
    return me_internal_fail(ME_ERR_ARG, "me_generate_fks: momenta and ps_weights must be device memory");
  double masses[4];
  int nout = 0;
  cudaStream_t st = nullptr;
  const int rc = me_internal_final_masses(h, masses, &nout, &st);
  if (rc != ME_OK) return rc;
  const double mass = masses[0];
  if (!(2.0 * mass < sqrt_s)) return me_internal_fail(ME_ERR_ARG, "me_generate_fks: sqrt_s below the final-state masses");
  const int threads = 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  // massless three-body volume (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!) = s / (256 pi^3)
  const double w3 = sqrt_s * sqrt_s / (256.0 * M_PI * M_PI * M_PI);
  if (isr)
    k_fks_points<true><<<blocks, threads, 0, st>>>(seed, stream, first_point, sqrt_s, mass, w3, n, momenta, ps_weights);
  else
    k_fks_points<false><<<blocks, threads, 0, st>>>(seed, stream, first_point, sqrt_s, mass, w3, n, momenta, ps_weights);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return me_internal_fail(ME_ERR_CUDA, (std::string("me_generate_fks: ") + cudaGetErrorString(e)).c_str());
  return ME_OK;
}

extern "C" int me_unweight(me_handle* h, const double* weights, int64_t n, double w_max, uint64_t seed, uint32_t stream,
                           int64_t first_point, int32_t* kept, double* kept_weights, int64_t* n_kept, double* w_max_used,
                           int64_t* n_over) {
  if (!h || !n_kept) return me_internal_fail(ME_ERR_ARG, "me_unweight: NULL handle or n_kept");
  if (n < 0 || n > (int64_t)INT32_MAX || first_point < 0 || !(w_max == w_max))
    return me_internal_fail(ME_ERR_ARG, "me_unweight: bad n, first_point or w_max");
  *n_kept = 0;
  if (n_over) *n_over = 0;
  if (w_max_used) *w_max_used = w_max > 0.0 ? w_max : 0.0;
  if (n == 0) return ME_OK;
  if (!weights || !kept || !on_device(weights) || !on_device(kept) || (kept_weights && !on_device(kept_weights)))
    return me_internal_fail(ME_ERR_ARG, "me_unweight: weights, kept and kept_weights must be device memory");
  double masses[4];
  int nout = 0;
  cudaStream_t st = nullptr;
  const int rc = me_internal_final_masses(h, masses, &nout, &st);  // the handle's device and stream
  if (rc != ME_OK) return rc;
  const long nb = (long)((n + UW_THREADS - 1) / UW_THREADS);
  int* d_counts = nullptr;
  unsigned long long* d_u64 = nullptr;  // [0] max |w| bits, [1] overweight count, [2] kept count
  auto cuda_fail = [&](cudaError_t e) {
    cudaFreeAsync(d_counts, st);
    cudaFreeAsync(d_u64, st);
    return me_internal_fail(ME_ERR_CUDA, (std::string("me_unweight: ") + cudaGetErrorString(e)).c_str());
  };
  cudaError_t e = cudaMallocAsync(&d_counts, nb * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_u64, 3 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_u64, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e);
  UwArgs a{weights, (long)n, w_max, nullptr, seed, stream, (long long)first_point};
  if (!(w_max > 0.0)) {
    const unsigned g = (unsigned)(nb < 4096 ? nb : 4096);
    k_uw_absmax<<<g, UW_THREADS, 0, st>>>(weights, (long)n, d_u64);
    a.wmax_bits = d_u64;
  }
  k_uw_count<<<(unsigned)nb, UW_THREADS, 0, st>>>(a, d_counts, d_u64 + 1);
  k_uw_scan<<<1, 1024, 0, st>>>(d_counts, nb, d_u64 + 2);
  k_uw_scatter<<<(unsigned)nb, UW_THREADS, 0, st>>>(a, d_counts, kept, kept_weights);
  e = cudaGetLastError();
  unsigned long long host[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, d_u64, sizeof host, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaFreeAsync(d_counts, st);
  if (e == cudaSuccess) {
    d_counts = nullptr;
    e = cudaFreeAsync(d_u64, st);
  }
  if (e == cudaSuccess) {
    d_u64 = nullptr;
    e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  *n_kept = (int64_t)host[2];
  if (n_over) *n_over = (int64_t)host[1];
  if (w_max_used) {
    double wm = w_max;
    if (!(w_max > 0.0)) std::memcpy(&wm, &host[0], sizeof wm);
    *w_max_used = wm;
  }
  return ME_OK;
}
