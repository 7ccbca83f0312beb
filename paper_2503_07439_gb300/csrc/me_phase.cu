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

template <int NOUT>
__global__ void k_rambo(uint64_t seed, uint32_t stream, long long first, double rs, Masses ms, double w_massless, long n,
                        double* __restrict__ p, double* __restrict__ wgt) {
  const double* masses = ms.m;
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
  double k[NOUT][4];
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
