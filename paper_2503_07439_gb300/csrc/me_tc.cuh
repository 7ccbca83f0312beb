// Colour sum J^dagger C J on the tensor cores (mma.sync m16n8k16, bf16 in, f32 accumulate)
// for the 24 colour flows of g g -> t tbar g g.
//
// A warp holds the partial amplitudes of 32 helicities (one per lane): the 32 x 24
// complex block J times the real symmetric 24 x 24 colour matrix C is a dense
// contraction, Z = J C.  C is scaled to integers (54 C has entries of magnitude <= 512,
// all exactly representable in bf16); each amplitude is split into three bf16 terms
// a1 + a2 + a3 (residual ~2^-24 |a|), so the products are exact and the f32
// accumulation gives Z to float32 accuracy.  Each lane then forms
// sum_f Re(J_f)Re(Z_f) + Im(J_f)Im(Z_f) for its own helicity.
//
// Shapes: M = 32 helicities (2 m-tiles), K = 24 flows padded to 32 (2 k-steps),
// N = 24 flows (3 n-tiles); real and imaginary parts are two independent products.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "me_math.cuh"

namespace me {

constexpr int TC_NF = 24;
constexpr int TC_LDA = 40;  // bf16 row stride of the staged block (conflict-free fragment loads)
constexpr float TC_SCALE = 54.0f;
// per-warp shared memory: max(2 x 32 x 40 bf16, 2 x 32 x 24 f32) bytes
constexpr int TC_SMEM_PER_WARP = 2 * 32 * TC_NF * 4;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragments of 54 C (K x N = 32 x 24, zero-padded rows 24..31): [kstep][ntile][2]
struct TcColourB {
  uint32_t b[2][3][2];
};

__device__ __forceinline__ TcColourB tc_load_colour(const double* C) {
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  TcColourB f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 3; ++nt)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int k0 = ks * 16 + tig * 2 + r * 8, n = nt * 8 + gid;
        const float v0 = k0 < TC_NF ? rintf((float)(TC_SCALE * C[k0 * TC_NF + n])) : 0.0f;
        const float v1 = k0 + 1 < TC_NF ? rintf((float)(TC_SCALE * C[(k0 + 1) * TC_NF + n])) : 0.0f;
        f.b[ks][nt][r] = pack_bf16(v0, v1);
      }
  return f;
}

// J: this lane's 24 partial amplitudes; smem: TC_SMEM_PER_WARP bytes owned by the warp.
// Must be called by all 32 lanes of the warp together.
__device__ __forceinline__ float tc_colour_sum(const cx<float>* J, const TcColourB& cb, unsigned char* smem) {
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(smem);  // [2 re/im][32 rows][TC_LDA]
  float acc[2][2][3][4];  // [re/im][mtile][ntile][frag]
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 3; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[c][mt][nt][q] = 0.0f;
  float rem_re[TC_NF], rem_im[TC_NF];
#pragma unroll
  for (int f = 0; f < TC_NF; ++f) {
    rem_re[f] = J[f].re;
    rem_im[f] = J[f].im;
  }
#pragma unroll
  for (int split = 0; split < 3; ++split) {
    // stage this split of the lane's row (bf16 term and remainder), zero padding
    __syncwarp();
#pragma unroll
    for (int f = 0; f < TC_NF; ++f) {
      const __nv_bfloat16 hr = __float2bfloat16_rn(rem_re[f]);
      const __nv_bfloat16 hi = __float2bfloat16_rn(rem_im[f]);
      rem_re[f] -= __bfloat162float(hr);
      rem_im[f] -= __bfloat162float(hi);
      sa[(0 * 32 + lane) * TC_LDA + f] = hr;
      sa[(1 * 32 + lane) * TC_LDA + f] = hi;
    }
#pragma unroll
    for (int f = TC_NF; f < 32; ++f) {
      sa[(0 * 32 + lane) * TC_LDA + f] = __float2bfloat16_rn(0.0f);
      sa[(1 * 32 + lane) * TC_LDA + f] = __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const __nv_bfloat16* base = sa + (c * 32 + mt * 16) * TC_LDA + ks * 16 + tig * 2;
          uint32_t a[4];
          a[0] = *reinterpret_cast<const uint32_t*>(base + gid * TC_LDA);
          a[1] = *reinterpret_cast<const uint32_t*>(base + (gid + 8) * TC_LDA);
          a[2] = *reinterpret_cast<const uint32_t*>(base + gid * TC_LDA + 8);
          a[3] = *reinterpret_cast<const uint32_t*>(base + (gid + 8) * TC_LDA + 8);
#pragma unroll
          for (int nt = 0; nt < 3; ++nt) mma_bf16_16816(acc[c][mt][nt], a, cb.b[ks][nt]);
        }
  }
  // Z fragments -> shared memory [re/im][row][flow] f32, then each lane reads its row
  __syncwarp();
  float* sz = reinterpret_cast<float*>(smem);
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 3; ++nt) {
        const int r0 = mt * 16 + gid, col = nt * 8 + tig * 2;
        sz[(c * 32 + r0) * TC_NF + col] = acc[c][mt][nt][0];
        sz[(c * 32 + r0) * TC_NF + col + 1] = acc[c][mt][nt][1];
        sz[(c * 32 + r0 + 8) * TC_NF + col] = acc[c][mt][nt][2];
        sz[(c * 32 + r0 + 8) * TC_NF + col + 1] = acc[c][mt][nt][3];
      }
  __syncwarp();
  float s = 0.0f;
#pragma unroll
  for (int f = 0; f < TC_NF; ++f) s += J[f].re * sz[lane * TC_NF + f] + J[f].im * sz[(32 + lane) * TC_NF + f];
  __syncwarp();
  return s * (1.0f / TC_SCALE);
}

}  // namespace me
