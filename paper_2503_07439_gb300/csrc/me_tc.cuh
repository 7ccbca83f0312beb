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


// ---------------------------------------------------------------- tcgen05 colour sum
// The same contraction on the fifth-generation tensor cores: the operands in shared
// memory, the accumulator Z in tensor memory (TMEM), one thread of a warp issuing the
// matrix instructions and an mbarrier that the tensor core arrives on when they are done.
//
// The three bf16 terms of an amplitude are laid side by side along K, and the colour
// matrix is repeated three times along K, so that one product sums the terms:
//   A[row][24 s + f] = term s of J_f (s = 0, 1, 2), A[row][72..79] = 0,
//   B[24 s + f][n]   = 54 C[f][n],                   B[72..79][n] = 0,   n < 24 (N padded to 32),
//   Z = A B = J (54 C)      (M = 128 rows, N = 32, K = 80 = five k-steps of 16).
// Real and imaginary parts are two such products into two 32-column TMEM ranges.
//
// Shared-memory operand layout (K-major, no swizzle): 8 x 16-byte core matrices, the
// eight rows of a core matrix 16 bytes apart; core matrices adjacent along K are
// TC5_LBO = 128 bytes apart, 8-row groups TC5_GROUP bytes apart.  Element (row, k) of an
// operand sits at (row / 8) * TC5_GROUP + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2.
//
// The CTA holds one 128-row A tile per part; warp w owns rows 32 w .. 32 w + 31 (lane l:
// row 32 w + l).  Each warp issues its own products over all 128 rows into its own TMEM
// columns (64 w .. 64 w + 63) and reads back only its own lane quarter, so warps never
// wait for one another: the rows of the other warps enter only accumulator lanes that
// the issuing warp ignores.  The tensor work is four times the minimum, which costs
// nothing measurable here (the colour sum is a few per cent of an event's arithmetic).
constexpr int TC5_KCH = 10;                  // 16-byte K chunks per row (80 bf16)
constexpr int TC5_LBO = 128;                 // bytes between core matrices along K
constexpr int TC5_GROUP = TC5_KCH * 128;     // bytes between 8-row groups
constexpr int TC5_A_BYTES = 16 * TC5_GROUP;  // one 128-row operand
constexpr int TC5_B_BYTES = 4 * TC5_GROUP;   // 32 rows of 54 C (24 flows + 8 zero)
constexpr int TC5_CTRL = 64;                 // 4 mbarriers (8 B each) + the TMEM address
constexpr int TC5_SMEM = 2 * TC5_A_BYTES + TC5_B_BYTES + TC5_CTRL;
constexpr uint32_t TC5_COLS = 256;           // TMEM columns per CTA (64 per warp)
constexpr int TC5_SPIN = 1 << 20;            // bound on the polls of one completion wait
// instruction descriptor of kind::f16: f32 accumulator (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC5_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (8-row group) byte
// offsets, each >> 4 in 14 bits; bits 46-48 = 0b001; base offset 0; no swizzle
__device__ __forceinline__ uint64_t tc5_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((TC5_LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((TC5_GROUP >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool tc5_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// every lane of the warp polls until all see the phase complete, at most TC5_SPIN times
__device__ __forceinline__ bool tc5_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < TC5_SPIN; ++it)
    if (__all_sync(0xffffffffu, tc5_try_wait(bar, parity))) return true;
  return false;
}

__device__ __forceinline__ void tc5_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(a), "l"(b), "r"(TC5_IDESC), "r"(accumulate)
      : "memory");
}

// 24 consecutive accumulator columns of this warp's lane quarter (one per register),
// loaded and waited for in one statement so that no use of them can move above the wait
__device__ __forceinline__ void tc5_ld24(uint32_t taddr, float* v) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%25];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
      : "r"(taddr), "r"(taddr + 16)
      : "memory");
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}

struct Tc5 {
  unsigned char* a;  // A tiles (real, imaginary), then B, then the control words
  uint32_t tmem;     // TMEM base address (lane 0, first column)
  uint32_t parity;   // phase of this warp's mbarrier to wait for next
  bool ok;           // false once a wait ran out
};

__device__ __forceinline__ uint32_t tc5_bar(const Tc5& t, int warp) {
  return smem_addr(t.a + 2 * TC5_A_BYTES + TC5_B_BYTES + 8 * warp);
}

// Called by all 128 threads of the CTA at the start: stores 54 C as B, zeroes the padding
// chunk of every A row, initialises the mbarriers and allocates the TMEM columns (warp 0).
__device__ __forceinline__ Tc5 tc5_setup(unsigned char* smem, const double* C) {
  const int tid = threadIdx.x, warp = tid >> 5;
  Tc5 t{smem, 0u, 0u, true};
  unsigned char* b = smem + 2 * TC5_A_BYTES;
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(b + TC5_B_BYTES);
  for (int c = tid; c < 32 * TC5_KCH; c += blockDim.x) {  // one 16-byte chunk (n, kc) each
    const int n = c / TC5_KCH, kc = c % TC5_KCH;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = kc * 8 + 2 * e + h;
        v[h] = (k < 3 * TC_NF && n < TC_NF) ? rintf((float)(TC_SCALE * C[(k % TC_NF) * TC_NF + n])) : 0.0f;
      }
      w[e] = pack_bf16(v[0], v[1]);
    }
    *reinterpret_cast<uint4*>(b + (n >> 3) * TC5_GROUP + kc * 128 + (n & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  {
    const int off = (tid >> 3) * TC5_GROUP + (TC5_KCH - 1) * 128 + (tid & 7) * 16;
    *reinterpret_cast<uint4*>(smem + off) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(smem + TC5_A_BYTES + off) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int w = 0; w < 4; ++w) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc5_bar(t, w)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(ctrl + 8)),
                 "r"(TC5_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  t.tmem = *reinterpret_cast<volatile uint32_t*>(ctrl + 8);
  return t;
}

// Called by all 128 threads at the end: frees the TMEM columns (warp 0).  A warp whose
// wait ran out first waits once more, with the same bound, for its products in flight.
__device__ __forceinline__ void tc5_teardown(Tc5& t) {
  const int warp = threadIdx.x >> 5;
  if (!t.ok) tc5_wait(tc5_bar(t, warp), t.parity);
  tc5_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc5_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(TC5_COLS) : "memory");
  }
}

// Step 1 of a colour sum: J, this lane's 24 partial amplitudes, becomes row 32 w + lane of
// the CTA's operand tiles, and lane 0 issues the products into the warp's TMEM columns.
// Called by all 32 lanes of a warp together; tc5_collect returns the result.  Between
// the two the warp is free to do other work (the tensor core runs meanwhile); the
// operand row may be rewritten only after the collect.
__device__ __forceinline__ void tc5_issue(const cx<float>* J, Tc5& t) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, row = threadIdx.x;
  if (!t.ok) return;
  unsigned char* const are = t.a;
  unsigned char* const aim = t.a + TC5_A_BYTES;
  const int roff = (row >> 3) * TC5_GROUP + (row & 7) * 16;
  float rr[TC_NF], ri[TC_NF];
#pragma unroll
  for (int f = 0; f < TC_NF; ++f) {
    rr[f] = J[f].re;
    ri[f] = J[f].im;
  }
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint32_t wr[4], wi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int f = 8 * c + 2 * e;
        const __nv_bfloat162 hr = __floats2bfloat162_rn(rr[f], rr[f + 1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(ri[f], ri[f + 1]);
        rr[f] -= __low2float(hr);
        rr[f + 1] -= __high2float(hr);
        ri[f] -= __low2float(hi);
        ri[f + 1] -= __high2float(hi);
        wr[e] = *reinterpret_cast<const uint32_t*>(&hr);
        wi[e] = *reinterpret_cast<const uint32_t*>(&hi);
      }
      *reinterpret_cast<uint4*>(are + roff + (3 * s + c) * 128) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
      *reinterpret_cast<uint4*>(aim + roff + (3 * s + c) * 128) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
    }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    tc5_fence_after();
    const uint32_t cols = t.tmem + (uint32_t)(64 * warp);
    const uint32_t sre = smem_addr(are), sim = smem_addr(aim), sb = smem_addr(t.a + 2 * TC5_A_BYTES);
#pragma unroll
    for (int k = 0; k < TC5_KCH / 2; ++k) tc5_mma(cols, tc5_desc(sre + 256 * k), tc5_desc(sb + 256 * k), k > 0);
#pragma unroll
    for (int k = 0; k < TC5_KCH / 2; ++k) tc5_mma(cols + 32, tc5_desc(sim + 256 * k), tc5_desc(sb + 256 * k), k > 0);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc5_bar(t, warp))
                 : "memory");
  }
  __syncwarp();
}

// Step 2: waits for the warp's products, reads this lane's row of Z = J (54 C) and returns
// J^dagger C J, with J read again from re[f], im[f] (the same values as at the issue).
// Returns NaN (and t.ok = false) if the tensor core did not signal completion in time.
__device__ __forceinline__ float tc5_collect(const float* re, const float* im, Tc5& t) {
  const int warp = threadIdx.x >> 5;
  if (!t.ok) return __int_as_float(0x7fc00000);
  if (!tc5_wait(tc5_bar(t, warp), t.parity)) {
    t.ok = false;
    return __int_as_float(0x7fc00000);
  }
  t.parity ^= 1u;
  tc5_fence_after();
  float zr[TC_NF], zi[TC_NF];
  const uint32_t taddr = t.tmem + (uint32_t)(64 * warp) + ((uint32_t)(32 * warp) << 16);
  tc5_ld24(taddr, zr);
  tc5_ld24(taddr + 32, zi);
  float sum = 0.0f;
#pragma unroll
  for (int f = 0; f < TC_NF; ++f) sum += re[f] * zr[f] + im[f] * zi[f];
  tc5_fence_before();
  __syncwarp();
  return sum * (1.0f / TC_SCALE);
}

// Both steps at once.
__device__ __forceinline__ float tc5_colour_sum(const cx<float>* J, Tc5& t) {
  tc5_issue(J, t);
  float re[TC_NF], im[TC_NF];
#pragma unroll
  for (int f = 0; f < TC_NF; ++f) {
    re[f] = J[f].re;
    im[f] = J[f].im;
  }
  return tc5_collect(re, im, t);
}

}  // namespace me
