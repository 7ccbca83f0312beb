// Persistent serving kernels: one resident kernel per process family takes the requests
// of that family from a ring of work descriptors in host memory that the GPU reads over
// the CPU-GPU link, instead of one launch sequence per request (the points stay on the
// device for as long as there is work, Sec. 4.3).
//
// Protocol (host side in me_serve.cu):
//  * the host stages a request's momenta (and weights) in pinned host buffers, fills
//    descriptor r % P_RING, and publishes it by writing seq = r + 1 last (release);
//  * block 0 (the leader) waits for descriptor r with a bounded wait (time and
//    iterations), then tells the other blocks through a word in device memory: go = r + 1,
//    or go = EXIT_BIT | r when it stops at r (idle for longer than the limit: status
//    ME_ERR_TIMEOUT; or the host asked it to stop) -- so every block stops at the same
//    request and no request is left half done;
//  * block b evaluates tiles b, b + G, ... of the request (static assignment; no claims),
//    re-evaluating its unstable points in float64 from a shared-memory queue (mixed
//    precision), then counts itself done; the last block publishes the completion record
//    (seq = r + 1, written last) and clears the request's counters for ring reuse.
// Every wait is bounded, in time and in iterations: the leader's by the idle limit, the
// others' by the idle limit plus four seconds, after which they set the error word and
// return, so the kernel always ends.
#pragma once
#include "../../include/me.h"
#include "me_kernels.cuh"

namespace me {

constexpr int P_RING = 64;
constexpr unsigned P_EXIT_BIT = 0x80000000u;

struct PDesc {          // pinned host memory, written by the host
  const double* p;      // device-visible address of the momenta [4][n_ext][n]
  const double* w;      // device-visible weights or null
  double* out;          // device-visible output [n]
  long long n;
  int pid, kind;        // kind: K_TREE or K_REAL
  double nlo;           // Born factor (n-body NLO entry), else 1
  unsigned seq;         // r + 1 once the descriptor of request r is complete
  int pad;
};
struct PDone {          // pinned host memory, written by the kernel
  unsigned seq;         // r + 1 once request r is complete
  int status;
  int n_rescued;
  int pad;
};
struct PCtl {           // pinned host memory
  int stop;             // host -> kernel: stop at the next wait for work
  int exit_status;      // kernel -> host: ME_ERR_TIMEOUT (idle) or ME_OK (stopped)
  unsigned exit_pos;    // request position the kernel stopped at
  int error;            // a follower's wait ran out (never expected)
};
struct PDev {           // device memory, cleared before every launch
  unsigned go;
  unsigned done_blocks[P_RING];
  unsigned rescued[P_RING];
};

__device__ __forceinline__ unsigned p_ld_acquire_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void p_st_release_sys(unsigned* p, unsigned v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned p_ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void p_st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long p_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// |M|^2 of one point, one lane (the Born kinds of the served families)
template <int PID, typename T>
__device__ __forceinline__ double tree_point(const double* __restrict__ p, long n, long ev, const KParams& kp) {
  constexpr int NEXT = Proc<PID>::NEXT;
  r4<double> k[NEXT];
  load_event<NEXT>(p, n, ev, k);
  const Kin<PID, T> K = prepare<PID, T>(k, kp.cp);
  T acc = T(0);
  for (int b = 0; b < n_live_blocks<PID>(); ++b)
    amplitude_block<PID, T>(K, live_block_hel<PID>(b), kp.cp, [&](int, const cx<T>* J) { acc += colour_sum<PID, T>(kp.tab, J); });
  // Algorithm 2: evaluated, then zeroed where the point fails the cuts
  return (!kp.cut.mask || pass_cuts<PID>(k, kp.cut)) ? 2.0 * (double)acc * kp.avg_inv : 0.0;
}

// Family (BPID: its Born process, RPID: its real process), precision fixed per server.
template <int BPID, int RPID, bool MIXED>
__global__ void __launch_bounds__(QT, 1) k_serve(const PDesc* __restrict__ descs, PDone* __restrict__ dones,
                                                 PCtl* __restrict__ ctl, PDev* __restrict__ dev, KParams kpB,
                                                 KParams kpR, unsigned pos0, unsigned long long idle_ns) {
  using T = typename std::conditional<MIXED, float, double>::type;
  __shared__ int q[2 * QT];
  __shared__ int qn, verdict;
  __shared__ const double* s_p;
  __shared__ const double* s_w;
  __shared__ double* s_out;
  __shared__ long long s_n;
  __shared__ int s_pid, s_kind;
  __shared__ double s_nlo;
  const unsigned self = 1u << (threadIdx.x & 31u);
  const unsigned long long follower_extra_ns = 4000000000ull;
  for (unsigned r = pos0;; ++r) {
    const int slot = (int)(r % P_RING);
    if (threadIdx.x == 0) {
      int v = 0;
      if (blockIdx.x == 0) {
        const unsigned long long t0 = p_now_ns();
        unsigned ns = 64;
        int status = ME_ERR_TIMEOUT;
        for (long it = 0; it < (1L << 24); ++it) {  // and at most ~2^24 sleeps of <= 2 us
          if (p_ld_acquire_sys(&descs[slot].seq) == r + 1) {
            v = 1;
            break;
          }
          if (*(volatile const int*)&ctl->stop) {
            status = ME_OK;
            break;
          }
          if (p_now_ns() - t0 > idle_ns) break;
          __nanosleep(ns);
          ns = ns < 2048 ? 2 * ns : ns;
        }
        if (!v) {
          ctl->exit_status = status;
          ctl->exit_pos = r;
          __threadfence_system();
        }
        p_st_release_gpu(&dev->go, v ? r + 1 : (P_EXIT_BIT | r));
      } else {
        const unsigned long long t0 = p_now_ns();
        unsigned ns = 64;
        for (long it = 0; it < (1L << 25); ++it) {
          const unsigned g = p_ld_acquire_gpu(&dev->go);
          if (g & P_EXIT_BIT) {
            v = r < (g & ~P_EXIT_BIT) ? 1 : 0;
            break;
          }
          if (g >= r + 1) {
            v = 1;
            break;
          }
          if (p_now_ns() - t0 > idle_ns + follower_extra_ns) {
            atomicExch(&ctl->error, 1);
            break;
          }
          __nanosleep(ns);
          ns = ns < 2048 ? 2 * ns : ns;
        }
        // the leader saw the descriptor complete; read it once it is visible here too
        if (v) {
          const unsigned long long t1 = p_now_ns();
          for (long it = 0; p_ld_acquire_sys(&descs[slot].seq) != r + 1; ++it) {
            if (p_now_ns() - t1 > follower_extra_ns || it > (1L << 25)) {
              atomicExch(&ctl->error, 1);
              v = 0;
              break;
            }
            __nanosleep(64);
          }
        }
      }
      if (v) {
        const PDesc* d = &descs[slot];
        s_p = *(const double* const volatile*)&d->p;
        s_w = *(const double* const volatile*)&d->w;
        s_out = *(double* const volatile*)&d->out;
        s_n = *(volatile const long long*)&d->n;
        s_pid = *(volatile const int*)&d->pid;
        s_kind = *(volatile const int*)&d->kind;
        s_nlo = *(volatile const double*)&d->nlo;
      }
      verdict = v;
      qn = 0;
    }
    __syncthreads();
    if (!verdict) return;
    const double* p = s_p;
    const double* w = s_w;
    double* out = s_out;
    const long n = (long)s_n;
    const bool real = s_kind == K_REAL;
    const long ntile = (n + QT - 1) / QT;
    int done = 0;
    for (long t = blockIdx.x;; t += gridDim.x) {
      const bool last = t >= ntile;  // uniform over the block
      if (!last) {
        const long ev = t * QT + threadIdx.x;
        if (ev < n) {
          const double wt = w ? w[ev] : 1.0;
          if (real) {
            const RealSubOut o = real_sub_event<RPID, T, 1>(p, n, ev, kpR, 0, self);
            out[ev] = wt * o.W;
            if (MIXED && unstable_point(o, kpR)) q[atomicAdd(&qn, 1)] = (int)ev;
          } else {
            out[ev] = wt * tree_point<BPID, T>(p, n, ev, kpB) * s_nlo;
          }
        }
      }
      __syncthreads();
      if (MIXED) {
        // a full queue, or the rest once this block's tiles are done
        const int qc = qn;
        if (qc >= QT || (last && qc > 0)) {
          const int take = qc < QT ? qc : QT;
          if ((int)threadIdx.x < take) {
            const int e = q[threadIdx.x];
            const RealSubOut o = real_sub_event<RPID, double, 1>(p, n, e, kpR, 0, self);
            out[e] = (w ? w[e] : 1.0) * o.W;
          }
          const int rest = qc - take;
          __syncthreads();
          if ((int)threadIdx.x < rest) q[threadIdx.x] = q[QT + threadIdx.x];
          done += take;
          __syncthreads();
          // on the pass after the block's last tile nothing was added, so fewer than QT
          // were queued and rest is 0: the queue is empty when the request is done
          if (threadIdx.x == 0) qn = rest;
        }
      }
      if (last) break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence_system();  // this block's outputs before its count
      if (done) atomicAdd(&dev->rescued[slot], (unsigned)done);
      const unsigned c = atomicAdd(&dev->done_blocks[slot], 1u) + 1u;
      if (c == gridDim.x) {
        __threadfence();
        const unsigned resc = atomicExch(&dev->rescued[slot], 0u);
        atomicExch(&dev->done_blocks[slot], 0u);  // free for request r + P_RING
        dones[slot].n_rescued = (int)resc;
        dones[slot].status = ME_OK;
        __threadfence_system();
        p_st_release_sys(&dones[slot].seq, r + 1);
      }
    }
    __syncthreads();
  }
}

// launch one family's persistent kernel (me_inst_serve.cu): family 0 e+e- (ee_uu, ee_uug),
// 1 g g (gg_tt, gg_ttg), 2 u ubar (uu_tt, uu_ttg)
cudaError_t launch_serve(int family, bool mixed, unsigned blocks, const PDesc* descs, PDone* dones, PCtl* ctl,
                         PDev* dev, const KParams& kpB, const KParams& kpR, unsigned pos0, unsigned long long idle_ns,
                         cudaStream_t st);

}  // namespace me
