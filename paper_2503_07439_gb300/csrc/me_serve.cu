// Request loop: continuous batching of phase-space batches from many integration
// channels (multi-event interface of Sec. 4.4, kept on the device between requests as
// argued in Sec. 4.3).  Each of the n_slots slots owns a host thread, a CUDA stream,
// pinned staging buffers and one handle per process.  A slot thread takes the oldest
// queued request whenever the device-memory budget allows, stages it (host copy into
// pinned memory, then asynchronous copies), launches it on its stream and waits for it
// on the host, so staging, launches and completions of different requests proceed in
// parallel and their kernels overlap on the GPU.  Completion is detected by polling a
// CUDA event (never a device-side wait).
// After one ordinary request of a (process, kind, weights) key, a slot captures that
// key's launch sequence -- main kernel, float64 rescue, reduction, with the batch size
// read on the device -- in a CUDA graph once, and replays it for every later request of
// the key (momenta copied with the slot's fixed stride).
// With persistent = 1 the e+e-, g g and u ubar families instead run on one persistent
// kernel each (me_persist.cuh): a family thread stages each request in pinned host
// memory, publishes a work descriptor to the family's ring, launches the kernel when none
// is running, and retires requests as their completion records appear.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_persist.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
  uint64_t ticket;
  int pid;
  std::string process;
  int kind;
  const double* p;
  const double* w;
  int64_t n;
  double* out;
  int n_ext;
  size_t bytes;
  clk::time_point t_submit, t_admit;
  me_result res;
  bool done = false;
};

// captured launch sequence of one (process, kind, weights) key on one slot
struct Prog {
  cudaGraphExec_t exec = nullptr;
  bool warmed = false;  // an ordinary request of the key ran (lane layouts chosen)
  bool tried = false;   // capture attempted at the current capacity
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double *d_p = nullptr, *d_w = nullptr, *d_out = nullptr;
  double *h_p = nullptr, *h_w = nullptr, *h_out = nullptr;
  int* h_resc = nullptr;
  int* d_n = nullptr;  // batch size read by the graph's kernels
  int* h_n = nullptr;
  size_t cap = 0;   // points
  int cap_ext = 6;  // legs the buffers are sized for
  me_handle* handles[16] = {};
  std::map<int, Prog> progs;
  Req* cur = nullptr;
};

// One persistent process family: its ring, control words, staging and kernel state.
struct Family {
  int id = -1;
  int pid_born = -1, pid_real = -1;
  cudaStream_t st = nullptr;
  cudaEvent_t kdone = nullptr;
  me::PDesc* descs = nullptr;  // pinned, mapped (host view)
  me::PDone* dones = nullptr;
  me::PCtl* ctl = nullptr;
  me::PDesc* d_descs = nullptr;  // device views of the same
  me::PDone* d_dones = nullptr;
  me::PCtl* d_ctl = nullptr;
  me::PDev* dev = nullptr;  // device memory
  me::KParams kpB{}, kpR{};
  double* h_buf[me::P_RING] = {};  // staging per ring slot: momenta, weights, output
  double* d_buf[me::P_RING] = {};
  size_t cap[me::P_RING] = {};     // doubles
  Req* inflight[me::P_RING] = {};
  clk::time_point t_pub[me::P_RING];
  unsigned next = 0, oldest = 0, kpos0 = 0;
  bool running = false;
  std::deque<Req*> queue;
  std::thread worker;
  std::atomic<int64_t> launches{0}, timeouts{0}, served{0};
};

int family_of(int pid) {
  if (pid == me::P_EE_UU || pid == me::P_EE_UUG) return 0;
  if (pid == me::P_GG_TT || pid == me::P_GG_TTG) return 1;
  if (pid == me::P_UU_TT || pid == me::P_UU_TTG) return 2;
  return -1;
}

void drop_graphs(Slot& s) {
  for (auto& kv : s.progs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    kv.second.exec = nullptr;
    kv.second.tried = false;
  }
}

}  // namespace

struct me_server {
  me_server_params prm;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<Slot> slots;
  std::vector<std::thread> workers;  // one per slot
  Family fam[3];                     // persistent families (persistent = 1)
  bool stop = false;
  int64_t mem_in_use = 0;
  uint64_t next_ticket = 1;
  std::atomic<int64_t> graph_runs{0}, plain_runs{0};
  // slot threads hold this shared while they call into CUDA and exclusively while they
  // capture a graph, so that no allocation, free or synchronisation of another slot
  // runs concurrently with a stream capture
  std::shared_mutex cuda_mu;
};

static int sfail(int code, const std::string& m) { return me_internal_fail(code, m.c_str()); }

static int slot_reserve(Slot& s, int64_t n, int n_ext) {
  if ((size_t)n <= s.cap && n_ext <= s.cap_ext) return ME_OK;
  size_t c = std::max<size_t>((size_t)n, 4096);
  drop_graphs(s);  // captured with the old buffers and stride
  cudaFree(s.d_p);
  cudaFree(s.d_w);
  cudaFree(s.d_out);
  cudaFreeHost(s.h_p);
  cudaFreeHost(s.h_w);
  cudaFreeHost(s.h_out);
  s.d_p = s.d_w = s.d_out = s.h_p = s.h_w = s.h_out = nullptr;
  s.cap = 0;
  const size_t pb = c * 4 * (size_t)s.cap_ext * sizeof(double);
  if (cudaMalloc(&s.d_p, pb) != cudaSuccess || cudaMalloc(&s.d_w, c * 8) != cudaSuccess ||
      cudaMalloc(&s.d_out, c * 8) != cudaSuccess || cudaMallocHost(&s.h_p, pb) != cudaSuccess ||
      cudaMallocHost(&s.h_w, c * 8) != cudaSuccess || cudaMallocHost(&s.h_out, c * 8) != cudaSuccess)
    return ME_ERR_OOM;
  s.cap = c;
  return ME_OK;
}

// Capture the launch sequence of the request's key once (slot thread, with the server's
// CUDA lock held exclusively).  A failed capture leaves the ordinary launches.
static void capture(me_server* sv, Slot& s, Req* r) {
  me_handle* h = s.handles[r->pid];
  Prog& pg = s.progs[r->pid * 8 + r->kind * 2 + (r->w ? 1 : 0)];
  if (!h || !sv->prm.use_graphs || !pg.warmed || pg.tried || pg.exec) return;
  pg.tried = true;
  cudaStreamSynchronize(s.st);
  if (me_internal_prepare_counted(h, r->kind, (int64_t)s.cap) == ME_OK) {
    cudaGraph_t g = nullptr;
    cudaGetLastError();
    if (cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int lrc = me_internal_launch_counted(h, r->kind, s.d_p, r->w ? s.d_w : nullptr, (int64_t)s.cap, s.d_n,
                                                 s.d_out);
      const cudaError_t e = cudaStreamEndCapture(s.st, &g);
      if (lrc == ME_OK && e == cudaSuccess && g && cudaGraphInstantiate(&pg.exec, g, 0) != cudaSuccess)
        pg.exec = nullptr;
      if (g) cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();
}

static bool wants_capture(me_server* sv, Slot& s, Req* r) {
  if (!sv->prm.use_graphs || !s.handles[r->pid] || (size_t)r->n > s.cap || r->n_ext > s.cap_ext) return false;
  auto it = s.progs.find(r->pid * 8 + r->kind * 2 + (r->w ? 1 : 0));
  return it != s.progs.end() && it->second.warmed && !it->second.tried && !it->second.exec;
}

// stage and launch one admitted request on its slot (slot thread, without the lock)
static int start(me_server* sv, Slot& s, Req* r) {
  cudaSetDevice(sv->prm.device);
  (void)cudaGetLastError();  // each call below is checked on its own
  int rc = slot_reserve(s, r->n, r->n_ext);
  if (rc != ME_OK) return rc;
  me_handle*& h = s.handles[r->pid];
  if (!h) {
    me_params p = sv->prm.params;
    p.device = sv->prm.device;
    if ((rc = me_init(r->process.c_str(), &p, &h)) != ME_OK) return rc;
    if ((rc = me_set_stream(h, s.st)) != ME_OK) return rc;
  }
  const size_t pb = (size_t)r->n * 4 * r->n_ext * sizeof(double);
  std::memcpy(s.h_p, r->p, pb);
  if (r->w) std::memcpy(s.h_w, r->w, (size_t)r->n * 8);
  Prog& pg = s.progs[r->pid * 8 + r->kind * 2 + (r->w ? 1 : 0)];
  if (cudaEventRecord(s.e0, s.st) != cudaSuccess) return sfail(ME_ERR_CUDA, "event record failed");
  if (pg.exec) {
    // momenta rows (4 x n_ext rows of n points) at the slot's stride, then the count
    cudaError_t e = cudaMemcpy2DAsync(s.d_p, s.cap * sizeof(double), s.h_p, (size_t)r->n * sizeof(double),
                                      (size_t)r->n * sizeof(double), (size_t)4 * r->n_ext, cudaMemcpyHostToDevice, s.st);
    if (e == cudaSuccess && r->w) e = cudaMemcpyAsync(s.d_w, s.h_w, (size_t)r->n * 8, cudaMemcpyHostToDevice, s.st);
    *s.h_n = (int)r->n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_n, s.h_n, sizeof(int), cudaMemcpyHostToDevice, s.st);
    if (e == cudaSuccess) e = cudaGraphLaunch(pg.exec, s.st);
    if (e == cudaSuccess) {
      sv->graph_runs.fetch_add(1);
    } else {  // retire the graph; this request and later ones take the ordinary launches
      std::fprintf(stderr, "me_server: graph replay failed (%s); ordinary launches from now on\n", cudaGetErrorString(e));
      cudaGetLastError();
      cudaGraphExecDestroy(pg.exec);
      pg.exec = nullptr;
    }
  }
  if (!pg.exec) {
    cudaError_t e = cudaMemcpyAsync(s.d_p, s.h_p, pb, cudaMemcpyHostToDevice, s.st);
    if (e == cudaSuccess && r->w) e = cudaMemcpyAsync(s.d_w, s.h_w, (size_t)r->n * 8, cudaMemcpyHostToDevice, s.st);
    if (e != cudaSuccess) return sfail(ME_ERR_CUDA, std::string("staging: ") + cudaGetErrorString(e));
    const double* dw = r->w ? s.d_w : nullptr;
    if (r->kind == ME_KIND_BORN) rc = me_eval_born(h, s.d_p, dw, r->n, s.d_out);
    else if (r->kind == ME_KIND_REAL_SUBTRACTED) rc = me_eval_real_subtracted(h, s.d_p, dw, r->n, s.d_out);
    else rc = me_eval_nbody_nlo(h, s.d_p, dw, r->n, s.d_out);
    if (rc != ME_OK) return rc;
    pg.warmed = true;
    sv->plain_runs.fetch_add(1);
  }
  if ((rc = me_internal_rescued_async(h, s.h_resc)) != ME_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(s.h_out, s.d_out, (size_t)r->n * 8, cudaMemcpyDeviceToHost, s.st);
  if (e == cudaSuccess) e = cudaEventRecord(s.e1, s.st);
  if (e != cudaSuccess) return sfail(ME_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  return ME_OK;
}

static void finish(Req* r, Slot& s, int status) {
  r->res.status = status;
  r->res.n = r->n;
  double a = 0, b = 0;
  if (status == ME_OK) {
    std::memcpy(r->out, s.h_out, (size_t)r->n * 8);
    for (int64_t i = 0; i < r->n; ++i) {
      a += r->out[i];
      b += r->out[i] * r->out[i];
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, s.e0, s.e1);
    r->res.t_device_us = 1e3 * ms;
    r->res.n_rescued = *s.h_resc;
  }
  r->res.sum_w = a;
  r->res.sum_w2 = b;
  auto now = clk::now();
  r->res.t_queue_us = std::chrono::duration<double, std::micro>(r->t_admit - r->t_submit).count();
  r->res.t_total_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
}

// Host-side wait for a slot's completion event: a short spin for small requests, then
// sleeps growing to 200 us.  Every kernel of the path runs to completion on its own
// (no device-side waits), so the event always completes or reports an error.
static cudaError_t wait_event(cudaEvent_t e) {
  const auto t0 = clk::now();
  int sleep_us = 0;
  for (;;) {
    const cudaError_t q = cudaEventQuery(e);
    if (q != cudaErrorNotReady) return q;
    if (std::chrono::duration<double, std::micro>(clk::now() - t0).count() < 100.0) {
      std::this_thread::yield();
      continue;
    }
    sleep_us = std::min(200, std::max(10, 2 * sleep_us));
    std::this_thread::sleep_for(std::chrono::microseconds(sleep_us));
  }
}

// One slot: admit the oldest request when the memory budget allows (first in, first
// out: a request that does not fit blocks the ones behind it), run it, retire it.
static void slot_loop(me_server* sv, int si) {
  Slot& s = sv->slots[si];
  cudaSetDevice(sv->prm.device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    Req* r = nullptr;
    if (!sv->pending.empty()) {
      Req* head = sv->pending.front();
      if (sv->mem_in_use + (int64_t)head->bytes <= sv->prm.mem_budget_bytes || sv->mem_in_use == 0) {
        r = head;
        sv->pending.pop_front();
        sv->mem_in_use += (int64_t)r->bytes;
        r->t_admit = clk::now();
      }
    }
    if (!r) {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    lk.unlock();
    s.cur = r;
    if (wants_capture(sv, s, r)) {
      std::unique_lock<std::shared_mutex> cx(sv->cuda_mu);
      capture(sv, s, r);
    }
    int rc;
    {
      std::shared_lock<std::shared_mutex> cs(sv->cuda_mu);
      rc = start(sv, s, r);
    }
    if (rc == ME_OK) {
      const cudaError_t e = wait_event(s.e1);
      if (e != cudaSuccess) rc = sfail(ME_ERR_CUDA, std::string("completion: ") + cudaGetErrorString(e));
    }
    if (rc != ME_OK)
      std::fprintf(stderr, "me_server: request %llu (%s, kind %d, n %lld) failed: %s\n",
                   (unsigned long long)r->ticket, r->process.c_str(), r->kind, (long long)r->n, me_last_error());
    finish(r, s, rc);
    s.cur = nullptr;
    lk.lock();
    sv->mem_in_use -= (int64_t)r->bytes;
    r->done = true;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();  // memory was released: the head may fit now
  }
}

// ---------------------------------------------------------------- persistent families
static const char* kFamBorn[3] = {"ee_uu", "gg_tt", "uu_tt"};
static const char* kFamReal[3] = {"ee_uug", "gg_ttg", "uu_ttg"};

static int family_init(me_server* sv, Family& f, int id) {
  f.id = id;
  me_params prm = sv->prm.params;
  prm.device = sv->prm.device;
  int rc = me_internal_device_kparams(kFamBorn[id], &prm, &f.kpB, &f.pid_born);
  if (rc == ME_OK) rc = me_internal_device_kparams(kFamReal[id], &prm, &f.kpR, &f.pid_real);
  if (rc != ME_OK) return rc;
  if (cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&f.kdone, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc(&f.descs, me::P_RING * sizeof(me::PDesc), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&f.dones, me::P_RING * sizeof(me::PDone), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&f.ctl, sizeof(me::PCtl), cudaHostAllocMapped) != cudaSuccess ||
      cudaMalloc(&f.dev, sizeof(me::PDev)) != cudaSuccess)
    return sfail(ME_ERR_CUDA, "me_server_create: persistent family allocation failed");
  std::memset(f.descs, 0, me::P_RING * sizeof(me::PDesc));
  std::memset(f.dones, 0, me::P_RING * sizeof(me::PDone));
  std::memset(f.ctl, 0, sizeof(me::PCtl));
  if (cudaHostGetDevicePointer((void**)&f.d_descs, f.descs, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&f.d_dones, f.dones, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&f.d_ctl, f.ctl, 0) != cudaSuccess)
    return sfail(ME_ERR_CUDA, "me_server_create: mapped pointers");
  return ME_OK;
}

static void family_free(Family& f) {
  for (int i = 0; i < me::P_RING; ++i) cudaFreeHost(f.h_buf[i]);
  cudaFreeHost(f.descs);
  cudaFreeHost(f.dones);
  cudaFreeHost(f.ctl);
  cudaFree(f.dev);
  if (f.kdone) cudaEventDestroy(f.kdone);
  if (f.st) cudaStreamDestroy(f.st);
}

// Retire request r of ring slot `slot` with `status` (family thread).
static void family_finish(me_server* sv, Family& f, int slot, int status) {
  Req* r = f.inflight[slot];
  f.inflight[slot] = nullptr;
  r->res.status = status;
  r->res.n = r->n;
  double a = 0, b = 0;
  if (status == ME_OK) {
    const double* o = f.h_buf[slot] + (size_t)r->n * (4 * r->n_ext + 1);
    std::memcpy(r->out, o, (size_t)r->n * 8);
    for (int64_t i = 0; i < r->n; ++i) {
      a += r->out[i];
      b += r->out[i] * r->out[i];
    }
    r->res.n_rescued = f.dones[slot].n_rescued;
  }
  r->res.sum_w = a;
  r->res.sum_w2 = b;
  const auto now = clk::now();
  r->res.t_queue_us = std::chrono::duration<double, std::micro>(r->t_admit - r->t_submit).count();
  r->res.t_device_us = std::chrono::duration<double, std::micro>(now - f.t_pub[slot]).count();
  r->res.t_total_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->mem_in_use -= (int64_t)r->bytes;
  r->done = true;
  ++f.served;
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

// Stage request r in ring slot `slot` and publish its descriptor (family thread).
static int family_publish(me_server* sv, Family& f, Req* r) {
  const int slot = (int)(f.next % me::P_RING);
  const size_t need = (size_t)r->n * (4 * r->n_ext + 2);  // momenta, weights, output
  if (need > f.cap[slot]) {
    std::shared_lock<std::shared_mutex> cs(sv->cuda_mu);
    cudaFreeHost(f.h_buf[slot]);
    f.h_buf[slot] = f.d_buf[slot] = nullptr;
    f.cap[slot] = 0;
    const size_t c = std::max<size_t>(need, 4096 * 28);
    if (cudaHostAlloc(&f.h_buf[slot], c * 8, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&f.d_buf[slot], f.h_buf[slot], 0) != cudaSuccess)
      return sfail(ME_ERR_OOM, "persistent staging allocation failed");
    f.cap[slot] = c;
  }
  const size_t pn = (size_t)r->n * 4 * r->n_ext;
  std::memcpy(f.h_buf[slot], r->p, pn * 8);
  if (r->w) std::memcpy(f.h_buf[slot] + pn, r->w, (size_t)r->n * 8);
  me::PDesc& d = f.descs[slot];
  d.p = f.d_buf[slot];
  d.w = r->w ? f.d_buf[slot] + pn : nullptr;
  d.out = f.d_buf[slot] + pn + r->n;
  d.n = r->n;
  d.pid = r->pid;
  d.kind = r->kind == ME_KIND_REAL_SUBTRACTED ? me::K_REAL : me::K_TREE;
  d.nlo = 1.0;
  if (r->kind == ME_KIND_NBODY_NLO) {  // the n-body NLO factor of e+e- -> u ubar
    const me_params& pp = sv->prm.params;
    const double a_s = pp.alpha_s * (4.0 / 3.0) / (2.0 * M_PI);
    d.nlo = 1.0 + a_s * (5.0 - 2.0 * M_PI * M_PI / 3.0 - (3.0 + 4.0 * std::log(pp.xi_cut)) * std::log(0.5 * pp.delta));
  }
  f.inflight[slot] = r;
  f.t_pub[slot] = clk::now();
  __atomic_store_n(&d.seq, f.next + 1, __ATOMIC_RELEASE);  // last: the descriptor is complete
  ++f.next;
  return ME_OK;
}

// Launch the family's kernel at the first unprocessed position (family thread).
static int family_launch(me_server* sv, Family& f) {
  std::shared_lock<std::shared_mutex> cs(sv->cuda_mu);
  cudaSetDevice(sv->prm.device);
  f.ctl->exit_status = 0;
  f.ctl->error = 0;
  f.ctl->stop = 0;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->prm.device);
  // one block on half of the SMs per family (255 registers x 128 threads: two blocks fit
  // an SM), so the three families and the slots' kernels are resident together
  const unsigned blocks = (unsigned)std::max(1, sms / 2);
  cudaError_t e = cudaMemsetAsync(f.dev, 0, sizeof(me::PDev), f.st);
  if (e == cudaSuccess)
    e = me::launch_serve(f.id, sv->prm.params.precision == ME_PREC_MIXED, blocks, f.d_descs, f.d_dones, f.d_ctl,
                         f.dev, f.kpB, f.kpR, f.kpos0, (unsigned long long)sv->prm.persistent_idle_us * 1000ull, f.st);
  if (e == cudaSuccess) e = cudaEventRecord(f.kdone, f.st);
  if (e != cudaSuccess) return sfail(ME_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
  f.running = true;
  ++f.launches;
  return ME_OK;
}

static void family_loop(me_server* sv, int id) {
  Family& f = sv->fam[id];
  cudaSetDevice(sv->prm.device);
  for (;;) {
    bool stopping;
    // admit the oldest queued requests while the ring has room and memory allows
    std::vector<Req*> admit;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      stopping = sv->stop;
      while (!f.queue.empty() && f.next + (unsigned)admit.size() - f.oldest < (unsigned)me::P_RING) {
        Req* head = f.queue.front();
        if (sv->mem_in_use + (int64_t)head->bytes > sv->prm.mem_budget_bytes && sv->mem_in_use != 0) break;
        f.queue.pop_front();
        sv->mem_in_use += (int64_t)head->bytes;
        head->t_admit = clk::now();
        admit.push_back(head);
      }
      if (admit.empty() && f.oldest == f.next && !f.running) {
        if (stopping) break;
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    for (Req* r : admit) {
      const int rc = family_publish(sv, f, r);
      if (rc != ME_OK) {  // not published: retire it with the error
        const int slot = (int)(f.next % me::P_RING);
        f.inflight[slot] = r;
        f.t_pub[slot] = clk::now();
        family_finish(sv, f, slot, rc);
      }
    }
    if (f.oldest != f.next && !f.running && family_launch(sv, f) != ME_OK) {
      while (f.oldest != f.next) family_finish(sv, f, (int)(f.oldest++ % me::P_RING), ME_ERR_CUDA);
    }
    if (stopping && f.running) f.ctl->stop = 1;
    // completions, in ring order
    bool progress = !admit.empty();
    while (f.oldest != f.next) {
      const int slot = (int)(f.oldest % me::P_RING);
      const unsigned seq = __atomic_load_n(&f.dones[slot].seq, __ATOMIC_ACQUIRE);
      if (seq != f.oldest + 1) break;
      family_finish(sv, f, slot, f.dones[slot].status);
      ++f.oldest;
      progress = true;
    }
    if (f.running) {
      cudaError_t q;
      {
        std::shared_lock<std::shared_mutex> cs(sv->cuda_mu);
        q = cudaEventQuery(f.kdone);
      }
      if (q != cudaErrorNotReady) {
        f.running = false;
        progress = true;
        // completions published just before the kernel ended
        while (f.oldest != f.next) {
          const int slot = (int)(f.oldest % me::P_RING);
          if (__atomic_load_n(&f.dones[slot].seq, __ATOMIC_ACQUIRE) != f.oldest + 1)
            break;
          family_finish(sv, f, slot, f.dones[slot].status);
          ++f.oldest;
        }
        if (f.ctl->exit_status == ME_ERR_TIMEOUT) ++f.timeouts;
        f.kpos0 = f.ctl->exit_pos;
        if (q != cudaSuccess || f.ctl->error || f.kpos0 != f.oldest) {
          std::fprintf(stderr, "me_server: persistent kernel of family %d ended abnormally (%s)\n", id,
                       q != cudaSuccess ? cudaGetErrorString(q) : "wait limit");
          cudaGetLastError();
          // requests it did not finish fail; the next launch starts after them
          while (f.oldest != f.next) family_finish(sv, f, (int)(f.oldest++ % me::P_RING), ME_ERR_TIMEOUT);
          f.kpos0 = f.next;
        }
      }
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(f.oldest != f.next ? 5 : 50));
  }
  // stopped: the kernel (if any) has been told to stop and has ended
  if (f.running) {
    f.ctl->stop = 1;
    cudaEventSynchronize(f.kdone);
    f.running = false;
  }
}

extern "C" {

void me_default_server_params(me_server_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->version = ME_PARAMS_VERSION;
  p->device = 0;
  p->n_slots = 4;
  p->max_queue = 4096;
  p->mem_budget_bytes = (int64_t)8 << 30;
  p->use_graphs = 1;
  p->persistent = 0;
  p->persistent_idle_us = 2000;
  me_default_params(&p->params);
  p->params.precision = ME_PREC_MIXED;
}

int me_server_create(const me_server_params* prm, me_server** out) {
  if (!prm || !out) return sfail(ME_ERR_ARG, "me_server_create: NULL argument");
  *out = nullptr;
  if (prm->version != ME_PARAMS_VERSION || prm->n_slots < 1 || prm->n_slots > 64 || prm->max_queue < 1 ||
      prm->mem_budget_bytes <= 0 || (prm->persistent && (prm->persistent_idle_us < 100 || prm->persistent_idle_us > 10000000)))
    return sfail(ME_ERR_ARG, "me_server_create: bad parameters");
  if (cudaSetDevice(prm->device) != cudaSuccess) return sfail(ME_ERR_CUDA, "me_server_create: bad device");
  me_server* sv = new me_server();
  sv->prm = *prm;
  sv->slots.resize(prm->n_slots);
  for (auto& s : sv->slots) {
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s.e0) != cudaSuccess || cudaEventCreate(&s.e1) != cudaSuccess ||
        cudaMallocHost(&s.h_resc, sizeof(int)) != cudaSuccess || cudaMallocHost(&s.h_n, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s.d_n, sizeof(int)) != cudaSuccess) {
      me_server_destroy(sv);
      return sfail(ME_ERR_CUDA, "me_server_create: stream/event allocation failed");
    }
    *s.h_resc = 0;
  }
  if (prm->persistent) {
    for (int id = 0; id < 3; ++id) {
      const int rc = family_init(sv, sv->fam[id], id);
      if (rc != ME_OK) {
        me_server_destroy(sv);
        return rc;
      }
    }
    for (int id = 0; id < 3; ++id) sv->fam[id].worker = std::thread(family_loop, sv, id);
  }
  for (int i = 0; i < prm->n_slots; ++i) sv->workers.emplace_back(slot_loop, sv, i);
  *out = sv;
  return ME_OK;
}

int me_submit(me_server* sv, const me_request* rq, me_ticket* out) {
  if (!sv || !rq || !out || !rq->process || !rq->momenta || !rq->out || rq->n < 0)
    return sfail(ME_ERR_ARG, "me_submit: bad request");
  const int pid = me_internal_process_id(rq->process);
  if (pid < 0) return sfail(ME_ERR_PROCESS, std::string("me_submit: unknown process ") + rq->process);
  if (rq->kind < ME_KIND_BORN || rq->kind > ME_KIND_NBODY_NLO) return sfail(ME_ERR_ARG, "me_submit: bad kind");
  static const int next_of[] = {4, 5, 4, 5, 6, 4, 5};
  Req* r = new Req();
  r->pid = pid;
  r->process = rq->process;
  r->kind = rq->kind;
  r->p = rq->momenta;
  r->w = rq->ps_weights;
  r->n = rq->n;
  r->out = rq->out;
  r->n_ext = next_of[pid];
  r->bytes = (size_t)rq->n * (4 * r->n_ext + 2) * sizeof(double);
  r->t_submit = clk::now();
  std::memset(&r->res, 0, sizeof(r->res));
  std::lock_guard<std::mutex> lk(sv->mu);
  if ((int64_t)r->bytes > sv->prm.mem_budget_bytes) {
    delete r;
    return sfail(ME_ERR_BUSY, "me_submit: request larger than the memory budget");
  }
  if ((int)sv->pending.size() >= sv->prm.max_queue) {
    delete r;
    return sfail(ME_ERR_BUSY, "me_submit: queue full");
  }
  r->ticket = sv->next_ticket++;
  sv->reqs[r->ticket] = r;
  // a family's kernel evaluates its Born process (Born, and the n-body NLO weight for
  // e+e- -> u ubar) and the subtracted real of its real process; anything else (gg_ttgg,
  // or a kind a process does not have, which then fails there) goes to the slots
  const int fam = sv->prm.persistent ? family_of(pid) : -1;
  const bool fam_born = fam >= 0 && pid == sv->fam[fam].pid_born &&
                        (r->kind == ME_KIND_BORN || (r->kind == ME_KIND_NBODY_NLO && pid == me::P_EE_UU));
  const bool fam_real = fam >= 0 && pid == sv->fam[fam].pid_real && r->kind == ME_KIND_REAL_SUBTRACTED;
  if (fam_born || fam_real)
    sv->fam[fam].queue.push_back(r);
  else
    sv->pending.push_back(r);
  *out = r->ticket;
  sv->cv_work.notify_all();
  return ME_OK;
}

int me_poll(me_server* sv, me_ticket t, me_result* out, int64_t timeout_us) {
  if (!sv || !out) return sfail(ME_ERR_ARG, "me_poll: NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(t);
  if (it == sv->reqs.end()) return sfail(ME_ERR_ARG, "me_poll: unknown ticket");
  Req* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_us < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
    return sfail(ME_ERR_TIMEOUT, "me_poll: not finished within the timeout");
  *out = r->res;
  sv->reqs.erase(it);
  delete r;
  return ME_OK;
}

int me_server_persistent_stats(me_server* sv, int64_t* launches, int64_t* idle_timeouts, int64_t* requests) {
  if (!sv || !launches || !idle_timeouts || !requests) return sfail(ME_ERR_ARG, "me_server_persistent_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *launches = *idle_timeouts = *requests = 0;
  for (auto& f : sv->fam) {
    *launches += f.launches.load();
    *idle_timeouts += f.timeouts.load();
    *requests += f.served.load();
  }
  return ME_OK;
}

int me_server_stats(me_server* sv, int64_t* graph_runs, int64_t* plain_runs) {
  if (!sv || !graph_runs || !plain_runs) return sfail(ME_ERR_ARG, "me_server_stats: NULL argument");
  *graph_runs = sv->graph_runs.load();
  *plain_runs = sv->plain_runs.load();
  return ME_OK;
}

void me_server_destroy(me_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers)
    if (t.joinable()) t.join();
  for (auto& f : sv->fam)
    if (f.worker.joinable()) f.worker.join();
  cudaSetDevice(sv->prm.device);
  for (auto& f : sv->fam) family_free(f);
  for (auto& s : sv->slots) {
    if (s.st) cudaStreamSynchronize(s.st);
    drop_graphs(s);
    for (auto* h : s.handles) me_destroy(h);
    cudaFree(s.d_p);
    cudaFree(s.d_w);
    cudaFree(s.d_out);
    cudaFreeHost(s.h_p);
    cudaFreeHost(s.h_w);
    cudaFreeHost(s.h_out);
    cudaFreeHost(s.h_resc);
    cudaFreeHost(s.h_n);
    cudaFree(s.d_n);
    if (s.e0) cudaEventDestroy(s.e0);
    if (s.e1) cudaEventDestroy(s.e1);
    if (s.st) cudaStreamDestroy(s.st);
  }
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}

}  // extern "C"
