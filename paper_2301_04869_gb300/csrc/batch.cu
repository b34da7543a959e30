// Multi-instance runner: many independent reduced-space IPM instances (any
// bus counts, any scenario counts) solved together on one GPU.
//
// The paper runs one two-stage problem at a time and spreads its scenarios
// over MPI ranks; on one GB300 the free parallelism is across instances.
// Host worker threads each drive one instance at a time through the
// ordinary IPM iteration on their own CUDA stream, so the instances' kernels
// overlap on the device.  The dense reduced-Hessian contraction (the FP64
// K_hat = sum_i Z_i^T Y_i, most of the flops) is not launched per instance:
// an instance that reaches it records an event and joins a rendezvous, and
// once every active instance has arrived (or a short window has passed) one
// persistent launch contracts all of their (instance, tile, scenario group)
// work items.  Converged instances leave the rendezvous, so they are masked
// out of later launches.  ipm_run_instances adds admission under a device
// memory budget: contexts are created (symbolic analysis included, on the
// worker threads) only while their estimated footprint fits, and destroyed
// as soon as their solution has been copied out.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {

struct Group;

struct Slot {
  Group *grp = nullptr;
  ipm_ctx *c = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
};

// rendezvous of the grouped contraction
struct Group {
  std::mutex m;
  std::condition_variable cv;
  int active = 0;
  std::vector<Slot *> arrived;
  long long gen = 0;
  double window_us = 2000.0;
  int dev = 0;
  cudaStream_t gst = nullptr;
  int *counter = nullptr;
  // double-buffered work-item tables (pinned host -> device)
  GemmItem *h_items[2] = {}, *d_items[2] = {};
  size_t cap[2] = {};
  cudaEvent_t used[2] = {};
  int ring = 0;
  std::vector<GemmItem> items;
  // statistics
  long long launches = 0, n_items = 0, n_inst = 0;
  int max_active = 0;
  cudaError_t err = cudaSuccess;

  bool init(int device, double window) {
    dev = device;
    window_us = window;
    if (cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaMalloc(&counter, sizeof(int)) != cudaSuccess) return false;
    for (auto &e : used)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
  }
  void release() {
    if (gst) cudaStreamSynchronize(gst);
    for (int k = 0; k < 2; ++k) {
      if (h_items[k]) cudaFreeHost(h_items[k]);
      if (d_items[k]) cudaFree(d_items[k]);
      if (used[k]) cudaEventDestroy(used[k]);
    }
    if (counter) cudaFree(counter);
    if (gst) cudaStreamDestroy(gst);
  }

  void join() {
    std::lock_guard<std::mutex> lk(m);
    ++active;
    max_active = std::max(max_active, active);
  }
  void leave() {
    std::lock_guard<std::mutex> lk(m);
    --active;
    if (!arrived.empty() && (int)arrived.size() >= active) launch_locked();
    cv.notify_all();
  }

  // One persistent launch over the work items of every arrived instance.
  // Called with m held.
  void launch_locked() {
    items.clear();
    for (Slot *s : arrived) {
      const ipm_ctx *c = s->c;
      const long long krows = (long long)c->S.N * c->S.nx;
      const int nt1 = c->nt1;
      int t = 0;
      for (int i = 0; i < nt1; ++i)
        for (int j = i; j < nt1; ++j, ++t)
          for (int g = 0; g < c->ngroups; ++g) {
            GemmItem it{};
            it.A = c->Z;
            it.B = c->Y;
            it.P = c->partial + ((size_t)g * c->ntiles + t) * 4096;
            it.r0 = (long long)g * c->kchunk;
            it.r1 = std::min(krows, it.r0 + c->kchunk);
            it.nu = c->S.nu;
            it.i0 = i * 64;
            it.j0 = j * 64;
            items.push_back(it);
          }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const GemmItem &a, const GemmItem &b) { return a.r1 - a.r0 > b.r1 - b.r0; });
    const int k = ring;
    ring ^= 1;
    cudaSetDevice(dev);
    cudaEventSynchronize(used[k]);  // the table's previous launch has consumed it
    if (items.size() > cap[k]) {
      if (h_items[k]) cudaFreeHost(h_items[k]);
      if (d_items[k]) cudaFree(d_items[k]);
      h_items[k] = d_items[k] = nullptr;
      cap[k] = items.size() * 2;
      cudaError_t e1 = cudaMallocHost(&h_items[k], cap[k] * sizeof(GemmItem));
      cudaError_t e2 = cudaMalloc(&d_items[k], cap[k] * sizeof(GemmItem));
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        err = e1 != cudaSuccess ? e1 : e2;
        cap[k] = 0;
      }
    }
    if (cap[k] >= items.size() && !items.empty()) {
      std::memcpy(h_items[k], items.data(), items.size() * sizeof(GemmItem));
      cudaMemcpyAsync(d_items[k], h_items[k], items.size() * sizeof(GemmItem), cudaMemcpyHostToDevice, gst);
      for (Slot *s : arrived) cudaStreamWaitEvent(gst, s->ready, 0);
      launch_gemm_grouped(d_items[k], (int)items.size(), counter, gst);
      cudaEventRecord(used[k], gst);
      ++launches;
      n_items += (long long)items.size();
      n_inst += (long long)arrived.size();
    } else {
      // no table (allocation failed): each instance contracts on its own stream
      for (Slot *s : arrived) {
        const ipm_ctx *c = s->c;
        cudaStreamWaitEvent(gst, s->ready, 0);
        launch_gemm_tn64((long long)c->S.N * c->S.nx, c->kchunk, c->S.nu, c->ngroups, c->Z, c->Y, c->tiles,
                         c->ntiles, c->partial, gst);
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) err = e;
    for (Slot *s : arrived) cudaEventRecord(s->done, gst);
    arrived.clear();
    ++gen;
    cv.notify_all();
  }
};

// ipm_ctx::gemm_hook: runs on the instance's own thread inside its condensation
void group_hook(void *arg, ipm_ctx *c, cudaStream_t st) {
  Slot *s = static_cast<Slot *>(arg);
  Group *G = s->grp;
  (void)c;
  cudaEventRecord(s->ready, st);
  {
    std::unique_lock<std::mutex> lk(G->m);
    const long long my = G->gen;
    G->arrived.push_back(s);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((long long)std::max(0.0, G->window_us));
    while (G->gen == my) {
      if ((int)G->arrived.size() >= G->active || std::chrono::steady_clock::now() >= deadline) {
        G->launch_locked();
        break;
      }
      G->cv.wait_until(lk, deadline);
    }
  }
  cudaStreamWaitEvent(st, s->done, 0);
}

void fill_stats(const Group &G, double wall_ms, double *stats) {
  if (!stats) return;
  stats[0] = (double)G.launches;
  stats[1] = (double)G.n_items;
  stats[2] = G.launches ? (double)G.n_inst / (double)G.launches : 0.0;
  stats[3] = (double)G.max_active;
  stats[4] = wall_ms;
  for (int k = 5; k < IPM_BATCH_N_STATS; ++k) stats[k] = 0.0;
}

int n_workers(const ipm_batch_options &o, int n) {
  int t = o.n_threads > 0 ? o.n_threads : 8;
  return std::max(1, std::min(t, n));
}

// distinct generator buses (gen_bus entries are required to be distinct)
void dims_of(const ipm_network &net, long long &nx, long long &nu) {
  const long long n = net.n_bus, ng = net.n_gen;
  nx = (n - 1) + (n - ng);
  nu = ng + (ng - 1);
}

}  // namespace

extern "C" {

ipm_status ipm_batch_default_options(ipm_batch_options *o) {
  if (!o) return IPM_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->n_threads = 8;
  o->group_contraction = 1;
  o->window_us = 2000.0;
  return IPM_OK;
}

ipm_status ipm_solve_batch(ipm_ctx **ctxs, int n, void **streams, const ipm_batch_options *bopt, int *iters,
                           double *kkt_err, int *status, double *stats) {
  if (!ctxs || n < 0 || !iters || !kkt_err || !status) return IPM_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return IPM_ERR_ARG;
  ipm_batch_options bo;
  if (bopt) bo = *bopt;
  else ipm_batch_default_options(&bo);
  if (!(bo.window_us >= 0)) return IPM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IPM_ERR_CUDA;
  Group G;
  if (!G.init(dev, bo.window_us)) {
    G.release();
    return IPM_ERR_CUDA;
  }
  const int T = n_workers(bo, n);
  std::vector<cudaStream_t> own(T, nullptr);
  for (int t = 0; t < T && !streams; ++t)
    if (cudaStreamCreateWithFlags(&own[t], cudaStreamNonBlocking) != cudaSuccess) {
      for (auto s : own)
        if (s) cudaStreamDestroy(s);
      G.release();
      return IPM_ERR_CUDA;
    }
  std::vector<Slot> slots(n);
  bool ev_ok = true;
  for (int i = 0; i < n; ++i) {
    slots[i].grp = &G;
    slots[i].c = ctxs[i];
    ev_ok = ev_ok && cudaEventCreateWithFlags(&slots[i].ready, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&slots[i].done, cudaEventDisableTiming) == cudaSuccess;
  }
  // largest instances first (longest-processing-time order)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const auto &A = ctxs[a]->S, &B = ctxs[b]->S;
    return (double)A.N * A.nx * A.nu * A.nu > (double)B.N * B.nx * B.nu * B.nu;
  });
  std::atomic<int> next(0);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
      const int i = order[q];
      ipm_ctx *c = ctxs[i];
      cudaStream_t st = streams ? (cudaStream_t)streams[i] : own[w];
      if (bo.group_contraction && ev_ok) {
        c->gemm_hook = group_hook;
        c->gemm_hook_arg = &slots[i];
        G.join();
      }
      int it = 0;
      double e = 0.0;
      status[i] = ipm_solve(c, &it, &e, st);
      iters[i] = it;
      kkt_err[i] = e;
      if (c->gemm_hook) {
        c->gemm_hook = nullptr;
        c->gemm_hook_arg = nullptr;
        G.leave();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker, t);
  for (auto &th : pool) th.join();
  cudaStreamSynchronize(G.gst);
  const double wall =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  fill_stats(G, wall, stats);
  for (auto &s : slots) {
    if (s.ready) cudaEventDestroy(s.ready);
    if (s.done) cudaEventDestroy(s.done);
  }
  for (auto s : own)
    if (s) cudaStreamDestroy(s);
  const cudaError_t gerr = G.err;
  G.release();
  if (gerr != cudaSuccess) return IPM_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (status[i] != IPM_OK) return (ipm_status)status[i];
  return IPM_OK;
}

ipm_status ipm_run_instances(const ipm_network *nets, int n, const int *n_scen, const double *const *pd,
                             const double *const *qd, const ipm_options *opt, const ipm_batch_options *bopt,
                             long long mem_budget, double *const *states_out, int *iters, double *kkt_err,
                             int *status, double *stats) {
  if (!nets || n < 0 || !n_scen || !pd || !qd || !iters || !kkt_err || !status || mem_budget <= 0)
    return IPM_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (n_scen[i] < 1 || !pd[i] || !qd[i] || nets[i].n_bus < 2 || nets[i].n_gen < 1) return IPM_ERR_ARG;
  ipm_batch_options bo;
  if (bopt) bo = *bopt;
  else ipm_batch_default_options(&bo);
  if (!(bo.window_us >= 0)) return IPM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IPM_ERR_CUDA;
  // footprint estimate: Z and Y (or the mixed operands, no larger), the
  // per-scenario K_uu blocks, and a margin for vectors, LU values and tiles
  std::vector<long long> est(n);
  for (int i = 0; i < n; ++i) {
    long long nx, nu;
    dims_of(nets[i], nx, nu);
    const long long N = n_scen[i];
    est[i] = 16 * N * nx * nu + 8 * N * nu * nu + 8 * 96 * N * nx + (64LL << 20);
  }
  Group G;
  if (!G.init(dev, bo.window_us)) {
    G.release();
    return IPM_ERR_CUDA;
  }
  const int T = n_workers(bo, n);
  std::vector<cudaStream_t> own(T, nullptr);
  for (int t = 0; t < T; ++t)
    if (cudaStreamCreateWithFlags(&own[t], cudaStreamNonBlocking) != cudaSuccess) {
      for (auto s : own)
        if (s) cudaStreamDestroy(s);
      G.release();
      return IPM_ERR_CUDA;
    }
  std::vector<Slot> slots(T);
  for (int t = 0; t < T; ++t) {
    slots[t].grp = &G;
    cudaEventCreateWithFlags(&slots[t].ready, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&slots[t].done, cudaEventDisableTiming);
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return est[a] > est[b]; });
  std::mutex bm;
  std::condition_variable bcv;
  long long in_use = 0;
  std::atomic<int> next(0);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
      const int i = order[q];
      iters[i] = 0;
      kkt_err[i] = 0.0;
      {
        // admission: wait until the estimate fits (an instance alone always runs)
        std::unique_lock<std::mutex> lk(bm);
        bcv.wait(lk, [&] { return in_use == 0 || in_use + est[i] <= mem_budget; });
        in_use += est[i];
      }
      ipm_ctx *c = nullptr;
      ipm_status s = ipm_create(&nets[i], n_scen[i], pd[i], qd[i], opt, &c);
      if (s == IPM_OK) {
        if (bo.group_contraction) {
          slots[w].c = c;
          c->gemm_hook = group_hook;
          c->gemm_hook_arg = &slots[w];
          G.join();
        }
        int it = 0;
        double e = 0.0;
        s = ipm_solve(c, &it, &e, own[w]);
        iters[i] = it;
        kkt_err[i] = e;
        if (c->gemm_hook) {
          c->gemm_hook = nullptr;
          G.leave();
        }
        if (states_out && states_out[i]) {
          const ipm_status g = ipm_get_state(c, states_out[i], 0, own[w]);
          if (s == IPM_OK) s = g;
        }
        ipm_destroy(c);
      }
      status[i] = s;
      {
        std::lock_guard<std::mutex> lk(bm);
        in_use -= est[i];
      }
      bcv.notify_all();
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker, t);
  for (auto &th : pool) th.join();
  cudaStreamSynchronize(G.gst);
  const double wall =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  fill_stats(G, wall, stats);
  for (auto &s : slots) {
    if (s.ready) cudaEventDestroy(s.ready);
    if (s.done) cudaEventDestroy(s.done);
  }
  for (auto s : own)
    if (s) cudaStreamDestroy(s);
  const cudaError_t gerr = G.err;
  G.release();
  if (gerr != cudaSuccess) return IPM_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (status[i] != IPM_OK) return (ipm_status)status[i];
  return IPM_OK;
}

}  // extern "C"
