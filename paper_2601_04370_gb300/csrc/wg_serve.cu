// Serving runtime of libwg.so: wg_submit / wg_poll / wg_cancel / wg_autotune.
//
// One scheduler thread per context. Whenever the GPU is free it takes a batch
// from the queue (continuous batching: FIFO, up to max_slots requests,
// admitted while the batch's device memory fits the HBM budget), traces all
// forward passes of the batch in fused persistent launches (each design on
// its own CTAs; a batch whose device work was captured before replays the
// CUDA graph), then runs the loss and adjoint of loss+gradient requests on
// the same stream, copies the outputs and completes the tickets.
//
// With max_slots > 1 loss+gradient requests go to a second lane instead: a
// thread with its own internal context (scratch, workspaces) and a stream of
// lower priority runs them FIFO (forward with the eyebox-ray list, loss,
// adjoint), while the first lane keeps fusing forward requests on a stream of
// higher priority. The two overlap on the GPU (the forward lane's CTAs are
// scheduled first whenever the adjoint's kernels leave SMs free), so a short
// forward request never waits for a long adjoint to finish. Forward-only
// requests of this mode skip the eyebox-ray list (no adjoint follows them),
// which also leaves each design's list to the gradient lane alone.
// max_slots = 1 keeps one lane: every request FIFO, one design per launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wg.h"
#include "wg_host.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

enum TicketState { QUEUED, RUNNING, DONE };

struct Ticket {
  wg_ticket id = 0;
  wg_request req;
  std::vector<float> lam, fx, fy;  // the request's configuration arrays (cfg points here)
  long long tally_n = 0, grad_n = 0;
  long long rays = 0;
  size_t dev_bytes = 0;
  TicketState state = QUEUED;
  bool cancel = false;
  wg_result result;
  std::string err;
  Clock::time_point t_submit, t_start, t_done;
};

// launch shape chosen for a class of evaluations, and what was timed for it
struct Tuned {
  int chunk = 0;  // rays per chunk (0: default)
  int bps = 0;    // CTAs per SM (0: occupancy limit)
  float ms = 0.0f;  // the chosen shape's time (0: read from the cache file)
  int n_tried = 0;
  int tried_chunk[WG_TUNE_MAX_TRIED] = {};
  int tried_bps[WG_TUNE_MAX_TRIED] = {};
  float tried_ms[WG_TUNE_MAX_TRIED] = {};
};

struct Graph {
  uint64_t sig = 0;
  cudaGraphExec_t exec = nullptr;
  std::unique_ptr<wgh::FusedBatch> fb;  // its pinned staging (the graph copies from it)
};

struct Serve {
  wg_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Ticket*> queue;
  std::unordered_map<wg_ticket, std::unique_ptr<Ticket>> all;
  wg_ticket next_id = 1;
  bool stop = false;
  std::thread th;
  cudaStream_t stream = nullptr;
  // device arena of the running batch (tallies, dL/dtally, gradients)
  void* arena = nullptr;
  size_t arena_n = 0;
  // autotuned launch shapes by class, and the captured graphs (LRU by key)
  std::mutex fused_mu;  // one fused forward at a time (context workspace, graphs)
  std::mutex tune_mu;
  std::map<uint64_t, Tuned> tune;
  std::list<std::pair<uint64_t, Graph>> graphs;
  // compositions seen once (captured when they come again), and the staging
  // reused by batches that run without a graph
  std::list<uint64_t> seen;
  std::unique_ptr<wgh::FusedBatch> direct_fb;
  // gradient lane (max_slots > 1)
  bool two_lanes = false;
  std::deque<Ticket*> gqueue;
  std::condition_variable cv_gwork;
  std::thread gth;
  wg_ctx* gctx = nullptr;
  cudaStream_t gstream = nullptr;
  void* garena = nullptr;
  size_t garena_n = 0;
};

constexpr size_t kMaxGraphs = 16;
constexpr size_t kMaxSeen = 256;

// class of an evaluation for the autotuned table
uint64_t tune_key(const wg_design* d, const wg_trace_cfg* cfg) {
  int K = 1, n_dev = 0, period = 0, acc = 0;
  wgh::design_shape(d, &K, &n_dev, &period, &acc);
  const int F = cfg->pol == WG_POL_PAIR ? 2 : 1;
  const int lbin = std::min(7, (n_dev / std::max(1, K)) / 32);
  const long long cells = (long long)cfg->n_lambda * cfg->n_fx * cfg->n_fy;
  const long long per_cell = (cfg->n_rays + cells - 1) / std::max(1ll, cells);
  const int rbin = per_cell < 512 ? 0 : per_cell < 4096 ? 1 : 2;
  return (uint64_t)acc * 10000 + (uint64_t)F * 1000 + (uint64_t)period * 100 + (uint64_t)lbin * 10 + (uint64_t)rbin;
}

void load_tune_cache(Serve& S) {
  const char* path = wgh::ctx_autotune_cache(S.ctx);
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  unsigned long long key;
  int chunk, bps;
  while (fscanf(f, "%llu %d %d", &key, &chunk, &bps) == 3) {
    Tuned t;
    t.chunk = chunk;
    t.bps = bps;
    S.tune[key] = t;
  }
  fclose(f);
}

void save_tune_cache(Serve& S) {
  const char* path = wgh::ctx_autotune_cache(S.ctx);
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  for (const auto& kv : S.tune) fprintf(f, "%llu %d %d\n", (unsigned long long)kv.first, kv.second.chunk, kv.second.bps);
  fclose(f);
}

wg_status ensure_buf(void*& p, size_t& n, size_t bytes) {
  if (bytes <= n) return WG_OK;
  if (p) cudaFree(p);
  p = nullptr;
  n = 0;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return wgh::set_error(WG_ENOMEM, "serving: device arena allocation failed");
  }
  n = bytes;
  return WG_OK;
}
wg_status ensure_arena(Serve& S, size_t bytes) { return ensure_buf(S.arena, S.arena_n, bytes); }

// Times candidate launch shapes on a bounded sample of (d, cfg) and stores
// the fastest for its class.
wg_status autotune(Serve& S, const wg_design* d, const wg_trace_cfg* cfg0, cudaStream_t stream) {
  wg_trace_cfg cfg = *cfg0;
  const long long cells = (long long)cfg.n_lambda * cfg.n_fx * cfg.n_fy;
  const long long per_cell = (cfg.n_rays + cells - 1) / std::max(1ll, cells);
  cfg.n_rays = std::min<long long>(cfg.n_rays, std::max<long long>(cells, 1ll << 19));
  cfg.ray_begin = 0;
  cfg.ray_end = 0;
  cfg.flags |= WG_TRACE_NO_EXIT_LIST;
  const long long tn = wgh::tally_doubles(d, &cfg);
  if (tn < 0) return WG_EINVAL;
  double* tally = nullptr;
  if (cudaMalloc(&tally, sizeof(double) * (size_t)tn) != cudaSuccess) {
    cudaGetLastError();
    return wgh::set_error(WG_ENOMEM, "autotune: allocation failed");
  }
  const long long sample_cell = (cfg.n_rays + cells - 1) / cells;
  Tuned best;
  double best_ms = 1e30;
  const int chunks[3] = {1024, 2048, 4096};
  wg_status st = WG_OK;
  for (int bps = 1; bps <= 2 && st == WG_OK; ++bps) {
    for (int ci = 0; ci < 3 && st == WG_OK; ++ci) {
      if (ci > 0 && chunks[ci - 1] >= std::min(per_cell, sample_cell)) break;  // same split as the previous size
      wgh::FusedJob job{};
      job.design = d;
      job.cfg = &cfg;
      job.tally = tally;
      job.chunk_rays = chunks[ci];
      double ms = 0.0;
      for (int rep = 0; rep < 2 && st == WG_OK; ++rep) {  // the first run warms up
        {
          std::lock_guard<std::mutex> lk(S.fused_mu);
          st = wgh::fused_forward(S.ctx, &job, 1, bps, stream);
        }
        if (st == WG_OK && job.status != WG_OK) st = job.status;
        ms = job.stats.kernel_ms;
      }
      if (st == WG_OK && best.n_tried < WG_TUNE_MAX_TRIED) {
        best.tried_chunk[best.n_tried] = chunks[ci];
        best.tried_bps[best.n_tried] = bps;
        best.tried_ms[best.n_tried] = (float)ms;
        ++best.n_tried;
      }
      if (st == WG_OK && ms < best_ms) {
        best_ms = ms;
        best.chunk = chunks[ci];
        best.bps = bps;
        best.ms = (float)ms;
      }
    }
  }
  cudaFree(tally);
  if (st != WG_OK) return st;
  {
    std::lock_guard<std::mutex> lk(S.tune_mu);
    S.tune[tune_key(d, cfg0)] = best;
    save_tune_cache(S);
  }
  return WG_OK;
}

Tuned lookup_tune(Serve& S, const wg_design* d, const wg_trace_cfg* cfg, bool* found) {
  std::lock_guard<std::mutex> lk(S.tune_mu);
  auto it = S.tune.find(tune_key(d, cfg));
  *found = it != S.tune.end();
  return *found ? it->second : Tuned{};
}

// Forward passes of the batch: replays the captured graph of an identical
// batch, else runs (and captures) the fused launches.
wg_status run_forward(Serve& S, std::vector<wgh::FusedJob>& jobs, int bps, bool* replayed) {
  *replayed = false;
  std::lock_guard<std::mutex> fused_lock(S.fused_mu);
  const int n = (int)jobs.size();
  // composition key: what the graph cache is looked up by
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](const void* x, size_t m) {
    const uint8_t* b = static_cast<const uint8_t*>(x);
    for (size_t i = 0; i < m; ++i) {
      key ^= b[i];
      key *= 1099511628211ull;
    }
  };
  mix(&bps, sizeof(bps));
  for (const auto& j : jobs) {
    mix(&j.design, sizeof(j.design));
    mix(&j.tally, sizeof(j.tally));
    mix(&j.chunk_rays, sizeof(j.chunk_rays));
    mix(&j.cfg->n_lambda, 4 * sizeof(int32_t));
    mix(&j.cfg->n_rays, sizeof(j.cfg->n_rays));
    mix(&j.cfg->eb_nx, 3 * sizeof(int32_t));
    mix(&j.cfg->ray_begin, 2 * sizeof(int64_t));
  }
  Graph* g = nullptr;
  for (auto it = S.graphs.begin(); it != S.graphs.end(); ++it)
    if (it->first == key) {
      S.graphs.splice(S.graphs.begin(), S.graphs, it);  // most recently used first
      g = &S.graphs.front().second;
      break;
    }
  if (g) {
    wg_status st = wgh::fused_prepare(S.ctx, jobs.data(), n, bps, *g->fb);
    if (st != WG_OK) return st;
    if (wgh::fused_signature(S.ctx, jobs.data(), *g->fb) == g->sig) {
      if (cudaGraphLaunch(g->exec, S.stream) != cudaSuccess || cudaStreamSynchronize(S.stream) != cudaSuccess) {
        cudaGetLastError();
        return wgh::set_error(WG_EDEVICE, "serving: graph replay failed");
      }
      *replayed = true;
      return wgh::fused_finish(S.ctx, jobs.data(), *g->fb);
    }
    // something the graph baked in changed: drop it and capture anew
    cudaGraphExecDestroy(g->exec);
    S.graphs.pop_front();
    g = nullptr;
  } else {
    // a composition met for the first time runs directly on the reused
    // staging; capturing pays off only for one that comes back
    bool again = false;
    for (auto it = S.seen.begin(); it != S.seen.end(); ++it)
      if (*it == key) {
        again = true;
        S.seen.erase(it);
        break;
      }
    if (!again) {
      S.seen.push_front(key);
      while (S.seen.size() > kMaxSeen) S.seen.pop_back();
      if (!S.direct_fb) S.direct_fb = std::make_unique<wgh::FusedBatch>();
      wg_status st = wgh::fused_prepare(S.ctx, jobs.data(), n, bps, *S.direct_fb);
      if (st != WG_OK) return st;
      st = wgh::fused_enqueue(S.ctx, jobs.data(), *S.direct_fb, S.stream);
      if (st != WG_OK) return st;
      if (cudaStreamSynchronize(S.stream) != cudaSuccess) {
        cudaGetLastError();
        return wgh::set_error(WG_EDEVICE, "serving: forward batch failed");
      }
      return wgh::fused_finish(S.ctx, jobs.data(), *S.direct_fb);
    }
  }
  auto fb = std::make_unique<wgh::FusedBatch>();
  wg_status st = wgh::fused_prepare(S.ctx, jobs.data(), n, bps, *fb);
  if (st != WG_OK) return st;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool captured = false;
  if (cudaStreamBeginCapture(S.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    st = wgh::fused_enqueue(S.ctx, jobs.data(), *fb, S.stream);
    const cudaError_t e = cudaStreamEndCapture(S.stream, &graph);
    if (st == WG_OK && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) captured = true;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
  }
  if (captured) {
    if (cudaGraphLaunch(exec, S.stream) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(exec);
      return wgh::set_error(WG_EDEVICE, "serving: graph launch failed");
    }
  } else {
    st = wgh::fused_enqueue(S.ctx, jobs.data(), *fb, S.stream);  // not capturable here: run it directly
    if (st != WG_OK) return st;
  }
  if (cudaStreamSynchronize(S.stream) != cudaSuccess) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    return wgh::set_error(WG_EDEVICE, "serving: forward batch failed");
  }
  st = wgh::fused_finish(S.ctx, jobs.data(), *fb);
  if (captured) {
    Graph ng;
    ng.sig = wgh::fused_signature(S.ctx, jobs.data(), *fb);
    ng.exec = exec;
    ng.fb = std::move(fb);
    S.graphs.emplace_front(key, std::move(ng));
    while (S.graphs.size() > kMaxGraphs) {
      cudaGraphExecDestroy(S.graphs.back().second.exec);
      S.graphs.pop_back();
    }
  }
  return st;
}

void run_batch(Serve& S, std::vector<Ticket*>& batch) {
  wg_ctx* c = S.ctx;
  const int n = (int)batch.size();
  // device buffers: per request its tally, and for loss+gradient requests
  // dL/dtally and the gradient
  std::vector<size_t> o_tally(n), o_G(n), o_grad(n);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  for (int i = 0; i < n; ++i) {
    Ticket& t = *batch[i];
    o_tally[i] = take(sizeof(double) * (size_t)t.tally_n);
    if (t.req.kind == WG_REQ_LOSS_GRAD) {
      o_G[i] = take(sizeof(double) * (size_t)t.tally_n);
      o_grad[i] = take(sizeof(double) * (size_t)std::max(1ll, t.grad_n));
    }
  }
  wg_status st = ensure_arena(S, off);
  auto fail_all = [&](wg_status e, const char* msg) {
    for (Ticket* t : batch) {
      t->result.status = e;
      t->err = msg;
    }
  };
  if (st != WG_OK) return fail_all(st, "serving: device arena allocation failed");
  uint8_t* A = static_cast<uint8_t*>(S.arena);
  // launch shapes: autotune classes seen for the first time, then group the
  // batch by CTAs per SM (one fused forward per group)
  std::vector<Tuned> shape(n);
  for (int i = 0; i < n; ++i) {
    Ticket& t = *batch[i];
    bool found = false;
    shape[i] = lookup_tune(S, t.req.design, &t.req.cfg, &found);
    if (!found) {
      if (autotune(S, t.req.design, &t.req.cfg, S.stream) == WG_OK)
        shape[i] = lookup_tune(S, t.req.design, &t.req.cfg, &found);
    }
  }
  const auto t_fwd = Clock::now();
  for (int bps = 0; bps <= 2; ++bps) {
    std::vector<wgh::FusedJob> jobs;
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
      if (shape[i].bps != bps) continue;
      wgh::FusedJob j{};
      j.design = batch[i]->req.design;
      j.cfg = &batch[i]->req.cfg;
      j.tally = reinterpret_cast<double*>(A + o_tally[i]);
      j.chunk_rays = shape[i].chunk;
      jobs.push_back(j);
      idx.push_back(i);
    }
    if (jobs.empty()) continue;
    bool replayed = false;
    st = run_forward(S, jobs, bps, &replayed);
    for (size_t q = 0; q < jobs.size(); ++q) {
      Ticket& t = *batch[idx[q]];
      t.result.stats = jobs[q].stats;
      t.result.graph_replayed = replayed ? 1 : 0;
      t.result.status = st != WG_OK ? st : jobs[q].status;
      if (st != WG_OK) {
        t.err = wg_last_error();
      } else if (jobs[q].status != WG_OK) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "serving: device error word 0x%x (1 blob staging, 2 idle wait, 4 ray mapping, 8 record bounds, "
                 "16 iteration cap) on %d CTAs for %lld chunks",
                 jobs[q].error_word, jobs[q].n_cta, jobs[q].n_chunks);
        t.err = buf;
      }
    }
  }
  (void)t_fwd;
  // loss and adjoint of loss+gradient requests, then the outputs
  for (int i = 0; i < n; ++i) {
    Ticket& t = *batch[i];
    if (t.result.status != WG_OK || t.cancel) continue;
    double* tally = reinterpret_cast<double*>(A + o_tally[i]);
    wg_trace_cfg cfg = t.req.cfg;
    cfg.stream = S.stream;
    if (t.req.kind == WG_REQ_LOSS_GRAD) {
      double* G = reinterpret_cast<double*>(A + o_G[i]);
      double* grad = reinterpret_cast<double*>(A + o_grad[i]);
      double loss[4] = {0, 0, 0, 0};
      wg_status e = wg_loss(c, t.req.design, &cfg, t.req.loss_kind, t.req.w_f, t.req.w_e, tally, loss, G);
      if (e == WG_OK) e = wg_trace_backward(c, t.req.design, &cfg, G, grad, nullptr, nullptr);
      if (e == WG_OK && t.req.grad_thickness)
        e = cudaMemcpyAsync(t.req.grad_thickness, grad, sizeof(double) * (size_t)t.grad_n, cudaMemcpyDefault,
                            S.stream) == cudaSuccess
                ? WG_OK
                : WG_EDEVICE;
      if (e == WG_OK && t.req.loss) memcpy(t.req.loss, loss, sizeof(loss));
      if (e != WG_OK) {
        t.result.status = e;
        t.err = wg_last_error();
      }
    }
    if (t.result.status == WG_OK && t.req.tally &&
        cudaMemcpyAsync(t.req.tally, tally, sizeof(double) * (size_t)t.tally_n, cudaMemcpyDefault, S.stream) !=
            cudaSuccess) {
      cudaGetLastError();
      t.result.status = WG_EDEVICE;
      t.err = "serving: tally copy failed";
    }
  }
  if (cudaStreamSynchronize(S.stream) != cudaSuccess) {
    cudaGetLastError();
    fail_all(WG_EDEVICE, "serving: batch failed on the device");
  }
}

// One loss+gradient request on the gradient lane: forward (with the
// eyebox-ray list), loss, adjoint, outputs; all on the lane's own context.
void run_grad(Serve& S, Ticket& t) {
  const size_t a_tally = ((sizeof(double) * (size_t)t.tally_n) + 255) & ~(size_t)255;
  const size_t a_grad = ((sizeof(double) * (size_t)std::max(1ll, t.grad_n)) + 255) & ~(size_t)255;
  wg_status e = ensure_buf(S.garena, S.garena_n, 2 * a_tally + a_grad);
  if (e != WG_OK) {
    t.result.status = e;
    t.err = "serving: device arena allocation failed";
    return;
  }
  uint8_t* A = static_cast<uint8_t*>(S.garena);
  double* tally = reinterpret_cast<double*>(A);
  double* G = reinterpret_cast<double*>(A + a_tally);
  double* grad = reinterpret_cast<double*>(A + 2 * a_tally);
  wg_trace_cfg cfg = t.req.cfg;
  cfg.stream = S.gstream;
  wg_stats st;
  memset(&st, 0, sizeof(st));
  double loss[4] = {0, 0, 0, 0};
  e = wg_trace_forward(S.gctx, t.req.design, &cfg, tally, &st);
  t.result.stats = st;
  if (e == WG_OK && !t.cancel) e = wg_loss(S.gctx, t.req.design, &cfg, t.req.loss_kind, t.req.w_f, t.req.w_e, tally, loss, G);
  if (e == WG_OK && !t.cancel) e = wg_trace_backward(S.gctx, t.req.design, &cfg, G, grad, nullptr, nullptr);
  if (e == WG_OK && t.req.grad_thickness &&
      cudaMemcpyAsync(t.req.grad_thickness, grad, sizeof(double) * (size_t)t.grad_n, cudaMemcpyDefault, S.gstream) !=
          cudaSuccess) {
    cudaGetLastError();
    e = WG_EDEVICE;
  }
  if (e == WG_OK && t.req.tally &&
      cudaMemcpyAsync(t.req.tally, tally, sizeof(double) * (size_t)t.tally_n, cudaMemcpyDefault, S.gstream) !=
          cudaSuccess) {
    cudaGetLastError();
    e = WG_EDEVICE;
  }
  if (cudaStreamSynchronize(S.gstream) != cudaSuccess) {
    cudaGetLastError();
    if (e == WG_OK) e = WG_EDEVICE;
  }
  if (e == WG_OK && t.req.loss) memcpy(t.req.loss, loss, sizeof(loss));
  if (e != WG_OK) {
    t.result.status = e;
    t.err = wg_last_error();
  }
}

void gscheduler(Serve* Sp) {
  Serve& S = *Sp;
  cudaSetDevice(wgh::ctx_device(S.ctx));
  for (;;) {
    Ticket* t = nullptr;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      S.cv_gwork.wait(lk, [&] { return S.stop || !S.gqueue.empty(); });
      if (S.stop) break;
      t = S.gqueue.front();
      S.gqueue.pop_front();
      t->state = RUNNING;
      t->t_start = Clock::now();
      t->result.status = WG_OK;
      t->result.batch_size = 1;
    }
    run_grad(S, *t);
    {
      std::lock_guard<std::mutex> lk(S.mu);
      t->t_done = Clock::now();
      if (t->cancel) t->result.status = WG_ECANCELED;
      t->state = DONE;
    }
    S.cv_done.notify_all();
  }
}

void scheduler(Serve* Sp) {
  Serve& S = *Sp;
  cudaSetDevice(wgh::ctx_device(S.ctx));
  for (;;) {
    std::vector<Ticket*> batch;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      S.cv_work.wait(lk, [&] { return S.stop || !S.queue.empty(); });
      if (S.stop) break;
      size_t budget = wgh::ctx_hbm_budget(S.ctx);
      if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
        budget = (size_t)(0.8 * (double)fr) + S.arena_n;  // the arena is reused by this batch
      }
      const size_t max_slots = (size_t)std::max(1, wgh::ctx_max_slots(S.ctx));
      size_t bytes = 0;
      long long rays = 0;
      const auto now = Clock::now();
      while (!S.queue.empty() && batch.size() < max_slots) {
        Ticket* t = S.queue.front();
        if (t->cancel) {  // dropped while queued
          S.queue.pop_front();
          t->state = DONE;
          t->result.status = WG_ECANCELED;
          t->t_start = t->t_done = now;
          continue;
        }
        if (!batch.empty() && (bytes + t->dev_bytes > budget || rays + t->rays > wgh::ctx_max_batch_rays(S.ctx)))
        break;  // next batch
        S.queue.pop_front();
        bytes += t->dev_bytes;
        rays += t->rays;
        t->state = RUNNING;
        t->t_start = now;
        batch.push_back(t);
      }
      S.cv_done.notify_all();
    }
    if (batch.empty()) continue;
    for (Ticket* t : batch) {
      t->result.status = WG_OK;
      t->result.batch_size = (int32_t)batch.size();
    }
    run_batch(S, batch);
    {
      std::lock_guard<std::mutex> lk(S.mu);
      const auto now = Clock::now();
      for (Ticket* t : batch) {
        t->t_done = now;
        if (t->cancel) t->result.status = WG_ECANCELED;
        t->state = DONE;
      }
    }
    S.cv_done.notify_all();
  }
}

// Creation of a context's runtime is serialized: two threads making their
// first wg_submit / wg_autotune at once must not start two schedulers (one of
// them would outlive the context).
std::mutex g_serve_create_mu;

Serve* serve_of(wg_ctx* c, bool create) {
  void** slot = wgh::ctx_serve_slot(c);
  std::lock_guard<std::mutex> lk(g_serve_create_mu);
  if (!*slot && create) {
    Serve* S = new Serve();
    S->ctx = c;
    cudaSetDevice(wgh::ctx_device(c));
    S->two_lanes = wgh::ctx_max_slots(c) > 1;
    int lo = 0, hi = 0;  // numerically lower = higher priority
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
      cudaGetLastError();
      lo = hi = 0;
    }
    if (cudaStreamCreateWithPriority(&S->stream, cudaStreamNonBlocking, S->two_lanes ? hi : lo) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return nullptr;
    }
    if (S->two_lanes) {
      wg_init_opts o;
      memset(&o, 0, sizeof(o));
      o.device = wgh::ctx_device(c);
      o.max_slots = 1;
      o.wait_limit_ns = wgh::ctx_wait_limit(c);
      if (wg_init(&S->gctx, &o) != WG_OK ||
          cudaStreamCreateWithPriority(&S->gstream, cudaStreamNonBlocking, lo) != cudaSuccess) {
        cudaGetLastError();
        if (S->gctx) wg_shutdown(S->gctx);
        cudaStreamDestroy(S->stream);
        delete S;
        return nullptr;
      }
    }
    load_tune_cache(*S);
    S->th = std::thread(scheduler, S);
    if (S->two_lanes) S->gth = std::thread(gscheduler, S);
    *slot = S;
  }
  return static_cast<Serve*>(*slot);
}

}  // namespace

namespace wgh {

void serve_shutdown(wg_ctx* c) {
  void** slot = ctx_serve_slot(c);
  Serve* S = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_serve_create_mu);
    S = static_cast<Serve*>(*slot);
    *slot = nullptr;
  }
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (Ticket* t : S->queue) {
      t->state = DONE;
      t->result.status = WG_ECANCELED;
    }
    S->queue.clear();
    for (Ticket* t : S->gqueue) {
      t->state = DONE;
      t->result.status = WG_ECANCELED;
    }
    S->gqueue.clear();
  }
  S->cv_work.notify_all();
  S->cv_gwork.notify_all();
  if (S->th.joinable()) S->th.join();
  if (S->gth.joinable()) S->gth.join();
  S->cv_done.notify_all();
  cudaSetDevice(ctx_device(c));
  if (S->stream) cudaStreamSynchronize(S->stream);
  if (S->gstream) {
    cudaStreamSynchronize(S->gstream);
    cudaStreamDestroy(S->gstream);
  }
  if (S->garena) cudaFree(S->garena);
  if (S->gctx) wg_shutdown(S->gctx);
  for (auto& g : S->graphs) cudaGraphExecDestroy(g.second.exec);
  S->graphs.clear();
  if (S->arena) cudaFree(S->arena);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // namespace wgh

extern "C" wg_status wg_submit(wg_ctx* c, const wg_request* req, wg_ticket* ticket) {
  if (!c || !req || !ticket) return wgh::set_error(WG_EINVAL, "wg_submit: NULL argument");
  if (req->kind != WG_REQ_FORWARD && req->kind != WG_REQ_LOSS_GRAD)
    return wgh::set_error(WG_EINVAL, "wg_submit: kind must be WG_REQ_FORWARD or WG_REQ_LOSS_GRAD");
  if (!req->design) return wgh::set_error(WG_EINVAL, "wg_submit: NULL design");
  if (req->kind == WG_REQ_LOSS_GRAD && req->loss_kind != 0 && req->loss_kind != 1)
    return wgh::set_error(WG_EINVAL, "wg_submit: loss_kind must be 0 (CV) or 1 (variance)");
  if (req->cfg.ray_records) return wgh::set_error(WG_EINVAL, "wg_submit: per-ray records are not served");
  if (req->cfg.lut_bins) return wgh::set_error(WG_EINVAL, "wg_submit: the coating table is not served");
  auto t = std::make_unique<Ticket>();
  t->req = *req;
  const wg_trace_cfg& src = req->cfg;
  if (src.n_lambda < 1 || src.n_fx < 1 || src.n_fy < 1 || !src.lambda_nm || !src.field_x_deg || !src.field_y_deg)
    return wgh::set_error(WG_EINVAL, "wg_submit: cfg needs its wavelength and field arrays");
  t->lam.assign(src.lambda_nm, src.lambda_nm + src.n_lambda);
  t->fx.assign(src.field_x_deg, src.field_x_deg + src.n_fx);
  t->fy.assign(src.field_y_deg, src.field_y_deg + src.n_fy);
  t->req.cfg.lambda_nm = t->lam.data();
  t->req.cfg.field_x_deg = t->fx.data();
  t->req.cfg.field_y_deg = t->fy.data();
  t->req.cfg.stream = nullptr;
  t->tally_n = wgh::tally_doubles(req->design, &t->req.cfg);
  if (t->tally_n < 0) return WG_EINVAL;  // the message is set
  t->grad_n = wgh::design_params(req->design);
  {
    const long long cells = (long long)src.n_lambda * src.n_fx * src.n_fy;
    const long long per_cell = (src.n_rays + cells - 1) / std::max(1ll, cells);
    t->rays = per_cell * cells * (req->kind == WG_REQ_LOSS_GRAD ? 3 : 1);  // a backward costs about two forwards
  }
  const bool bwd = req->kind == WG_REQ_LOSS_GRAD;
  t->dev_bytes = wgh::eval_device_bytes(req->design, &t->req.cfg, bwd);
  size_t budget = wgh::ctx_hbm_budget(c);
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaSetDevice(wgh::ctx_device(c));
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
    budget = (size_t)(0.8 * (double)tot);
  }
  if (t->dev_bytes > budget)
    return wgh::set_error(WG_ENOMEM, "wg_submit: the evaluation needs more device memory than the budget");
  memset(&t->result, 0, sizeof(t->result));
  Serve* S = serve_of(c, true);
  if (!S) return wgh::set_error(WG_EDEVICE, "wg_submit: could not start the serving runtime");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return wgh::set_error(WG_ECANCELED, "wg_submit: the context is shutting down");
    if (S->queue.size() + S->gqueue.size() >= (size_t)wgh::ctx_max_queue(c))
      return wgh::set_error(WG_EBUSY, "wg_submit: queue full");
    t->id = S->next_id++;
    t->t_submit = Clock::now();
    *ticket = t->id;
    if (S->two_lanes && bwd) {
      S->gqueue.push_back(t.get());
    } else {
      if (S->two_lanes) t->req.cfg.flags |= WG_TRACE_NO_EXIT_LIST;  // no adjoint follows
      S->queue.push_back(t.get());
    }
    S->all.emplace(t->id, std::move(t));
  }
  if (S->two_lanes && bwd) {
    S->cv_gwork.notify_one();
  } else {
    S->cv_work.notify_one();
  }
  return WG_OK;
}

extern "C" wg_status wg_poll(wg_ctx* c, wg_ticket ticket, int64_t timeout_us, wg_result* out) {
  if (!c) return wgh::set_error(WG_EINVAL, "wg_poll: NULL context");
  Serve* S = serve_of(c, false);
  if (!S) return wgh::set_error(WG_ENOTFOUND, "wg_poll: unknown ticket");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return wgh::set_error(WG_ENOTFOUND, "wg_poll: unknown ticket");
  Ticket* t = it->second.get();
  auto done = [&] { return t->state == DONE; };
  if (timeout_us < 0) {
    S->cv_done.wait(lk, done);
  } else if (timeout_us > 0) {
    S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  }
  if (!done()) return WG_ENOTREADY;
  if (out) {
    *out = t->result;
    out->queue_ms = ms_since(t->t_submit, t->t_start);
    out->run_ms = ms_since(t->t_start, t->t_done);
  }
  if (t->result.status != WG_OK && !t->err.empty()) wgh::set_error(t->result.status, t->err.c_str());
  S->all.erase(it);
  return WG_OK;
}

extern "C" wg_status wg_cancel(wg_ctx* c, wg_ticket ticket) {
  if (!c) return wgh::set_error(WG_EINVAL, "wg_cancel: NULL context");
  Serve* S = serve_of(c, false);
  if (!S) return wgh::set_error(WG_ENOTFOUND, "wg_cancel: unknown ticket");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return wgh::set_error(WG_ENOTFOUND, "wg_cancel: unknown ticket");
  Ticket* t = it->second.get();
  if (t->state == QUEUED) {
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), t), S->queue.end());
    S->gqueue.erase(std::remove(S->gqueue.begin(), S->gqueue.end(), t), S->gqueue.end());
    t->state = DONE;
    t->result.status = WG_ECANCELED;
    t->t_start = t->t_done = Clock::now();
    S->cv_done.notify_all();
  } else if (t->state == RUNNING) {
    t->cancel = true;
  }
  return WG_OK;
}

extern "C" wg_status wg_autotune(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg) {
  if (!c || !d || !cfg) return wgh::set_error(WG_EINVAL, "wg_autotune: NULL argument");
  Serve* S = serve_of(c, true);
  if (!S) return wgh::set_error(WG_EDEVICE, "wg_autotune: could not start the serving runtime");
  cudaStream_t s = nullptr;
  cudaSetDevice(wgh::ctx_device(c));
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return wgh::set_error(WG_EDEVICE, "wg_autotune: stream creation failed");
  }
  const wg_status st = autotune(*S, d, cfg, s);
  cudaStreamDestroy(s);
  return st;
}

extern "C" wg_status wg_autotune_info(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, wg_tune_info* out) {
  if (!c || !d || !cfg || !out) return wgh::set_error(WG_EINVAL, "wg_autotune_info: NULL argument");
  Serve* S = serve_of(c, true);
  if (!S) return wgh::set_error(WG_EDEVICE, "wg_autotune_info: could not start the serving runtime");
  bool found = false;
  const Tuned t = lookup_tune(*S, d, cfg, &found);
  if (!found) return wgh::set_error(WG_ENOTFOUND, "wg_autotune_info: no entry for this class");
  memset(out, 0, sizeof(*out));
  out->chunk_rays = t.chunk;
  out->ctas_per_sm = t.bps;
  out->best_ms = t.ms;
  out->n_tried = t.n_tried;
  for (int i = 0; i < t.n_tried; ++i) {
    out->tried_chunk_rays[i] = t.tried_chunk[i];
    out->tried_ctas_per_sm[i] = t.tried_bps[i];
    out->tried_ms[i] = t.tried_ms[i];
  }
  return WG_OK;
}

extern "C" wg_status wg_trace_forward_batch(wg_ctx* c, int32_t n, const wg_design* const* designs,
                                            const wg_trace_cfg* cfgs, double* const* tallies, wg_stats* stats,
                                            int32_t* graph_replayed) {
  if (!c || n < 1 || !designs || !cfgs || !tallies)
    return wgh::set_error(WG_EINVAL, "wg_trace_forward_batch: NULL argument or n < 1");
  cudaSetDevice(wgh::ctx_device(c));
  for (int i = 0; i < n; ++i) {
    if (!designs[i] || !tallies[i]) return wgh::set_error(WG_EINVAL, "wg_trace_forward_batch: NULL design or tally");
    if (cfgs[i].ray_records || cfgs[i].lut_bins)
      return wgh::set_error(WG_EINVAL, "wg_trace_forward_batch: no per-ray records or coating table in a batch");
    if (wgh::tally_doubles(designs[i], &cfgs[i]) < 0) return WG_EINVAL;  // the message is set
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, tallies[i]) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return wgh::set_error(WG_EINVAL, "wg_trace_forward_batch: tallies must be device memory");
    }
  }
  Serve* S = serve_of(c, true);
  if (!S) return wgh::set_error(WG_EDEVICE, "wg_trace_forward_batch: could not start the serving runtime");
  std::vector<wg_trace_cfg> cf(cfgs, cfgs + n);
  std::vector<Tuned> shape(n);
  for (int i = 0; i < n; ++i) {
    cf[i].stream = nullptr;
    bool found = false;
    shape[i] = lookup_tune(*S, designs[i], &cf[i], &found);
    if (!found && autotune(*S, designs[i], &cf[i], S->stream) == WG_OK)
      shape[i] = lookup_tune(*S, designs[i], &cf[i], &found);
  }
  if (graph_replayed) *graph_replayed = 1;
  wg_status result = WG_OK;
  for (int bps = 0; bps <= 2; ++bps) {
    std::vector<wgh::FusedJob> jobs;
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
      if (shape[i].bps != bps) continue;
      wgh::FusedJob j{};
      j.design = designs[i];
      j.cfg = &cf[i];
      j.tally = tallies[i];
      j.chunk_rays = shape[i].chunk;
      jobs.push_back(j);
      idx.push_back(i);
    }
    if (jobs.empty()) continue;
    bool replayed = false;
    const wg_status st = run_forward(*S, jobs, bps, &replayed);
    if (!replayed && graph_replayed) *graph_replayed = 0;
    if (st != WG_OK) return st;
    for (size_t q = 0; q < jobs.size(); ++q) {
      if (stats) stats[idx[q]] = jobs[q].stats;
      if (jobs[q].status != WG_OK && result == WG_OK) {
        result = jobs[q].status;
        char buf[160];
        snprintf(buf, sizeof(buf), "wg_trace_forward_batch: design %d: device error word 0x%x", idx[q],
                 jobs[q].error_word);
        wgh::set_error(result, buf);
      }
    }
  }
  return result;
}
