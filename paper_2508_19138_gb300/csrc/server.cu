// Serving runtime: a request loop over G-system solves of different device sizes (block size,
// block count, energy grid) arriving over time.
//
// * Admission: one device arena of hbm_budget_bytes is allocated at bt_server_create; every
//   admitted request borrows its workspace from it (first-fit, 256-byte aligned, coalescing
//   free list), so admission is "the workspace fits in the arena now".  Requests are admitted
//   strictly in arrival order; one that can never fit is rejected at submit (BT_ERR_BUDGET).
// * Continuous batching: `max_active` worker threads each own a CUDA stream.  A worker takes the
//   oldest queued request as soon as it fits, runs its energies in chunks of
//   `max_energies_per_chunk` (each chunk one batched solve), returns the arena block and takes
//   the next request.  Requests that arrive while others run are admitted as slots and memory
//   free up; their kernels overlap on the device through the separate streams.
// * Results are written to the caller's buffers exactly as bt_selinv_solve would write them:
//   the same kernels, the same chunking, so a request's output does not depend on what else
//   is running.
// * Latency = completion - submission (host steady clock); p50 / p99 over completed requests.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "arena.h"
#include "bt_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct Request {
  bt_request r;
  std::vector<double> energies;
  long long ticket = 0;
  Clock::time_point t_submit, t_start, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  bt_status result = BT_OK;
  size_t bytes = 0;
  bt_selinv_desc desc{};
};

}  // namespace

struct bt_server {
  bt_server_desc d{};
  char* arena_mem = nullptr;
  size_t arena_bytes = 0;
  bt::Arena arena;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<long long, Request*> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  long long next_ticket = 1;
  size_t used = 0, peak_used = 0;
  int active = 0, peak_active = 0;
  long long submitted = 0, completed = 0, failed = 0, rejected = 0, energies_done = 0;
  std::vector<double> latencies;
  bool have_start = false;
  Clock::time_point t_first_start, t_last_done;
  Clock::time_point t0 = Clock::now();
};

namespace {

void run_request(bt_server* s, Request* q, cudaStream_t st, size_t off) {
  bt_ctx* ctx = nullptr;
  std::string err;
  bt_status rc = bt::ctx_create(&q->desc, st, s->arena.base() + off, q->bytes, &ctx, &err);
  if (rc == BT_OK) {
    const bt_request& r = q->r;
    auto opt = [](const bt_bt& b) { return b.diag ? &b : nullptr; };
    const bt_bt_out* oR = (r.outR.diag || r.outR.upper || r.outR.lower) ? &r.outR : nullptr;
    const bt_bt_out* oL = (r.outL.diag || r.outL.upper || r.outL.lower) ? &r.outL : nullptr;
    const bt_bt_out* oG = (r.outG.diag || r.outG.upper || r.outG.lower) ? &r.outG : nullptr;
    rc = bt_selinv_solve(ctx, &r.H, opt(r.S), opt(r.sigR), opt(r.sigL), opt(r.sigG), q->energies.data(),
                         r.n_energies, oR, oL, oG, r.status_device);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == BT_OK) rc = BT_ERR_CUDA;
    bt_selinv_destroy(ctx);
  }
  q->result = rc;
}

void worker_main(bt_server* s) {
  cudaSetDevice(s->d.device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  for (;;) {
    Request* q = nullptr;
    size_t off = SIZE_MAX;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) break;
        if (!s->queue.empty()) {
          off = s->arena.alloc(s->queue.front()->bytes);
          if (off != SIZE_MAX) break;
        }
        s->cv.wait(lk);
      }
      if (off == SIZE_MAX) break;
      q = s->queue.front();
      s->queue.pop_front();
      q->state = 1;
      q->t_start = Clock::now();
      if (!s->have_start) { s->have_start = true; s->t_first_start = q->t_start; }
      s->used += q->bytes;
      s->peak_used = std::max(s->peak_used, s->used);
      ++s->active;
      s->peak_active = std::max(s->peak_active, s->active);
    }
    run_request(s, q, st, off);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(off, q->bytes);
      s->used -= q->bytes;
      --s->active;
      q->t_done = Clock::now();
      s->t_last_done = q->t_done;
      if (q->result == BT_OK) {
        q->state = 2;
        ++s->completed;
        s->energies_done += q->r.n_energies;
        s->latencies.push_back(std::chrono::duration<double>(q->t_done - q->t_submit).count());
      } else {
        q->state = 3;
        ++s->failed;
      }
    }
    s->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p / 100.0 * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" bt_status bt_server_create(const bt_server_desc* desc, bt_server** out) {
  if (!desc || !out) return BT_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->max_active < 1 || desc->max_active > 64 || desc->max_energies_per_chunk < 1 ||
      desc->hbm_budget_bytes < 256 || (desc->precision != BT_FP64 && desc->precision != BT_SPLIT))
    return BT_ERR_INVALID_ARG;
  bt_server* s = new (std::nothrow) bt_server();
  if (!s) return BT_ERR_OOM;
  s->d = *desc;
  if (cudaSetDevice(desc->device) != cudaSuccess) { cudaGetLastError(); delete s; return BT_ERR_CUDA; }
  if (cudaMalloc(&s->arena_mem, desc->hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return BT_ERR_OOM;
  }
  s->arena_bytes = desc->hbm_budget_bytes;
  s->arena.reset(s->arena_mem, s->arena_bytes);
  for (int i = 0; i < desc->max_active; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return BT_OK;
}

extern "C" bt_status bt_server_submit(bt_server* s, const bt_request* r, long long* ticket) {
  if (!s || !r || !ticket) return BT_ERR_INVALID_ARG;
  if (r->nb < 1 || r->bs < 1 || r->n_energies < 1 || !r->energies_host || !r->status_device || !r->H.diag)
    return BT_ERR_INVALID_ARG;
  Request* q = new (std::nothrow) Request();
  if (!q) return BT_ERR_OOM;
  q->r = *r;
  q->energies.assign(r->energies_host, r->energies_host + r->n_energies);
  bt_selinv_desc& d = q->desc;
  d.nb = r->nb;
  d.bs = r->bs;
  d.max_energies = std::min(r->n_energies, s->d.max_energies_per_chunk);
  d.system = BT_SYS_G;
  d.precision = s->d.precision;
  d.split_slices = s->d.split_slices;
  d.symmetrize = 1;
  d.obc = r->obc;
  d.eta = r->eta;
  d.kT = r->kT;
  d.mu_left = r->mu_left;
  d.mu_right = r->mu_right;
  d.decim_tol = 1e-14;
  d.decim_maxit = 100;
  size_t bytes = 0;
  bt_status rc = bt_selinv_workspace_bytes(&d, &bytes);
  std::lock_guard<std::mutex> lk(s->mu);
  if (rc != BT_OK) { ++s->rejected; delete q; return rc; }
  if (bytes > s->arena_bytes) { ++s->rejected; delete q; return BT_ERR_BUDGET; }
  q->bytes = bytes;
  q->ticket = s->next_ticket++;
  q->t_submit = Clock::now();
  s->reqs[q->ticket] = q;
  s->queue.push_back(q);
  ++s->submitted;
  *ticket = q->ticket;
  s->cv.notify_all();
  return BT_OK;
}

extern "C" bt_status bt_server_poll(bt_server* s, long long ticket, int* state) {
  if (!s || !state) return BT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BT_ERR_INVALID_ARG;
  *state = it->second->state;
  return it->second->state == 3 ? it->second->result : BT_OK;
}

extern "C" bt_status bt_server_wait(bt_server* s, long long ticket, double timeout_s, int* state) {
  if (!s || !state) return BT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BT_ERR_INVALID_ARG;
  Request* q = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (q->state < 2) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && q->state < 2) {
      *state = q->state;
      return BT_ERR_TIMEOUT;
    }
  }
  *state = q->state;
  return q->state == 3 ? q->result : BT_OK;
}

extern "C" bt_status bt_server_get_stats(bt_server* s, bt_server_stats* out) {
  if (!s || !out) return BT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  bt_server_stats st{};
  st.submitted = s->submitted;
  st.completed = s->completed;
  st.failed = s->failed;
  st.rejected = s->rejected;
  st.energies_done = s->energies_done;
  st.queued = (long long)s->queue.size();
  st.active = s->active;
  st.p50_latency_s = percentile(s->latencies, 50.0);
  st.p99_latency_s = percentile(s->latencies, 99.0);
  double sum = 0.0;
  for (double x : s->latencies) sum += x;
  st.mean_latency_s = s->latencies.empty() ? 0.0 : sum / (double)s->latencies.size();
  st.busy_seconds = s->have_start && s->completed + s->failed > 0
                        ? std::chrono::duration<double>(s->t_last_done - s->t_first_start).count()
                        : 0.0;
  st.energies_per_s = st.busy_seconds > 0 ? (double)s->energies_done / st.busy_seconds : 0.0;
  st.peak_bytes = s->peak_used;
  st.peak_active = s->peak_active;
  *out = st;
  return BT_OK;
}

extern "C" bt_status bt_server_destroy(bt_server* s) {
  if (!s) return BT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // queued requests are cancelled; running ones finish
    for (Request* q : s->queue) {
      q->state = 3;
      q->result = BT_ERR_INVALID_ARG;
    }
    s->queue.clear();
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->reqs) delete kv.second;
  if (s->arena_mem) cudaFree(s->arena_mem);
  delete s;
  return BT_OK;
}
