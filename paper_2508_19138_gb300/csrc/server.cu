// Serving runtime: a request loop over G-system solves of different device sizes (block size,
// block count, energy grid) arriving over time.  The paper has no counterpart (its energies are
// distributed over ranks once per iteration, Sec. 4.4); each unit of work is the solve of
// bt_selinv_solve (Sec. 3, Eq. 1; Sec. 4.3.2).
//
// * Work units: a request is split into energy chunks of max_energies_per_chunk energies; each
//   chunk is one work unit, solved by its own context on a workspace lent from the arena.
// * Admission: one device arena of hbm_budget_bytes is allocated at bt_server_create; a unit is
//   started when a worker is free and its workspace fits in the arena's free memory now.  The
//   unit to start is chosen by the scheduler of unit_sched.h: round robin over the requests
//   with units left (so every admitted request progresses chunk by chunk), small units passing
//   one that does not fit, with a bound on how often the oldest waiting request can be passed.
//   A request whose unit can never fit is rejected at submit (BT_ERR_BUDGET).
// * Continuous batching: max_active worker threads each own a CUDA stream; units of different
//   requests run concurrently and their kernels overlap on the device.
// * Failure handling (host watchdog of the units): a unit whose solve reports BT_ERR_TIMEOUT (a
//   bounded device wait expired) is put back at the front of its request and started again, up to
//   max_retries times; a unit that fails otherwise fails its request.  Requests still queued when
//   the server is destroyed end with BT_ERR_CANCELLED.
// * Results are written to the caller's buffers exactly as bt_selinv_solve would write them:
//   the same kernels and the same chunks, so a request's output does not depend on what else is
//   running.  Latency = completion - submission (host steady clock); p50 / p99 over completed
//   requests.
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
#include "unit_sched.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  bt_request r;
  std::vector<double> energies;
  long long ticket = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  bt_status result = BT_OK;
  size_t bytes = 0;  // workspace of one unit
  bt_selinv_desc desc{};
  int n_units = 0, next_unit = 0, running = 0, done = 0;
  std::deque<int> redo;          // units to start again (timed out)
  std::vector<int> tries;        // per unit
  bool dead = false;             // failed or cancelled: no further units start
  long long order = 0;           // scheduler key
  int skips = 0;
  int units_left() const { return dead ? 0 : (n_units - next_unit) + (int)redo.size(); }
};

// Per-energy element extents of the operands and outputs (for the pointer offsets of a unit).
long long in_diag_extent(const bt_bt& b, int nb, int bs) {
  return b.layout == BT_LAYOUT_DIAGVEC ? (long long)nb * bs : (long long)nb * bs * bs;
}
long long out_diag_extent(const bt_bt_out& o, int nb, int bs) {
  if (o.layout == BT_LAYOUT_DIAGVEC) return (long long)nb * bs;
  if (o.layout == BT_LAYOUT_PACKED_UPPER) return (long long)nb * bs * (bs + 1) / 2;
  return (long long)nb * bs * bs;
}
const void* at(const void* p, long long elems) { return p ? static_cast<const char*>(p) + sizeof(zd) * elems : p; }
void* at(void* p, long long elems) { return p ? static_cast<char*>(p) + sizeof(zd) * elems : p; }
bt_bt offset_in(const bt_bt& b, int nb, int bs, long long e0) {
  if (!b.per_energy) return b;
  bt_bt o = b;
  const long long off = (long long)(nb > 1 ? nb - 1 : 0) * bs * bs;
  o.diag = at(b.diag, e0 * in_diag_extent(b, nb, bs));
  o.upper = at(b.upper, e0 * off);
  o.lower = at(b.lower, e0 * off);
  return o;
}
bt_bt_out offset_out(const bt_bt_out& b, int nb, int bs, long long e0) {
  bt_bt_out o = b;
  const long long off = (long long)(nb > 1 ? nb - 1 : 0) * bs * bs;
  o.diag = at(b.diag, e0 * out_diag_extent(b, nb, bs));
  o.upper = at(b.upper, e0 * off);
  o.lower = at(b.lower, e0 * off);
  return o;
}

}  // namespace

struct bt_server {
  bt_server_desc d{};
  char* arena_mem = nullptr;
  size_t arena_bytes = 0;
  bt::Arena arena;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Request*> pending;   // requests with units still to start, in arrival order
  std::map<long long, Request*> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  long long next_ticket = 1, seq = 0;
  size_t used = 0, peak_used = 0;
  int active = 0, peak_active = 0;
  long long submitted = 0, completed = 0, failed = 0, rejected = 0, energies_done = 0, units_done = 0, retries = 0;
  std::vector<double> latencies;
  bool have_start = false;
  Clock::time_point t_first_start, t_last_done;
  double busy_acc = 0.0;          // closed intervals with active > 0
  Clock::time_point busy_since;   // start of the open interval (active > 0)
};

namespace {

int max_skips_of(const bt_server* s) { return s->d.max_skips > 0 ? s->d.max_skips : 2 * s->d.max_active; }

// Solves unit u of request q on stream st with the lent workspace; returns the call's status, or
// BT_ERR_TIMEOUT when the solve completed but an energy of the unit reports a device timeout.
bt_status run_unit(Request* q, int u, cudaStream_t st, char* ws, int* h_status) {
  const bt_request& r = q->r;
  const int chunk = q->desc.max_energies;
  const long long e0 = (long long)u * chunk;
  const int n = (int)std::min<long long>(chunk, r.n_energies - e0);
  bt_ctx* ctx = nullptr;
  std::string err;
  bt_status rc = bt::ctx_create(&q->desc, st, ws, q->bytes, &ctx, &err);
  if (rc != BT_OK) return rc;
  auto opt = [&](const bt_bt& b, bt_bt& tmp) -> const bt_bt* {
    if (!b.diag) return nullptr;
    tmp = offset_in(b, r.nb, r.bs, e0);
    return &tmp;
  };
  auto out = [&](const bt_bt_out& o, bt_bt_out& tmp) -> const bt_bt_out* {
    if (!(o.diag || o.upper || o.lower)) return nullptr;
    tmp = offset_out(o, r.nb, r.bs, e0);
    return &tmp;
  };
  bt_bt H, S, sR, sL, sG;
  bt_bt_out oR, oL, oG;
  const bt_bt* Hp = opt(r.H, H);
  rc = bt_selinv_solve(ctx, Hp, opt(r.S, S), opt(r.sigR, sR), opt(r.sigL, sL), opt(r.sigG, sG),
                       q->energies.data() + e0, n, out(r.outR, oR), out(r.outL, oL), out(r.outG, oG),
                       r.status_device + e0);
  if (rc == BT_OK && cudaMemcpyAsync(h_status, r.status_device + e0, sizeof(int) * n, cudaMemcpyDeviceToHost, st) !=
                         cudaSuccess)
    rc = BT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == BT_OK) rc = BT_ERR_CUDA;
  bt_selinv_destroy(ctx);
  if (rc == BT_OK)
    for (int i = 0; i < n; ++i)
      if (h_status[i] == BT_ERR_TIMEOUT) return BT_ERR_TIMEOUT;
  return rc;
}

void finish_request(bt_server* s, Request* q, bt_status rc) {
  q->t_done = Clock::now();
  s->t_last_done = q->t_done;
  if (rc == BT_OK) {
    q->state = 2;
    ++s->completed;
    s->latencies.push_back(std::chrono::duration<double>(q->t_done - q->t_submit).count());
  } else {
    q->state = 3;
    q->result = rc;
    ++s->failed;
  }
}

void worker_main(bt_server* s) {
  cudaSetDevice(s->d.device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  std::vector<int> h_status(s->d.max_energies_per_chunk);
  for (;;) {
    Request* q = nullptr;
    int u = -1;
    size_t off = SIZE_MAX;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        // requests without units to start leave the scheduler's list
        s->pending.erase(std::remove_if(s->pending.begin(), s->pending.end(),
                                        [](Request* x) { return x->units_left() == 0; }),
                         s->pending.end());
        if (s->stop && s->pending.empty()) break;
        std::vector<bt::SchedEntry> e(s->pending.size());
        for (size_t i = 0; i < e.size(); ++i)
          e[i] = bt::SchedEntry{s->pending[i]->order, s->pending[i]->units_left(), s->pending[i]->bytes,
                                s->pending[i]->skips};
        const int i = bt::sched_pick(e, max_skips_of(s), [&](size_t b) { return s->arena.can_alloc(b); });
        for (size_t k = 0; k < e.size(); ++k) s->pending[k]->skips = e[k].skips;
        if (i >= 0) {
          q = s->pending[i];
          off = s->arena.alloc(q->bytes);
          if (!q->redo.empty()) { u = q->redo.front(); q->redo.pop_front(); }
          else u = q->next_unit++;
          q->order = ++s->seq;
          break;
        }
        s->cv.wait(lk);
      }
      if (!q) break;
      if (q->state == 0) q->state = 1;
      ++q->running;
      ++q->tries[u];
      if (!s->have_start) { s->have_start = true; s->t_first_start = Clock::now(); }
      s->used += q->bytes;
      s->peak_used = std::max(s->peak_used, s->used);
      if (s->active == 0) s->busy_since = Clock::now();
      ++s->active;
      s->peak_active = std::max(s->peak_active, s->active);
    }
    const bt_status rc = run_unit(q, u, st, s->arena.base() + off, h_status.data());
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(off, q->bytes);
      s->used -= q->bytes;
      if (--s->active == 0) s->busy_acc += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
      --q->running;
      if (rc == BT_ERR_TIMEOUT && q->tries[u] <= s->d.max_retries && !q->dead) {
        q->redo.push_front(u);  // the watchdog starts the unit again
        ++s->retries;
        if (std::find(s->pending.begin(), s->pending.end(), q) == s->pending.end()) s->pending.push_back(q);
      } else if (rc != BT_OK) {
        if (!q->dead) {
          q->dead = true;
          q->result = rc;
        }
      } else {
        ++q->done;
        ++s->units_done;
        const int chunk = q->desc.max_energies;
        s->energies_done += std::min<long long>(chunk, q->r.n_energies - (long long)u * chunk);
      }
      if (q->running == 0 && q->state < 2 && (q->dead || q->done == q->n_units))
        finish_request(s, q, q->dead ? q->result : BT_OK);
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
      desc->hbm_budget_bytes < 256 || (desc->precision != BT_FP64 && desc->precision != BT_SPLIT) ||
      (desc->split_scope != 0 && desc->split_scope != 1) || desc->max_retries < 0 ||
      (desc->graph != 0 && desc->graph != 1))
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
  d.split_scope = s->d.precision == BT_SPLIT ? s->d.split_scope : 0;
  d.symmetrize = 1;
  d.obc = r->obc;
  d.eta = r->eta;
  d.kT = r->kT;
  d.mu_left = r->mu_left;
  d.mu_right = r->mu_right;
  d.decim_tol = 1e-14;
  d.decim_maxit = 100;
  // graph mode (optional): a unit's chunk is captured and launched as one graph, its decimation
  // and Newton loops on the device; the capture serves one launch only
  d.graph = s->d.graph ? 1 : 0;
  size_t bytes = 0;
  bt_status rc = bt_selinv_workspace_bytes(&d, &bytes);
  std::lock_guard<std::mutex> lk(s->mu);
  if (rc != BT_OK) { ++s->rejected; delete q; return rc; }
  if (bytes > s->arena_bytes) { ++s->rejected; delete q; return BT_ERR_BUDGET; }
  q->bytes = bytes;
  q->n_units = (r->n_energies + d.max_energies - 1) / d.max_energies;
  q->tries.assign(q->n_units, 0);
  q->ticket = s->next_ticket++;
  q->t_submit = Clock::now();
  q->order = ++s->seq;  // behind every request already in the rotation
  s->reqs[q->ticket] = q;
  s->pending.push_back(q);
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
  long long queued = 0;
  for (Request* q : s->pending) queued += q->state == 0;
  st.queued = queued;
  st.active = s->active;
  st.p50_latency_s = percentile(s->latencies, 50.0);
  st.p99_latency_s = percentile(s->latencies, 99.0);
  double sum = 0.0;
  for (double x : s->latencies) sum += x;
  st.mean_latency_s = s->latencies.empty() ? 0.0 : sum / (double)s->latencies.size();
  st.busy_seconds = s->busy_acc + (s->active > 0 ? std::chrono::duration<double>(Clock::now() - s->busy_since).count()
                                                   : 0.0);
  st.energies_per_s = st.busy_seconds > 0 ? (double)s->energies_done / st.busy_seconds : 0.0;
  st.peak_bytes = s->peak_used;
  st.peak_active = s->peak_active;
  st.units_done = s->units_done;
  st.retries = s->retries;
  *out = st;
  return BT_OK;
}

extern "C" bt_status bt_server_destroy(bt_server* s) {
  if (!s) return BT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // requests that have not started are cancelled; running units finish, and a request with
    // units running ends when they do (cancelled unless it had no unit left to start)
    for (Request* q : s->pending) {
      if (q->units_left() == 0) continue;
      q->dead = true;
      q->result = BT_ERR_CANCELLED;
      if (q->running == 0 && q->state < 2) finish_request(s, q, BT_ERR_CANCELLED);
    }
    s->pending.clear();
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->reqs) delete kv.second;
  if (s->arena_mem) cudaFree(s->arena_mem);
  delete s;
  return BT_OK;
}
