// Serving runtime: continuous batching of independent IRK problems on one GPU.
//
// A request is one initial-value problem (its own irk_config: grid, stage
// count, viscosity) advanced nsteps steps.  The server
//  - reserves an HBM budget once (one cudaMalloc) and sub-allocates each
//    request's solver arena from it with a first-fit free list, so a request
//    is admitted exactly when its arena fits in the free part of the budget
//    (admission by free HBM) and completed requests return memory without any
//    cudaFree (which would synchronise the device);
//  - runs up to `slots` requests at once, each on its own CUDA stream driven
//    by its own worker thread, so their kernels overlap on the device; a slot
//    that finishes takes the next admissible request at once (continuous
//    batching), while new requests keep arriving through irk_server_submit;
//  - keeps each request's state, stage vectors and Krylov bases resident in
//    its arena until it completes, and records the wall time of every step
//    (p50/p99 step latency) and of every request.
// Each request's numbers are those of the same request run alone: the
// solver's reductions use fixed grids per handle, so results are bit-equal.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/irk_batch.h"
#include "../../include/irk_serve.h"
#include "irk_internal.h"
#include "pool.h"

namespace {

using irk::PoolAllocator;

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  long long id = 0;
  irk_config cfg;
  std::vector<double> u;  // initial state in, final state out (host)
  double t0 = 0, dt = 0;
  int nsteps = 0;
  size_t bytes = 0, off = 0;
  bool in_batch = false;  // served by the batched driver (else by a stream worker)
  irk_status status = IRK_OK;
  irk_stats stats;
  std::string err;
  bool done = false;
  clk::time_point t_submit, t_admit, t_done;
  std::vector<double> step_ms;
};

}  // namespace

struct irk_server {
  int slots = 0;
  char* base = nullptr;
  PoolAllocator pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<long long, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  long long next_id = 1;
  int active = 0, peak_active = 0;
  long long completed = 0, failed = 0, steps = 0;
  bool any_submit = false;
  clk::time_point first_submit, last_done;
  std::vector<double> step_ms, req_ms, queue_ms;
  int device = 0;
  // batched form: one driver thread steps every resident request together
  bool batched = false;
  int batch_capacity = 0;
  int stream_min_n = 0;  // batched form: grids of n >= this go to the stream workers
  irk_batch* batch = nullptr;
  cudaStream_t bstream = nullptr;
};

namespace {

// Completion bookkeeping of one request (caller holds no lock).
void finish_request(irk_server* s, const std::shared_ptr<Request>& r, irk_status stt) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pool.release(r->off, r->bytes);
    --s->active;
    r->status = stt;
    r->t_done = clk::now();
    r->done = true;
    s->last_done = r->t_done;
    if (stt == IRK_OK) {
      ++s->completed;
      s->steps += (long long)r->step_ms.size();
      s->step_ms.insert(s->step_ms.end(), r->step_ms.begin(), r->step_ms.end());
      s->req_ms.push_back(ms_between(r->t_submit, r->t_done));
      s->queue_ms.push_back(ms_between(r->t_submit, r->t_admit));
    } else {
      ++s->failed;
    }
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
}

void worker_loop(irk_server* s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t st = s->streams[slot];
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        // oldest pending request whose arena fits in the free budget
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
          size_t off;
          if ((*it)->in_batch) continue;
          if (s->pool.alloc((*it)->bytes, &off)) {
            r = *it;
            r->off = off;
            s->pending.erase(it);
            break;
          }
        }
        if (r) break;
        s->cv_work.wait(lk);
      }
      r->t_admit = clk::now();
      ++s->active;
      s->peak_active = std::max(s->peak_active, s->active);
    }
    irk::TraceRange tr("serve_request");  // admission to release, on this worker's thread
    irk_handle* h = nullptr;
    irk_status stt = irk_create_in(&r->cfg, r->u.data(), 0, st, s->base + r->off, r->bytes, &h);
    memset(&r->stats, 0, sizeof(r->stats));
    if (stt == IRK_OK) {
      double t = r->t0;
      r->step_ms.reserve(r->nsteps);
      for (int k = 0; k < r->nsteps && stt == IRK_OK; ++k) {
        irk_stats one;
        const auto a = clk::now();
        stt = irk_step(h, t, r->dt, 1, &one);
        r->step_ms.push_back(ms_between(a, clk::now()));
        t += r->dt;
        r->stats.steps += one.steps;
        r->stats.newton_its += one.newton_its;
        r->stats.krylov_its += one.krylov_its;
        r->stats.prec_apps += one.prec_apps;
        r->stats.vcycles += one.vcycles;
        r->stats.kernel_launches += one.kernel_launches;
        r->stats.max_newton_its = std::max(r->stats.max_newton_its, one.max_newton_its);
        r->stats.final_rel_res = one.final_rel_res;
      }
      if (stt == IRK_OK) stt = irk_get_state(h, r->u.data(), 0);
      if (stt != IRK_OK) r->err = irk_last_error(h);
      irk_destroy(h);
    } else {
      r->err = irk_last_error(nullptr);
    }
    finish_request(s, r, stt);
  }
}

// Batched form: admit waiting requests into free batch slots as their arenas
// fit the budget, advance all residents by one step in one graph launch
// (irk_batch_step), retire the finished ones; repeat.  The wall time of a
// batched step is every resident's step latency.
void batch_loop(irk_server* s) {
  cudaSetDevice(s->device);
  struct Res {
    std::shared_ptr<Request> r;
    int slot;
  };
  std::vector<Res> res;
  std::vector<irk_stats> st(s->batch_capacity);
  std::vector<irk_status> sts(s->batch_capacity);
  for (;;) {
    std::vector<std::shared_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) {
          lk.unlock();
          for (auto& x : res) irk_batch_remove(s->batch, x.slot);
          return;
        }
        for (auto it = s->pending.begin();
             it != s->pending.end() && (int)(res.size() + admitted.size()) < s->batch_capacity;) {
          size_t off;
          if (!(*it)->in_batch) {
            ++it;
            continue;
          }
          if (s->pool.alloc((*it)->bytes, &off)) {
            (*it)->off = off;
            (*it)->t_admit = clk::now();
            admitted.push_back(*it);
            it = s->pending.erase(it);
            ++s->active;
          } else {
            ++it;
          }
        }
        s->peak_active = std::max(s->peak_active, s->active);
        if (!res.empty() || !admitted.empty()) break;
        s->cv_work.wait(lk);
      }
    }
    for (auto& r : admitted) {
      memset(&r->stats, 0, sizeof(r->stats));
      if (r->nsteps == 0) {
        finish_request(s, r, IRK_OK);
        continue;
      }
      int slot = -1;
      const irk_status a = irk_batch_add(s->batch, &r->cfg, r->u.data(), 0, r->dt,
                                         s->base + r->off, r->bytes, &slot);
      if (a != IRK_OK) {
        r->err = irk_batch_last_error(s->batch);
        finish_request(s, r, a);
        continue;
      }
      r->step_ms.reserve(r->nsteps);
      res.push_back({r, slot});
    }
    if (res.empty()) continue;
    const auto t0 = clk::now();
    const irk_status e = irk_batch_step(s->batch, st.data(), sts.data());
    const double ms = ms_between(t0, clk::now());
    std::vector<Res> keep;
    for (auto& x : res) {
      Request& q = *x.r;
      irk_status stt = e;
      if (stt == IRK_OK) {
        const irk_stats& one = st[x.slot];
        q.step_ms.push_back(ms);
        q.stats.steps += one.steps;
        q.stats.newton_its += one.newton_its;
        q.stats.krylov_its += one.krylov_its;
        q.stats.prec_apps += one.prec_apps;
        q.stats.vcycles += one.vcycles;
        q.stats.max_newton_its = std::max(q.stats.max_newton_its, one.max_newton_its);
        q.stats.final_rel_res = one.final_rel_res;
        stt = sts[x.slot];
      }
      if (stt == IRK_OK && (int)q.step_ms.size() < q.nsteps) {
        keep.push_back(x);
        continue;
      }
      if (stt == IRK_OK) stt = irk_batch_get_state(s->batch, x.slot, q.u.data(), 0);
      if (stt != IRK_OK && q.err.empty()) q.err = irk_batch_last_error(s->batch);
      irk_batch_remove(s->batch, x.slot);
      finish_request(s, x.r, stt);
    }
    res.swap(keep);
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

irk_status irk_server_create(int slots, size_t budget_bytes, irk_server** out) {
  if (!out || slots < 1 || slots > 256) return IRK_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return IRK_ERR_NO_DEVICE;
  }
  irk_server* s = new (std::nothrow) irk_server();
  if (!s) return IRK_ERR_NOMEM;
  cudaGetDevice(&s->device);
  if (budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return IRK_ERR_CUDA; }
    budget_bytes = fr / 2;  // half of the free HBM by default
  }
  if (cudaMalloc((void**)&s->base, budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return IRK_ERR_NOMEM;
  }
  s->pool.init(budget_bytes);
  s->slots = slots;
  s->streams.resize(slots);
  for (int k = 0; k < slots; ++k) {
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaStreamDestroy(s->streams[j]);
      cudaFree(s->base);
      delete s;
      return IRK_ERR_CUDA;
    }
  }
  for (int k = 0; k < slots; ++k) s->workers.emplace_back(worker_loop, s, k);
  *out = s;
  return IRK_OK;
}

irk_status irk_server_create_batched(int capacity, int stream_slots, int stream_min_n,
                                    size_t budget_bytes, irk_server** out) {
  if (!out || capacity < 1 || capacity > 64 || stream_slots < 0 || stream_slots > 256 ||
      (stream_slots > 0 && stream_min_n < 1))
    return IRK_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return IRK_ERR_NO_DEVICE;
  }
  irk_server* s = new (std::nothrow) irk_server();
  if (!s) return IRK_ERR_NOMEM;
  cudaGetDevice(&s->device);
  if (budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return IRK_ERR_CUDA; }
    budget_bytes = fr / 2;
  }
  if (cudaMalloc((void**)&s->base, budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return IRK_ERR_NOMEM;
  }
  s->pool.init(budget_bytes);
  s->slots = capacity + stream_slots;
  s->batched = true;
  s->batch_capacity = capacity;
  s->stream_min_n = stream_slots > 0 ? stream_min_n : 0;
  irk_status st = IRK_OK;
  if (cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = IRK_ERR_CUDA;
  }
  s->streams.resize(stream_slots);
  for (int k = 0; k < stream_slots && st == IRK_OK; ++k)
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->streams.resize(k);
      st = IRK_ERR_CUDA;
    }
  if (st == IRK_OK) st = irk_batch_create(capacity, s->bstream, &s->batch);
  if (st != IRK_OK) {
    for (auto q : s->streams) cudaStreamDestroy(q);
    if (s->bstream) cudaStreamDestroy(s->bstream);
    cudaFree(s->base);
    delete s;
    return st;
  }
  s->workers.emplace_back(batch_loop, s);
  for (int k = 0; k < stream_slots; ++k) s->workers.emplace_back(worker_loop, s, k);
  *out = s;
  return IRK_OK;
}

irk_status irk_server_submit(irk_server* s, const irk_config* cfg, const double* u0, double t0,
                             double dt, int nsteps, long long* id) {
  if (!s || !cfg || !u0 || !id || nsteps < 0 || !(dt > 0)) return IRK_ERR_INVALID;
  // the batched form serves a request in the batch unless its grid goes to
  // the stream workers (n >= stream_min_n when there are any)
  const bool in_batch = s->batched && !(s->stream_min_n > 0 && cfg->n >= s->stream_min_n);
  const size_t bytes = in_batch ? irk_batch_instance_bytes(cfg) : irk_config_device_bytes(cfg);
  if (bytes == 0) return IRK_ERR_INVALID;
  if (bytes > s->pool.size()) return IRK_ERR_NOMEM;  // could never be admitted
  auto r = std::make_shared<Request>();
  r->cfg = *cfg;
  const bool two_d = cfg->op == IRK_OP_BURGERS_2D || cfg->op == IRK_OP_VSF_2D;
  const size_t len = two_d ? (size_t)2 * cfg->n * cfg->n : (size_t)cfg->n;
  r->u.assign(u0, u0 + len);
  r->t0 = t0;
  r->dt = dt;
  r->nsteps = nsteps;
  r->bytes = bytes;
  r->in_batch = in_batch;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    if (!s->any_submit) {
      s->any_submit = true;
      s->first_submit = r->t_submit;
    }
    s->all[r->id] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_all();
  *id = r->id;
  return IRK_OK;
}

irk_status irk_server_wait(irk_server* s, long long id, double* u_out, irk_stats* stats,
                           double* step_ms) {
  if (!s) return IRK_ERR_INVALID;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return IRK_ERR_INVALID;
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    s->all.erase(it);
  }
  if (u_out) std::copy(r->u.begin(), r->u.end(), u_out);
  if (stats) *stats = r->stats;
  if (step_ms) std::copy(r->step_ms.begin(), r->step_ms.end(), step_ms);
  return r->status;
}

irk_status irk_server_stats_get(irk_server* s, irk_server_stats* o) {
  if (!s || !o) return IRK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(o, 0, sizeof(*o));
  o->submitted = s->next_id - 1;
  o->completed = s->completed;
  o->failed = s->failed;
  o->steps = s->steps;
  o->wall_s = s->any_submit && s->completed ? ms_between(s->first_submit, s->last_done) / 1e3 : 0.0;
  o->steps_per_s = o->wall_s > 0 ? s->steps / o->wall_s : 0.0;
  o->p50_step_ms = percentile(s->step_ms, 0.50);
  o->p99_step_ms = percentile(s->step_ms, 0.99);
  o->max_step_ms = s->step_ms.empty() ? 0.0 : *std::max_element(s->step_ms.begin(), s->step_ms.end());
  o->p50_request_ms = percentile(s->req_ms, 0.50);
  o->p99_request_ms = percentile(s->req_ms, 0.99);
  o->p50_queue_ms = percentile(s->queue_ms, 0.50);
  o->p99_queue_ms = percentile(s->queue_ms, 0.99);
  o->peak_active = s->peak_active;
  o->slots = s->slots;
  o->budget_bytes = s->pool.size();
  o->peak_bytes = s->pool.peak();
  return IRK_OK;
}

void irk_server_destroy(irk_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto st : s->streams) cudaStreamDestroy(st);
  if (s->batch) irk_batch_destroy(s->batch);
  if (s->bstream) cudaStreamDestroy(s->bstream);
  if (s->base) cudaFree(s->base);
  delete s;
}

}  // extern "C"
