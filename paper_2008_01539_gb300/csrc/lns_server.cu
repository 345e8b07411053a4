// lns_server.cu -- a request loop that advances many resident models on one GPU.
//
// Requests "advance model k by dt" arrive at any time (lns_server_submit) and are served by a
// pool of worker threads, each owning one CUDA stream: a worker takes the oldest queued request
// whose model is idle, moves the model to its stream and runs lns_timestep there, so the work of
// different models overlaps on the device (continuous batching: a request that arrives while
// others run starts as soon as a worker and its model are free).  The requests of one model run
// in arrival order, one at a time.
//
// Every model's state stays on the device.  Models are created on the device when first needed
// and admitted against an HBM budget: the device bytes of all resident models are counted through
// the library's allocator hook (stream-ordered cudaMallocAsync), and when a model does not fit,
// idle resident models are evicted, least recently used first, after saving their state and
// support set to the host (restored exactly when the model comes back).
//
// A request runs lns_advance over its interval: a step that fails to converge (LNS_ENOCONV,
// LNS_EKRYLOV) is undone and retried with half the step, and steps grow back after easy ones, down
// to a smallest step of dt * dt_min_fraction.  A request that fails even there leaves its model as
// it was.  The models' solves that fit the thread-block-cluster solver (up to 16 SMs) run side by
// side on the workers' streams; larger ones take the grid solver over every SM, one at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lns_internal.cuh"

namespace {

constexpr double kDefaultMinFraction = 1.0 / 65536.0;

struct Counting {  // allocator context of one model: bytes it holds on the device
  size_t bytes = 0;
};

void* counting_alloc(void* ctx, size_t bytes, void* stream) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) return nullptr;
  ((Counting*)ctx)->bytes += bytes;
  return p;
}

void counting_free(void* ctx, void* ptr, void* stream) {
  (void)ctx;
  cudaFreeAsync(ptr, (cudaStream_t)stream);
}

struct ServedModel {
  // host copy of the description
  lns_model_desc desc{};
  std::vector<int32_t> row_ptr, nbr, line_id, well_cell;
  std::vector<double> trans, pv_ref, depth, well_wi, well_bhp, p0, sw0;
  std::vector<uint8_t> always;
  lns_options opts{};
  // residency
  lns_model* m = nullptr;
  std::unique_ptr<Counting> counting;
  size_t dev_bytes = 0;      // measured at creation (or estimated before the first one)
  bool busy = false;
  bool has_support = false;  // the model has finished a timestep (its support set is in use)
  uint64_t last_used = 0;
  // state saved at eviction
  bool saved = false, saved_support = false;
  std::vector<double> p_saved, sw_saved;
  std::vector<uint32_t> supp_saved;
  // checkpoint of the request's starting state (device [2n]: p, sw; host support bits)
  double* ck = nullptr;
  std::vector<uint32_t> ck_supp;
};

struct Request {
  int64_t id;
  int32_t model;
  double dt;
  double t_submit;
};

}  // namespace

struct lns_server {
  lns_server_options o{};
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::deque<lns_completion> done;
  std::vector<std::unique_ptr<ServedModel>> models;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;  // one per worker, owned by the server (models keep using the
                                      // stream of their last request until they move)
  bool stop = false;
  int in_flight = 0;
  uint64_t tick = 0;
  size_t resident_bytes = 0;
  lns_server_stats st{};
  int device = 0;
  double min_fraction = kDefaultMinFraction;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

lns_status fail(lns_status s, const std::string& msg) {
  lns::set_last_error(msg.c_str());
  return s;
}

size_t estimate_bytes(const ServedModel& sm) {
  // a model holds about 500 B per cell (state, sets, line factors, Krylov vectors) and 96 B per
  // CSR entry (graph, blocks); used only until its first creation measures the real figure
  return (size_t)sm.desc.n_cells * 520 + (size_t)sm.desc.n_adj * 96 + (1u << 20);
}

// Save an idle resident model to the host and free its device memory (lock held).
lns_status evict(lns_server* s, ServedModel& sm, cudaStream_t stream) {
  const int n = sm.desc.n_cells;
  sm.p_saved.resize(n);
  sm.sw_saved.resize(n);
  sm.supp_saved.resize((n + 31) / 32);
  lns_status r = lns_set_stream(sm.m, stream);
  if (r == LNS_OK) r = lns_get_state(sm.m, sm.p_saved.data(), sm.sw_saved.data());
  if (r == LNS_OK) r = lns_get_support(sm.m, sm.supp_saved.data());
  if (r != LNS_OK) return r;
  sm.saved = true;
  sm.saved_support = sm.has_support;
  if (sm.ck) {
    cudaFreeAsync(sm.ck, stream);
    sm.ck = nullptr;
  }
  lns_model_destroy(sm.m);
  cudaStreamSynchronize(stream);
  sm.m = nullptr;
  s->resident_bytes -= std::min(s->resident_bytes, sm.dev_bytes);
  s->st.evictions++;
  return LNS_OK;
}

// Make room for `need` bytes by evicting idle models, least recently used first (lock held).
// Returns false if the idle models cannot free enough.
bool make_room(lns_server* s, size_t need, const ServedModel* keep, cudaStream_t stream) {
  if (s->o.hbm_budget_bytes <= 0) return true;
  const size_t budget = (size_t)s->o.hbm_budget_bytes;
  while (s->resident_bytes + need > budget) {
    ServedModel* lru = nullptr;
    for (auto& p : s->models)
      if (p->m && !p->busy && p.get() != keep && (!lru || p->last_used < lru->last_used)) lru = p.get();
    if (!lru) return false;
    if (evict(s, *lru, stream) != LNS_OK) return false;
  }
  return true;
}

// Create (or re-create) the device model on `stream` (lock not held; the model is marked busy).
lns_status admit(ServedModel& sm, cudaStream_t stream) {
  sm.counting.reset(new Counting());
  lns_allocator a{sm.counting.get(), counting_alloc, counting_free};
  lns_status r = lns_model_create(&sm.desc, &sm.opts, &a, stream, &sm.m);
  if (r != LNS_OK) return r;
  {  // solves of different models run side by side when they fit the cluster solver; the launch
     // shapes are the model class's cached ones, if measured
    lns_tuning t{};
    lns_get_tuning(sm.m, &t);
    t.cluster_max_rows = -1;
    r = lns_set_tuning(sm.m, &t);
    if (r != LNS_OK) return r;
  }
  if (sm.saved) {
    r = lns_set_state(sm.m, sm.p_saved.data(), sm.sw_saved.data(), nullptr, nullptr);
    if (r == LNS_OK && sm.saved_support) r = lns_set_support(sm.m, sm.supp_saved.data());
    if (r != LNS_OK) return r;
  }
  sm.dev_bytes = sm.counting->bytes + (size_t)sm.desc.n_cells * 2 * sizeof(double);  // + checkpoint
  return LNS_OK;
}

// One request: lns_advance over dt with the cut/grow controller (first step dt, smallest
// dt * min_fraction).  A request that fails leaves the model as it was before it.
lns_status advance(ServedModel& sm, double dt, double min_fraction, lns_step_stats* acc, cudaStream_t stream) {
  const int n = sm.desc.n_cells;
  if (!sm.ck && cudaMallocAsync((void**)&sm.ck, sizeof(double) * 2 * (size_t)std::max(n, 1), stream) != cudaSuccess) {
    sm.ck = nullptr;
    return fail(LNS_ENOMEM, "checkpoint allocation failed");
  }
  sm.ck_supp.resize((n + 31) / 32);
  lns_status r = lns_get_state_device(sm.m, sm.ck, sm.ck + n);
  if (r == LNS_OK) r = lns_get_support(sm.m, sm.ck_supp.data());
  if (r != LNS_OK) return r;
  const bool had_support = sm.has_support;
  const lns_dt_control ctl{dt, dt * min_fraction, dt, 2.0, 0.5, 4};
  lns_advance_stats a{};
  r = lns_advance(sm.m, dt, &ctl, &a);
  if (a.steps > 0) sm.has_support = true;
  acc->iterations += a.iterations;
  acc->krylov_iters += (int32_t)a.krylov_iters;
  acc->cell_updates += a.cell_updates;
  acc->dd_outer += a.cuts;  // counts the cuts
  if (r == LNS_OK) return r;
  lns_status q = lns_set_state_device(sm.m, sm.ck, sm.ck + n);
  if (q == LNS_OK) q = lns_set_support(sm.m, had_support ? sm.ck_supp.data() : nullptr);
  sm.has_support = had_support;
  return q != LNS_OK ? q : r;
}

void worker_loop(lns_server* s, cudaStream_t stream) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // the oldest request whose model is idle (requests of one model stay in order)
    auto it = s->queue.end();
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if (!s->models[q->model]->busy) {
        it = q;
        break;
      }
    if (it == s->queue.end()) {
      if (s->stop) break;
      s->cv_work.wait(lk);
      continue;
    }
    Request rq = *it;
    ServedModel& sm = *s->models[rq.model];
    // admission against the HBM budget
    bool created = false;
    if (!sm.m) {
      const size_t need = sm.dev_bytes ? sm.dev_bytes : estimate_bytes(sm);
      // a model that does not fit even with every idle model evicted waits for the running ones;
      // with nothing else resident it runs alone (the budget bounds co-residency)
      if (!make_room(s, need, &sm, stream) && !(s->resident_bytes == 0 && s->in_flight == 0)) {
        s->cv_work.wait(lk);  // wait for a request to finish and a model to become idle
        continue;
      }
      s->resident_bytes += need;
      created = true;
    }
    s->queue.erase(it);
    sm.busy = true;
    s->in_flight++;
    const size_t reserved = created ? (sm.dev_bytes ? sm.dev_bytes : estimate_bytes(sm)) : 0;
    lk.unlock();

    const double t_start = s->now();
    lns_step_stats acc{};
    lns_status r = LNS_OK;
    if (created) {
      r = admit(sm, stream);
    } else {
      r = lns_set_stream(sm.m, stream);
    }
    if (r == LNS_OK) r = advance(sm, rq.dt, s->min_fraction, &acc, stream);
    acc.status = r;
    const double t_done = s->now();

    lk.lock();
    if (created) {
      s->resident_bytes -= std::min(s->resident_bytes, reserved);
      if (sm.m) {
        s->resident_bytes += sm.dev_bytes;
        s->st.admissions++;
      }
    }
    if (sm.m && sm.counting) {  // buffers allocated during the first solves count as well
      const size_t now_bytes = sm.counting->bytes + (size_t)sm.desc.n_cells * 2 * sizeof(double);
      s->resident_bytes += now_bytes - std::min(now_bytes, sm.dev_bytes);
      sm.dev_bytes = std::max(sm.dev_bytes, now_bytes);
    }
    sm.busy = false;
    sm.last_used = ++s->tick;
    s->in_flight--;
    lns_completion c{};
    c.request_id = rq.id;
    c.model = rq.model;
    c.dt = rq.dt;
    c.status = r;
    c.t_submit = rq.t_submit;
    c.t_start = t_start;
    c.t_done = t_done;
    c.stats = acc;
    s->done.push_back(c);
    if (r == LNS_OK)
      s->st.completed++;
    else
      s->st.failed++;
    s->st.cell_updates += acc.cell_updates;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  lk.unlock();
  cudaStreamSynchronize(stream);
}

template <typename T>
std::vector<T> copy_of(const T* p, size_t n) {
  return p ? std::vector<T>(p, p + n) : std::vector<T>();
}

}  // namespace

extern "C" {

lns_status lns_server_create(const lns_server_options* o, lns_server** out) {
  if (!o || !out) return fail(LNS_EINVAL, "options and out must be non-NULL");
  if (o->workers < 1 || o->workers > 64) return fail(LNS_EINVAL, "workers must be in [1, 64]");
  if (o->hbm_budget_bytes < 0) return fail(LNS_EINVAL, "hbm_budget_bytes must be >= 0");
  if (o->dt_min_fraction < 0.0 || o->dt_min_fraction >= 1.0) return fail(LNS_EINVAL, "dt_min_fraction must be in [0, 1)");
  lns_server* s = new lns_server();
  s->o = *o;
  if (o->dt_min_fraction > 0.0) s->min_fraction = o->dt_min_fraction;
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->device);
  for (int w = 0; w < o->workers; w++) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto q : s->streams) cudaStreamDestroy(q);
      delete s;
      return fail(LNS_ECUDA, "cannot create the worker streams");
    }
    s->streams.push_back(st);
  }
  for (int w = 0; w < o->workers; w++) s->workers.emplace_back(worker_loop, s, s->streams[w]);
  *out = s;
  return LNS_OK;
}

lns_status lns_server_destroy(lns_server* s) {
  if (!s) return LNS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  // models are freed on the stream of their last request (still alive), then the streams go
  for (auto& p : s->models) {
    if (!p->m) continue;
    if (p->ck) {
      cudaFreeAsync(p->ck, s->streams[0]);
      p->ck = nullptr;
    }
    lns_set_stream(p->m, s->streams[0]);
    lns_model_destroy(p->m);
    p->m = nullptr;
  }
  for (auto q : s->streams) {
    cudaStreamSynchronize(q);
    cudaStreamDestroy(q);
  }
  delete s;
  return LNS_OK;
}

lns_status lns_server_add_model(lns_server* s, const lns_model_desc* d, const lns_options* opts, int32_t* id) {
  if (!s || !d || !id) return fail(LNS_EINVAL, "server, desc and id must be non-NULL");
  if (d->n_cells < 0 || d->n_adj < 0 || d->n_wells < 0) return fail(LNS_EINVAL, "negative sizes");
  std::unique_ptr<ServedModel> sm(new ServedModel());
  const size_t n = (size_t)d->n_cells, na = (size_t)d->n_adj, nw = (size_t)d->n_wells;
  sm->row_ptr = copy_of(d->row_ptr, n + 1);
  sm->nbr = copy_of(d->nbr, na);
  sm->trans = copy_of(d->trans, na);
  sm->pv_ref = copy_of(d->pv_ref, n);
  sm->depth = copy_of(d->depth, n);
  sm->line_id = copy_of(d->line_id, n);
  sm->always = copy_of(d->always_active, n);
  sm->well_cell = copy_of(d->well_cell, nw);
  sm->well_wi = copy_of(d->well_wi, nw);
  sm->well_bhp = copy_of(d->well_bhp, nw);
  sm->p0 = copy_of(d->p0, n);
  sm->sw0 = copy_of(d->sw0, n);
  sm->desc = *d;
  auto ptr = [](auto& v) { return v.empty() ? nullptr : v.data(); };
  sm->desc.row_ptr = ptr(sm->row_ptr);
  sm->desc.nbr = ptr(sm->nbr);
  sm->desc.trans = ptr(sm->trans);
  sm->desc.pv_ref = ptr(sm->pv_ref);
  sm->desc.depth = ptr(sm->depth);
  sm->desc.line_id = ptr(sm->line_id);
  sm->desc.always_active = ptr(sm->always);
  sm->desc.well_cell = ptr(sm->well_cell);
  sm->desc.well_wi = ptr(sm->well_wi);
  sm->desc.well_bhp = ptr(sm->well_bhp);
  sm->desc.p0 = ptr(sm->p0);
  sm->desc.sw0 = ptr(sm->sw0);
  if (opts) {
    sm->opts = *opts;
  } else {
    lns_options_default(&sm->opts);
  }
  // validate now: a model that cannot be created would fail every request
  {
    lns_status r = lns::validate_desc(&sm->desc);
    if (r == LNS_OK) r = lns::validate_opts(&sm->opts);
    if (r != LNS_OK) return r;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *id = (int32_t)s->models.size();
  s->models.push_back(std::move(sm));
  s->st.models = (int32_t)s->models.size();
  return LNS_OK;
}

lns_status lns_server_submit(lns_server* s, int32_t model, double dt, int64_t request_id) {
  if (!s) return fail(LNS_EINVAL, "server is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(LNS_EINVAL, "dt must be positive and finite");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (model < 0 || model >= (int32_t)s->models.size()) return fail(LNS_EINVAL, "unknown model");
    s->queue.push_back(Request{request_id, model, dt, s->now()});
    s->st.submitted++;
  }
  s->cv_work.notify_one();
  return LNS_OK;
}

lns_status lns_server_cancel(lns_server* s, int64_t request_id) {
  if (!s) return fail(LNS_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (q->id == request_id) {
      lns_completion c{};
      c.request_id = q->id;
      c.model = q->model;
      c.dt = q->dt;
      c.status = LNS_ESTATE;  // cancelled before it started; the model is unchanged
      c.t_submit = q->t_submit;
      c.t_start = c.t_done = s->now();
      s->queue.erase(q);
      s->done.push_back(c);
      s->st.cancelled++;
      s->cv_done.notify_all();
      return LNS_OK;
    }
  return fail(LNS_ESTATE, "request is not queued (unknown, running or finished)");
}

lns_status lns_server_poll(lns_server* s, lns_completion* out, int32_t cap, double timeout_s, int32_t* count) {
  if (!s || !count || (cap > 0 && !out)) return fail(LNS_EINVAL, "bad arguments");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_s > 0.0)
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [s] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < cap && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *count = k;
  return LNS_OK;
}

lns_status lns_server_drain(lns_server* s, double timeout_s) {
  if (!s) return fail(LNS_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [s] { return s->queue.empty() && s->in_flight == 0; });
  return ok ? LNS_OK : fail(LNS_ESTATE, "drain timed out");
}

lns_status lns_server_get_state(lns_server* s, int32_t model, double* p, double* sw) {
  if (!s) return fail(LNS_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  if (model < 0 || model >= (int32_t)s->models.size()) return fail(LNS_EINVAL, "unknown model");
  ServedModel& sm = *s->models[model];
  if (sm.busy) return fail(LNS_ESTATE, "model is running a request");
  const size_t n = (size_t)sm.desc.n_cells;
  if (!sm.m) {  // evicted or never admitted
    const std::vector<double>& ps = sm.saved ? sm.p_saved : sm.p0;
    const std::vector<double>& ss = sm.saved ? sm.sw_saved : sm.sw0;
    if (p) std::memcpy(p, ps.data(), n * sizeof(double));
    if (sw) std::memcpy(sw, ss.data(), n * sizeof(double));
    return LNS_OK;
  }
  return lns_get_state(sm.m, p, sw);
}

lns_status lns_server_get_stats(lns_server* s, lns_server_stats* out) {
  if (!s || !out) return fail(LNS_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->resident_bytes = (int64_t)s->resident_bytes;
  out->resident_models = 0;
  for (auto& p : s->models) out->resident_models += p->m ? 1 : 0;
  out->queued = (int32_t)s->queue.size();
  out->in_flight = s->in_flight;
  return LNS_OK;
}

double lns_server_now(lns_server* s) { return s ? s->now() : 0.0; }

}  // extern "C"
