// lns_capi.cu -- C ABI and host driver of the localized Newton solver.
//
// The host side only sequences kernels and reads back one small counter block per Newton
// iteration (n_A, convergence, expand/shrink, Krylov outcome); every step of the
// iteration -- active-set estimate, compaction, assembly, BiCGStab, update scatter -- runs
// in the kernels of k_sets.cu, k_assemble.cu and k_krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "lns_internal.cuh"

namespace {
thread_local std::string g_err;
}  // namespace

namespace lns {
static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace lns

using lns::Dev;
using lns::IterCounters;
using lns::LaunchCfg;

namespace {

lns_status fail(lns_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(LNS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(call)                   \
  do {                              \
    lns_status s_ = (call);         \
    if (s_ != LNS_OK) return s_;    \
  } while (0)

enum KClass { KC_COMPACT = 0, KC_SETS, KC_ASSEMBLE, KC_LINES, KC_KRYLOV, KC_UPDATE, KC_COUNT };
const char* kClassName[KC_COUNT] = {"compact", "active_set", "assemble", "line_setup", "bicgstab", "update"};

struct PendingEvent {
  int kc;
  bool on;    // this class is timed at the model's profiling level
  bool keep;  // the events belong to a captured graph (not returned to the pool)
  cudaEvent_t a, b;
  double bytes, flops;
};

}  // namespace

struct lns_model {
  Dev d{};
  lns_options o{};
  lns_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  int sms = 1;
  int device = 0;
  std::vector<void*> owned;
  double avg_degree = 0.0;
  int kgrid[2] = {0, 0};  // cooperative BiCGStab grid (FP64, FP32)
  lns::ClusterShape kcl[2][2] = {};  // cluster BiCGStab [fp32][lines] for the current krylov_cluster
  int kcl_max = -2;                  // krylov_cluster the shapes were computed for
  int fault_h = 0;                   // host copy of the injected solver fault (lns_debug_fault)
  lns_tuning tune{};                 // launch shapes and solver choice (lns_autotune / lns_set_tuning)
  bool tune_explicit = false;        // set by the caller: cached tunings do not replace it
  // batched advance (lns_batch_advance): the iteration split around the solve, each half captured
  cudaGraph_t bg[2] = {nullptr, nullptr};
  cudaGraphExec_t bx[2] = {nullptr, nullptr};
  int64_t bx_kernels[2] = {0, 0};
  bool bgraph_ok = true;
  // timestep state
  bool step_open = false;
  double dt = 0.0;
  int has_prev = 0;
  int is_expand = 1;
  int converged = 0;
  lns_step_stats cur{};
  // Algorithm 2 storage: per subdomain V_A^k, V_B^k, V_dB^k bitsets
  std::vector<uint32_t*> dd_va, dd_vb, dd_vdb;
  uint32_t* dd_vt = nullptr;
  uint32_t* dd_set = nullptr;  // the solved set of a visit's further steps (Algorithm 2 variants)
  std::vector<uint32_t> stage;  // host staging of caller bitsets
  // dt of the current solve, in device memory (d.stepp) via a pinned staging pair
  double* dt_host = nullptr;
  double dt_dev = -1.0;
  // one Newton iteration captured as a CUDA graph (single-stream models without profiling)
  bool graph_ok = true;
  double* ck_state = nullptr;  // lns_advance: p and Sw at the start of the step being tried
  uint32_t* ck_prev = nullptr;  // lns_advance: the support set seeding that step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_kernels = 0;
  std::vector<PendingEvent> graph_pending;  // event pairs recorded by the graph (profile level 2)
  // profiling
  std::vector<cudaEvent_t> ev_pool;
  std::vector<PendingEvent> pending;
  lns_kernel_time kt[KC_COUNT]{};
};

namespace {

LaunchCfg cfg(const lns_model* m) {
  LaunchCfg c{m->sms, m->stream};
  c.asm_block = m->tune.asm_block;
  c.asm_mult = m->tune.asm_blocks_per_sm;
  c.set_mult = m->tune.set_blocks_per_sm;
  return c;
}

// dt and 1/dt of the next solves to the device (only when dt changes; the previous upload of the
// pinned pair has completed: every solve ends with a stream synchronization)
lns_status set_dt(lns_model* m, double dt) {
  m->dt = dt;
  if (dt == m->dt_dev) return LNS_OK;
  m->dt_host[0] = dt;
  m->dt_host[1] = 1.0 / dt;
  cudaError_t e = cudaMemcpyAsync(m->d.stepp, m->dt_host, 2 * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e != cudaSuccess) return fail(LNS_ECUDA, std::string("dt upload: ") + cudaGetErrorString(e));
  m->dt_dev = dt;
  return LNS_OK;
}

void drop_graph(lns_model* m) {
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->gexec = nullptr;
  m->graph = nullptr;
  for (int k = 0; k < 2; k++) {
    if (m->bx[k]) cudaGraphExecDestroy(m->bx[k]);
    if (m->bg[k]) cudaGraphDestroy(m->bg[k]);
    m->bx[k] = nullptr;
    m->bg[k] = nullptr;
  }
  for (auto& pe : m->graph_pending) {
    m->ev_pool.push_back(pe.a);
    m->ev_pool.push_back(pe.b);
  }
  m->graph_pending.clear();
}

lns_status dalloc(lns_model* m, size_t bytes, void** out) {
  bytes = std::max<size_t>(bytes, 256);
  void* p = nullptr;
  if (m->has_alloc) {
    p = m->alloc.alloc(m->alloc.ctx, bytes, (void*)m->stream);
    if (!p) return fail(LNS_ENOMEM, "device allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(LNS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  m->owned.push_back(p);
  *out = p;
  return LNS_OK;
}

template <typename T>
lns_status dalloc_t(lns_model* m, size_t count, T** out) {
  void* p = nullptr;
  TRY(dalloc(m, count * sizeof(T), &p));
  *out = (T*)p;
  return LNS_OK;
}

double eff_p_scale(const lns_model* m) {
  if (m->o.p_scale > 0.0) return m->o.p_scale;
  double c = m->d.fl.c_r + m->d.fl.c_o;
  return c > 0.0 ? c : 1e-7;
}

// ---- profiling ----
// Record an event on the model's stream; under stream capture as an external event-record node,
// so that every launch of the graph records it (a plain record would only order the capture).
cudaError_t record(lns_model* m, cudaEvent_t e) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(m->stream, &cap);
  if (r != cudaSuccess) return r;
  if (cap != cudaStreamCaptureStatusNone) return cudaEventRecordWithFlags(e, m->stream, cudaEventRecordExternal);
  return cudaEventRecord(e, m->stream);
}

lns_status ev_begin(lns_model* m, int kc, PendingEvent* pe) {
  pe->kc = kc;
  pe->bytes = pe->flops = 0.0;
  pe->keep = false;
  pe->on = m->o.profile == 1 || (m->o.profile == 2 && kc == KC_KRYLOV);
  if (!pe->on) return LNS_OK;
  if (m->ev_pool.size() < 2) {
    for (int k = 0; k < 32; k++) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      m->ev_pool.push_back(e);
    }
  }
  pe->a = m->ev_pool.back();
  m->ev_pool.pop_back();
  pe->b = m->ev_pool.back();
  m->ev_pool.pop_back();
  CK(record(m, pe->a));
  return LNS_OK;
}

lns_status ev_end(lns_model* m, PendingEvent* pe, double bytes, double flops) {
  if (!pe->on) return LNS_OK;
  pe->bytes = bytes;
  pe->flops = flops;
  CK(record(m, pe->b));
  m->pending.push_back(*pe);
  return LNS_OK;
}

// After a stream synchronization: accumulate the recorded intervals.
lns_status ev_flush(lns_model* m) {
  for (auto& pe : m->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pe.a, pe.b));
    lns_kernel_time& k = m->kt[pe.kc];
    k.launches += 1;
    k.total_ms += ms;
    k.bytes += pe.bytes;
    k.flops += pe.flops;
    if (!pe.keep) {
      m->ev_pool.push_back(pe.a);
      m->ev_pool.push_back(pe.b);
    }
  }
  m->pending.clear();
  return LNS_OK;
}

// Algorithmic traffic models (bytes and flops per launch) from the row count; sT = 8 or 4.
double bytes_assemble(double nA, double deg, double sT) { return nA * (52.0 + 2 * sT + deg * (20.0 + 4 * sT)); }
// FP64 instructions (per thread) of the assembly and its property pass per active row: the count
// ncu reports on the 400x400 DFN case (291 per row at mean degree 4.0), split as 2 lanes x
// (70 + 19 per connection)
double flops_assemble(double nA, double deg) { return nA * 2.0 * (70.0 + 19.0 * deg); }
double bytes_krylov_iter(double nA, double deg, double sT) {
  return nA * (2.0 * (12.0 + deg * (4.0 + 6.0 * sT) + 2.0 * sT) + 34.0 * sT);
}
double flops_krylov_iter(double nA, double deg) { return nA * (2.0 * (8.0 * deg + 2.0) + 70.0); }

lns_status sync(lns_model* m) {
  CK(cudaStreamSynchronize(m->stream));
  return ev_flush(m);
}

lns_status read_counters(lns_model* m) {
  CK(cudaMemcpyAsync(m->d.ctr_h, m->d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
  return sync(m);
}

double bits2d(unsigned long long b) {
  double v;
  std::memcpy(&v, &b, sizeof(v));
  return v;
}

lns_status reset_iter(lns_model* m) {
  const Dev& d = m->d;
  CK(cudaMemsetAsync(d.ctr, 0, sizeof(IterCounters), m->stream));
  CK(cudaMemsetAsync(d.supp, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  CK(cudaMemsetAsync(d.reach, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  CK(cudaMemsetAsync(d.vb, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));  // V_B is written by the assembly
  return LNS_OK;
}

// Caller bitsets are copied with the bits past n_cells cleared, so no kernel sees a cell >= n.
lns_status bits_to_device(lns_model* m, uint32_t* dst, const uint32_t* host) {
  const int W = m->d.W, n = m->d.n;
  if (W == 0) return LNS_OK;
  m->stage.assign(host, host + W);
  const int rem = n - 32 * (W - 1);
  if (rem < 32) m->stage[W - 1] &= (1u << rem) - 1u;
  CK(cudaMemcpyAsync(dst, m->stage.data(), sizeof(uint32_t) * (size_t)W, cudaMemcpyHostToDevice, m->stream));
  CK(cudaStreamSynchronize(m->stream));  // the staging buffer is reused
  return LNS_OK;
}

lns_status bits_to_host(lns_model* m, uint32_t* host, const uint32_t* src) {
  CK(cudaMemcpyAsync(host, src, sizeof(uint32_t) * (size_t)m->d.W, cudaMemcpyDeviceToHost, m->stream));
  return LNS_OK;
}

// Shape of the cluster solver for the model's krylov_cluster option (queried once per value).
lns::ClusterShape cluster_shape(lns_model* m, int fp32, int lines) {
  const int want = m->o.krylov_cluster < 0 ? 16 : m->o.krylov_cluster;
  if (want != m->kcl_max) {
    for (int f = 0; f < 2; f++)
      for (int l = 0; l < 2; l++) m->kcl[f][l] = lns::krylov_cluster_shape(f, l, want);
    m->kcl_max = want;
  }
  lns::ClusterShape cl = m->kcl[fp32 ? 1 : 0][lines ? 1 : 0];
  if (cl.ctas > 0 && m->tune.cluster_max_rows >= 0) {  // the autotuner's threshold (< 0: capacity)
    if (m->tune.cluster_max_rows == 0) return lns::ClusterShape{0, -1};
    cl.cap = std::min(cl.cap, m->tune.cluster_max_rows);
  }
  return cl;
}

// Solve the local system on the set currently in d.va at the current state: compaction,
// assembly, line factors, BiCGStab.  Leaves the Krylov solution in d.kx.
lns_status local_solve(lns_model* m, int debug) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  const int fp32 = m->o.krylov_fp32;
  PendingEvent pe;
  TRY(ev_begin(m, KC_COMPACT, &pe));
  CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, c));
  TRY(ev_end(m, &pe, d.W * 4.0 * 2 + 0.0, 0.0));
  if (fp32 && !d.raw) TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.raw));
  TRY(ev_begin(m, KC_ASSEMBLE, &pe));
  const int lines = m->o.precond == LNS_PRECOND_BJAC;
  CK(lns::launch_assemble(d, eff_p_scale(m), fp32, lines, debug, c));
  TRY(ev_end(m, &pe, 0.0, 0.0));
  if (lines) {
    TRY(ev_begin(m, KC_LINES, &pe));
    CK(lns::launch_line_setup(d, fp32, c));
    TRY(ev_end(m, &pe, 0.0, 0.0));
  }
  TRY(ev_begin(m, KC_KRYLOV, &pe));
  CK(lns::launch_bicgstab(d, fp32, lines, m->o.krylov_rtol, m->o.krylov_maxit, m->kgrid[fp32 ? 1 : 0],
                          cluster_shape(m, fp32, lines), c));
  TRY(ev_end(m, &pe, 0.0, 0.0));
  return LNS_OK;
}

// Fill in the byte/flop models of the events recorded by local_solve once n_A and the
// Krylov iteration count are known (after the counter read-back).
void annotate_pending(lns_model* m) {
  const IterCounters& h = *m->d.ctr_h;
  const double sT = m->o.krylov_fp32 ? 4.0 : 8.0;
  const double nA = h.n_active;
  for (auto& pe : m->pending) {
    if (pe.kc == KC_ASSEMBLE) {
      pe.bytes = bytes_assemble(nA, m->avg_degree, sT);
      pe.flops = flops_assemble(nA, m->avg_degree);
    } else if (pe.kc == KC_KRYLOV) {
      pe.bytes = h.krylov_iters * bytes_krylov_iter(nA, m->avg_degree, sT);
      pe.flops = h.krylov_iters * flops_krylov_iter(nA, m->avg_degree);
    } else if (pe.kc == KC_UPDATE) {
      pe.bytes = nA * (4.0 + 2 * sT + 48.0);
      pe.flops = nA * 6.0;
    }
  }
}

lns_status krylov_outcome(lns_model* m) {
  const IterCounters& h = *m->d.ctr_h;
  if (h.krylov_status == 2) return fail(LNS_EKRYLOV, "BiCGStab breakdown");
  if (h.krylov_status == 3) return fail(LNS_ETIMEOUT, "BiCGStab grid barrier wait gave up (bounded wait ran out)");
  if (h.krylov_status == 1 && !(h.krylov_relres <= m->o.krylov_fail_rtol))
    return fail(LNS_EKRYLOV, "BiCGStab reached krylov_maxit with relative residual " + std::to_string(h.krylov_relres));
  return LNS_OK;
}

// m rounds of frontier expansion of d.reach (frontier list 0 already seeded).  Rounds run in
// chunks of 8; between chunks the frontier size is read and an empty frontier ends the
// expansion early (so m larger than the graph diameter costs no more than the diameter).
lns_status dilate(lns_model* m, int layers) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  int done = 0;
  while (done < layers) {
    const int chunk = std::min(8, layers - done);
    CK(lns::launch_dilate(d, d.reach, chunk, c));
    done += chunk;
    if (done >= layers) break;
    // chunk == 8 (even): the current frontier is list 0
    int cnt = 0;
    CK(cudaMemcpyAsync(&m->d.ctr_h->n_frontier[0], &d.ctr->n_frontier[0], sizeof(int), cudaMemcpyDeviceToHost,
                       m->stream));
    CK(cudaStreamSynchronize(m->stream));
    cnt = m->d.ctr_h->n_frontier[0];
    if (cnt == 0) break;
  }
  return LNS_OK;
}

// Initial active set of a timestep (Section 4.3 step 1, Section 5.2): previous step's
// support plus always-active cells, or on the first step the always-active cells and their
// m-layer neighbours.
lns_status initial_set(lns_model* m, uint32_t* out) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  if (m->has_prev) {
    CK(lns::launch_words_op(d, lns::kOr, out, d.prev, d.always, c));
    return LNS_OK;
  }
  CK(cudaMemsetAsync(d.reach, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  CK(cudaMemsetAsync(d.ctr, 0, sizeof(IterCounters), m->stream));
  if (d.n_always > 0) {
    CK(lns::launch_seed_frontier(d, d.always_list, d.n_always, d.reach, c));
    TRY(dilate(m, m->o.m_layers));
  }
  CK(lns::launch_words_op(d, lns::kCopy, out, d.reach, nullptr, c));
  return LNS_OK;
}

lns_status open_step(lns_model* m, double dt) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(LNS_EINVAL, "dt must be positive and finite");
  TRY(set_dt(m, dt));
  CK(cudaMemcpyAsync(d.pn, d.p, sizeof(double) * (size_t)d.n, cudaMemcpyDeviceToDevice, m->stream));
  CK(cudaMemcpyAsync(d.swn, d.sw, sizeof(double) * (size_t)d.n, cudaMemcpyDeviceToDevice, m->stream));
  if (m->o.mode == LNS_MODE_FULL) {
    CK(lns::launch_words_op(d, lns::kAll, d.va, nullptr, nullptr, c));
    CK(lns::launch_words_op(d, lns::kAll, d.uni, nullptr, nullptr, c));
  } else if (m->o.mode == LNS_MODE_RESIDUAL) {  // the first set comes from the first residual
    CK(cudaMemsetAsync(d.uni, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
    CK(cudaMemsetAsync(d.va, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  } else {
    CK(cudaMemsetAsync(d.uni, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
    TRY(initial_set(m, d.va));
  }
  m->step_open = true;
  m->is_expand = 1;
  m->converged = 0;
  std::memset(&m->cur, 0, sizeof(m->cur));
  return LNS_OK;
}

lns_status close_step(lns_model* m) {
  CK(lns::launch_step_support(m->d, m->o.eps_p, m->o.eps_sw, cfg(m)));
  m->has_prev = 1;
  m->step_open = false;
  return LNS_OK;
}

// The device work of one pass of Algorithm 1 lines 4-21 (or of standard Newton), ending with the
// read-back of the counter block.  Every size is read on the device, so the same sequence serves
// every iteration of every timestep.
lns_status enqueue_iteration(lns_model* m) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  const bool local = m->o.mode == LNS_MODE_LOCAL;
  TRY(reset_iter(m));
  TRY(local_solve(m, 0));  // the assembly also writes V_B of the set being solved
  PendingEvent pe;
  TRY(ev_begin(m, KC_UPDATE, &pe));
  // u^{nu+1} = u^nu + R_A^T du_A, and the flags of Algorithm 1 lines 8-14
  CK(lns::launch_flag(d, local ? d.vb : nullptr, 1, 0, 0, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop,
                      m->o.krylov_fp32, d.kx, m->o.krylov_fail_rtol, c));
  TRY(ev_end(m, &pe, 0.0, 0.0));
  if (local) {
    TRY(ev_begin(m, KC_SETS, &pe));
    TRY(dilate(m, m->o.m_layers));
    CK(lns::launch_alg1_combine(d, m->o.tol_dp, m->o.tol_cnv, -1, c));
    TRY(ev_end(m, &pe, 0.0, 0.0));
  }
  CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
  return LNS_OK;
}

// Capture enqueue_iteration once as a CUDA graph (one launch per Newton iteration instead of a
// dozen kernels, memsets and copies).  Used when nothing in the sequence needs the host: no
// profiling events, no multi-chunk expansion (m <= 8 layers is one launch), one stream.  A
// capture that fails leaves the model on the direct path.
lns_status ensure_graph(lns_model* m) {
  if (m->gexec) return LNS_OK;
  const int64_t before = lns::g_launches.load(std::memory_order_relaxed);
  cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    m->graph_ok = false;
    cudaGetLastError();
    return LNS_OK;
  }
  lns_status r = enqueue_iteration(m);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(m->stream, &g);
  if (r != LNS_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    m->graph_ok = false;
    return LNS_OK;
  }
  e = cudaGraphInstantiate(&m->gexec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    m->gexec = nullptr;
    m->graph_ok = false;
    return LNS_OK;
  }
  m->graph = g;
  m->graph_kernels = lns::g_launches.load(std::memory_order_relaxed) - before;
  lns::count_launches((int)-m->graph_kernels);  // nothing ran during the capture
  m->graph_pending = m->pending;  // event pairs now recorded by every launch of the graph
  for (auto& pe : m->graph_pending) pe.keep = true;
  m->pending.clear();
  return LNS_OK;
}

// An FP32 solve that failed numerically (not a barrier wait that gave up) and left the state
// and V_A untouched is redone in FP64 when the options ask for it.
bool wants_fp64_retry(const lns_model* m) {
  const IterCounters& h = *m->d.ctr_h;
  return m->o.krylov_fp32 && m->o.fp64_fallback && h.solve_failed && h.krylov_status != 3;
}

// Run `body` with the FP64 Krylov path (direct launches), then restore the FP32 option.  The redo
// solves the same system (same state and set); after a stop above krylov_fail_rtol (stagnation or
// krylov_maxit, a finite iterate) its BiCGStab starts from the FP32 iterate (kept in kx0) instead of
// zero, and after a breakdown from zero (the plain FP64 solve, bit for bit).
template <typename F>
lns_status with_fp64_krylov(lns_model* m, F body) {
  Dev& d = m->d;
  const size_t nA = (size_t)std::max(d.ctr_h->n_active, 0);
  const bool warm = d.ctr_h->krylov_status == 1 && std::isfinite(d.ctr_h->krylov_relres) && nA > 0;
  if (warm) CK(cudaMemcpyAsync(d.kx0, d.kx, nA * 2 * sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  m->o.krylov_fp32 = 0;
  d.krylov_warm = warm ? 1 : 0;
  const lns_status r = body();
  d.krylov_warm = 0;
  m->o.krylov_fp32 = 1;
  return r;
}

// A stalled FP32 solve (a stop above krylov_fail_rtol at stagnation or krylov_maxit, with a finite
// iterate) is solved once more in FP32 from its iterate before any FP64 redo: `body` enqueues the
// same solve again (same state and set) and waits for it.  *kit gets the stalled attempt's Krylov
// iterations (0 when nothing was stalled).
template <typename F>
lns_status fp32_restart(lns_model* m, F body, int* kit) {
  Dev& d = m->d;
  const IterCounters& h = *d.ctr_h;
  *kit = 0;
  if (!(wants_fp64_retry(m) && h.krylov_status == 1 && std::isfinite(h.krylov_relres) && h.n_active > 0))
    return LNS_OK;
  *kit = h.krylov_iters;
  CK(cudaMemcpyAsync(d.kx0, d.kx, (size_t)h.n_active * 2 * sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  d.krylov_warm = 1;
  const lns_status r = body();
  d.krylov_warm = 0;
  return r;
}

// Host side of one pass of Algorithm 1 lines 4-21 (or of standard Newton), after its device work
// has completed and the counter block is on the host: an FP32 solve that failed is redone in FP64,
// then the model's iteration state and the caller's statistics are updated.
lns_status finish_iteration(lns_model* m, lns_iter_stats* st) {
  Dev& d = m->d;
  const bool local = m->o.mode == LNS_MODE_LOCAL;
  annotate_pending(m);
  TRY(ev_flush(m));
  const IterCounters& h = *d.ctr_h;
  int retry = 0, kit_fp32 = 0;
  // a stall: one more FP32 solve from the stalled iterate first (the iteration is enqueued again
  // from the unchanged state and set), then FP64 if that stalls too
  TRY(fp32_restart(m, [&]() -> lns_status {
    TRY(enqueue_iteration(m));
    CK(cudaStreamSynchronize(m->stream));
    annotate_pending(m);
    return ev_flush(m);
  }, &kit_fp32));
  if (wants_fp64_retry(m)) {
    retry = 1;
    kit_fp32 += h.krylov_iters;
    TRY(with_fp64_krylov(m, [&]() -> lns_status {
      TRY(enqueue_iteration(m));
      CK(cudaStreamSynchronize(m->stream));
      annotate_pending(m);
      return ev_flush(m);
    }));
    m->cur.fp64_retries += 1;
  }
  const double maxdp = bits2d(h.max_dp_bits), cnv = bits2d(h.cnv_bits);
  m->converged = local ? h.converged : (maxdp < m->o.tol_dp && cnv < m->o.tol_cnv);
  m->is_expand = local ? h.is_expand : 0;
  m->cur.iterations += 1;
  m->cur.krylov_iters += kit_fp32 + h.krylov_iters;
  m->cur.cell_updates += h.n_active;
  m->cur.last_max_dp = maxdp;
  m->cur.last_cnv = cnv;
  if (st) {
    st->n_active = h.n_active;
    st->is_expand = m->is_expand;
    st->converged = m->converged;
    st->krylov_iters = kit_fp32 + h.krylov_iters;
    st->krylov_status = h.krylov_status;
    st->fp64_retry = retry;
    st->krylov_relres = h.krylov_relres;
    st->max_dp = maxdp;
    st->max_dsw = bits2d(h.max_dsw_bits);
    st->cnv = cnv;
    st->krylov_solver = h.krylov_solver;
    st->step_done = 0;
  }
  return krylov_outcome(m);
}

// One pass of Algorithm 1 lines 4-21 (or of standard Newton).
lns_status alg1_iteration(lns_model* m, lns_iter_stats* st) {
  Dev& d = m->d;
  if (m->o.krylov_fp32 && !d.raw) TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.raw));
  const bool graph = m->graph_ok && m->o.profile != 1 && m->o.m_layers <= 8;
  if (graph) TRY(ensure_graph(m));
  if (graph && m->gexec) {
    CK(cudaGraphLaunch(m->gexec, m->stream));
    lns::count_launches((int)m->graph_kernels);
    m->pending = m->graph_pending;
  } else {
    TRY(enqueue_iteration(m));
  }
  CK(cudaStreamSynchronize(m->stream));
  return finish_iteration(m, st);
}

// After an iteration: close the timestep when the loop condition of Algorithm 1 (or standard
// Newton's convergence) says so, or fail it at max_newton (lns_newton_iter's rule).
lns_status after_iteration(lns_model* m, lns_iter_stats* st) {
  const bool done = m->o.mode == LNS_MODE_FULL ? m->converged : (!m->is_expand && m->converged);
  if (done) {
    TRY(close_step(m));
    TRY(sync(m));
    if (st) st->step_done = 1;
  } else if (m->cur.iterations >= m->o.max_newton) {
    TRY(close_step(m));
    TRY(sync(m));
    if (st) st->step_done = 1;
    return fail(LNS_ENOCONV, "Newton loop reached max_newton");
  }
  return LNS_OK;
}

// ---------------------------------------------------------------------------------------
// Residual-based active sets (LNS_MODE_RESIDUAL; the estimate the paper compares against,
// Section 1 / Section 4.2).  Each iteration: the full-domain residual at u^nu flags the
// unconverged cells (CNV_i >= tol_cnv); converged when none is and (nu = 0 or) the last update's
// max |dp| < tol_dp; else V_A = the flagged cells inflated by m layers (an empty flagged set keeps
// V_A), one local solve on V_A, u += R_A^T du_A.
// ---------------------------------------------------------------------------------------
lns_status residual_timestep(lns_model* m, double dt, lns_step_stats* out) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  TRY(open_step(m, dt));
  const IterCounters& h = *d.ctr_h;
  double last_dp = 0.0;
  lns_status s = LNS_OK;
  for (int it = 0;; it++) {
    TRY(reset_iter(m));
    CK(lns::launch_residual_flags(d, m->o.tol_cnv, c));
    TRY(read_counters(m));
    const int n_unconv = h.n_frontier[0];
    const double cnv = bits2d(h.cnv_bits);
    if (n_unconv == 0 && (it == 0 || last_dp < m->o.tol_dp)) {
      m->converged = 1;
      break;
    }
    if (it >= m->o.max_newton) {
      s = fail(LNS_ENOCONV, "Newton loop reached max_newton");
      break;
    }
    if (n_unconv > 0) {  // reach = flagged cells; inflate by m layers from frontier list 0
      TRY(dilate(m, m->o.m_layers));
      CK(lns::launch_words_op(d, lns::kCopy, d.va, d.reach, nullptr, c));
    }
    CK(lns::launch_words_op(d, lns::kOr, d.uni, d.uni, d.va, c));
    auto solve = [&]() -> lns_status {
      TRY(reset_iter(m));
      TRY(local_solve(m, 0));
      PendingEvent pe;
      TRY(ev_begin(m, KC_UPDATE, &pe));
      CK(lns::launch_flag(d, nullptr, 1, 0, 0, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop,
                          m->o.krylov_fp32, d.kx, m->o.krylov_fail_rtol, c));
      TRY(ev_end(m, &pe, 0.0, 0.0));
      CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
      CK(cudaStreamSynchronize(m->stream));
      annotate_pending(m);
      return ev_flush(m);
    };
    TRY(solve());
    int kit_fp32 = 0;
    TRY(fp32_restart(m, solve, &kit_fp32));
    if (wants_fp64_retry(m)) {
      kit_fp32 += h.krylov_iters;
      TRY(with_fp64_krylov(m, solve));
      m->cur.fp64_retries += 1;
    }
    m->cur.iterations += 1;
    m->cur.krylov_iters += kit_fp32 + h.krylov_iters;
    m->cur.cell_updates += h.n_active;
    last_dp = bits2d(h.max_dp_bits);
    m->cur.last_max_dp = last_dp;
    m->cur.last_cnv = cnv;
    s = krylov_outcome(m);
    if (s != LNS_OK) break;
  }
  if (s == LNS_OK) {
    TRY(close_step(m));
  } else {
    m->step_open = false;
  }
  m->cur.status = s;
  if (out) *out = m->cur;
  return s;
}

// ---------------------------------------------------------------------------------------
// Algorithm 2 (Section 4.4).
// ---------------------------------------------------------------------------------------
lns_status dd_ensure(lns_model* m, size_t k) {
  while (m->dd_va.size() <= k) {
    uint32_t *a, *b, *c;
    TRY(dalloc_t(m, (size_t)m->d.W, &a));
    TRY(dalloc_t(m, (size_t)m->d.W, &b));
    TRY(dalloc_t(m, (size_t)m->d.W, &c));
    m->dd_va.push_back(a);
    m->dd_vb.push_back(b);
    m->dd_vdb.push_back(c);
  }
  return LNS_OK;
}

// Local solve of subdomain k (one Newton step with Dirichlet values from the current u),
// update scatter with Algorithm 2 stamps; vb: boundary set whose large updates seed the
// next expansion (nullptr in the Schwarz loop).  Returns own_big / converged via outputs.
lns_status dd_solve(lns_model* m, uint32_t* va_k, const uint32_t* vb, int solve_id, int* own_big, int* conv) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  auto once = [&]() -> lns_status {
    TRY(reset_iter(m));
    CK(lns::launch_words_op(d, lns::kCopy, d.va, va_k, nullptr, c));
    CK(lns::launch_words_op(d, lns::kOr, d.uni, d.uni, va_k, c));
    TRY(local_solve(m, 0));
    PendingEvent pe;
    TRY(ev_begin(m, KC_UPDATE, &pe));
    CK(lns::launch_flag(d, vb, 1, 1, solve_id, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop,
                        m->o.krylov_fp32, d.kx, m->o.krylov_fail_rtol, c));
    TRY(ev_end(m, &pe, 0.0, 0.0));
    if (vb) TRY(dilate(m, m->o.m_layers));
    CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    annotate_pending(m);
    return ev_flush(m);
  };
  TRY(once());
  const IterCounters& h = *d.ctr_h;
  int kit_fp32 = 0;
  TRY(fp32_restart(m, once, &kit_fp32));
  if (wants_fp64_retry(m)) {  // a failed solve scattered nothing and stamped nothing
    kit_fp32 += h.krylov_iters;
    TRY(with_fp64_krylov(m, once));
    m->cur.fp64_retries += 1;
  }
  const double maxdp = bits2d(h.max_dp_bits), cnv = bits2d(h.cnv_bits);
  *own_big = h.any_s;
  *conv = maxdp < m->o.tol_dp && cnv < m->o.tol_cnv;
  m->cur.iterations += 1;
  m->cur.krylov_iters += kit_fp32 + h.krylov_iters;
  m->cur.cell_updates += h.n_active;
  m->cur.last_max_dp = maxdp;
  m->cur.last_cnv = cnv;
  return krylov_outcome(m);
}

// Algorithm 2 lines 8-22 on the update already flagged (reach holds the m-layer expansion of
// E): next subdomain, V_T, boundary and halo sets.  Reads is_expand back.
lns_status dd_expand_sets(lns_model* m, uint32_t* vt, uint32_t* va_next, uint32_t* vb_next, uint32_t* vdb_next,
                          int* is_expand) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  CK(cudaMemsetAsync(&d.ctr->any_new, 0, sizeof(int), m->stream));
  CK(lns::launch_dd_combine(d, d.reach, vt, va_next, c));
  CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
  TRY(sync(m));
  *is_expand = (d.ctr_h->any_e && d.ctr_h->any_new) ? 1 : 0;
  if (*is_expand) {
    CK(lns::launch_boundary(d, vt, d.tmp0, c));  // V_B of V_T
    CK(lns::launch_words_op(d, lns::kAnd, vb_next, d.tmp0, va_next, c));
    CK(lns::launch_compact(d, va_next, d.fr1, nullptr, &d.ctr->n_frontier[1], c));
    CK(lns::launch_outer_halo(d, va_next, d.fr1, &d.ctr->n_frontier[1], vdb_next, c));
  } else {
    CK(cudaMemsetAsync(vb_next, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
    CK(cudaMemsetAsync(vdb_next, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  }
  return LNS_OK;
}

// Algorithm 2 variants: a subdomain visit's steps after its first (up to dd_local_newton in all),
// stopping at the first that converges; with dd_local_shrink, each solves the support of the
// previous step's update within the subdomain plus its always-active cells (empty: the visit ends).
// Every step stamps with the visit's solve id and can set own_big.
lns_status dd_refine(lns_model* m, uint32_t* va_k, int conv, int solve_id, int* own_big) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  for (int j = 2; j <= m->o.dd_local_newton && !conv; j++) {
    uint32_t* set = va_k;
    if (m->o.dd_local_shrink) {
      CK(lns::launch_words_op(d, lns::kAnd, m->dd_set, d.always, va_k, c));
      CK(lns::launch_words_op(d, lns::kOr, m->dd_set, m->dd_set, d.supp, c));  // supp of the previous step
      set = m->dd_set;
    }
    CK(cudaMemsetAsync(&d.ctr->n_frontier[1], 0, sizeof(int), m->stream));
    CK(lns::launch_compact(d, set, d.fr1, nullptr, &d.ctr->n_frontier[1], c));
    CK(cudaMemcpyAsync(&d.ctr_h->n_frontier[1], &d.ctr->n_frontier[1], sizeof(int), cudaMemcpyDeviceToHost,
                       m->stream));
    TRY(sync(m));
    if (d.ctr_h->n_frontier[1] == 0) break;
    if (m->cur.iterations >= m->o.max_newton * (m->o.max_dd_outer + 1))
      return fail(LNS_ENOCONV, "Algorithm 2 reached its local-solve limit");
    int ob = 0;
    TRY(dd_solve(m, set, nullptr, solve_id, &ob, &conv));
    if (ob) *own_big = 1;
  }
  return LNS_OK;
}

lns_status dd_timestep(lns_model* m, double dt, lns_step_stats* out) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  TRY(open_step(m, dt));
  if (!m->dd_vt) TRY(dalloc_t(m, (size_t)d.W, &m->dd_vt));
  if (!m->dd_set) TRY(dalloc_t(m, (size_t)d.W, &m->dd_set));
  TRY(dd_ensure(m, 0));
  CK(lns::launch_words_op(d, lns::kCopy, m->dd_va[0], d.va, nullptr, c));
  CK(lns::launch_words_op(d, lns::kCopy, m->dd_vt, d.va, nullptr, c));
  CK(lns::launch_boundary(d, d.va, m->dd_vb[0], c));
  CK(lns::launch_compact(d, d.va, d.fr1, nullptr, &d.ctr->n_frontier[1], c));
  CK(lns::launch_outer_halo(d, d.va, d.fr1, &d.ctr->n_frontier[1], m->dd_vdb[0], c));
  CK(cudaMemsetAsync(d.stamp, 0, sizeof(int) * (size_t)d.n, m->stream));
  std::vector<int> last_solve, own_big;
  int solve_id = 0, k = 0, is_expand = 1;
  lns_status st = LNS_OK;
  // expansion phase
  while (is_expand) {
    if (k >= m->o.max_newton) {
      st = fail(LNS_ENOCONV, "Algorithm 2 expansion reached max_newton subdomains");
      break;
    }
    TRY(dd_ensure(m, (size_t)k + 1));
    int ob = 0, conv = 0;
    solve_id++;
    TRY(dd_solve(m, m->dd_va[k], m->dd_vb[k], solve_id, &ob, &conv));
    last_solve.push_back(solve_id);
    own_big.push_back(ob);
    TRY(dd_expand_sets(m, m->dd_vt, m->dd_va[k + 1], m->dd_vb[k + 1], m->dd_vdb[k + 1], &is_expand));
    const lns_status rr = dd_refine(m, m->dd_va[k], conv, solve_id, &own_big.back());
    k++;
    if (rr != LNS_OK) {
      st = rr;
      break;
    }
  }
  const int N = k;
  m->cur.n_subdomains = N;
  // nonlinear DD loop (multiplicative Schwarz)
  int nu = 0;
  bool converged = false;
  while (st == LNS_OK && !converged) {
    if (nu >= m->o.max_dd_outer) {
      st = fail(LNS_ENOCONV, "Algorithm 2 reached max_dd_outer passes");
      break;
    }
    bool all_ok = true;
    for (int s = 0; s < N; s++) {
      CK(lns::launch_halo_check(d, m->dd_vdb[s], last_solve[s], c));
      CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
      TRY(sync(m));
      const int halo = d.ctr_h->halo_flag;
      if (!(own_big[s] || halo)) continue;
      if (m->cur.iterations >= m->o.max_newton * (m->o.max_dd_outer + 1)) {
        st = fail(LNS_ENOCONV, "Algorithm 2 reached its local-solve limit");
        break;
      }
      int ob = 0, conv = 0;
      solve_id++;
      TRY(dd_solve(m, m->dd_va[s], nullptr, solve_id, &ob, &conv));
      last_solve[s] = solve_id;
      own_big[s] = ob;
      if (!conv) all_ok = false;  // the pass converges when every visited subdomain was already converged
      const lns_status rr = dd_refine(m, m->dd_va[s], conv, solve_id, &own_big[s]);
      if (rr != LNS_OK) {
        st = rr;
        break;
      }
    }
    nu++;
    converged = all_ok;
  }
  m->cur.dd_outer = nu;
  TRY(close_step(m));
  TRY(sync(m));
  m->cur.status = st;
  if (out) *out = m->cur;
  return st;
}

// ---------------------------------------------------------------------------------------
// Batched advance: one Newton iteration of a member split around its solve, so that the host can
// read n_A of every member between the halves and launch only the solver that takes it (the same
// rule the device applies in a single model's iteration: n_A <= the cluster capacity).  Each half
// is captured once per member as a CUDA graph.
// ---------------------------------------------------------------------------------------
lns_status enqueue_pre(lns_model* m) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  TRY(reset_iter(m));
  CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, c));
  const int lines = m->o.precond == LNS_PRECOND_BJAC;
  CK(lns::launch_assemble(d, eff_p_scale(m), m->o.krylov_fp32, lines, 0, c));
  if (lines) CK(lns::launch_line_setup(d, m->o.krylov_fp32, c));
  CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
  return LNS_OK;
}

lns_status enqueue_post(lns_model* m) {
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  const bool local = m->o.mode == LNS_MODE_LOCAL;
  CK(lns::launch_flag(d, local ? d.vb : nullptr, 1, 0, 0, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop,
                      m->o.krylov_fp32, d.kx, m->o.krylov_fail_rtol, c));
  if (local) {
    TRY(dilate(m, m->o.m_layers));
    CK(lns::launch_alg1_combine(d, m->o.tol_dp, m->o.tol_cnv, -1, c));
  }
  CK(cudaMemcpyAsync(d.ctr_h, d.ctr, sizeof(IterCounters), cudaMemcpyDeviceToHost, m->stream));
  return LNS_OK;
}

// Run half k (0 before the solve, 1 after it) of a member's iteration: its graph, captured on first
// use, or direct launches (m_layers > 8: the expansion reads frontier sizes on the host).
lns_status run_half(lns_model* m, int k) {
  auto body = [&]() { return k == 0 ? enqueue_pre(m) : enqueue_post(m); };
  if (!(m->bgraph_ok && m->o.m_layers <= 8)) return body();
  if (!m->bx[k]) {
    const int64_t before = lns::g_launches.load(std::memory_order_relaxed);
    if (cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      m->bgraph_ok = false;
      return body();
    }
    lns_status r = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (r != LNS_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&m->bx[k], g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      m->bx[k] = nullptr;
      cudaGetLastError();
      m->bgraph_ok = false;
      lns::count_launches((int)-(lns::g_launches.load(std::memory_order_relaxed) - before));
      return body();
    }
    m->bg[k] = g;
    m->bx_kernels[k] = lns::g_launches.load(std::memory_order_relaxed) - before;
    lns::count_launches((int)-m->bx_kernels[k]);  // nothing ran during the capture
  }
  CK(cudaGraphLaunch(m->bx[k], m->stream));
  lns::count_launches((int)m->bx_kernels[k]);
  return LNS_OK;
}

// The solver of a batch member's system (n_A read by the host): the cluster solver whenever the
// system fits it.  The autotuner's threshold compares the two solvers' latency on a model alone;
// in a batch the members' cluster solves run concurrently on different SMs, which the grid solver
// (all SMs, one solve at a time) cannot.
lns::ClusterShape batch_shape(lns_model* m) {
  const int fp32 = m->o.krylov_fp32, lines = m->o.precond == LNS_PRECOND_BJAC;
  (void)cluster_shape(m, fp32, lines);  // the capacity for the current krylov_cluster
  return m->kcl[fp32 ? 1 : 0][lines ? 1 : 0];
}

int pick_solver(lns_model* m) {
  const lns::ClusterShape cl = batch_shape(m);
  return (cl.ctas > 0 && m->d.ctr_h->n_active <= cl.cap && m->fault_h != 1) ? 1 : 2;
}

// ---------------------------------------------------------------------------------------
// Autotuner: defaults, process-wide cache, measurement.
// ---------------------------------------------------------------------------------------
lns_tuning default_tuning() {
  lns_tuning t{};
  t.cluster_max_rows = -1;
  t.asm_block = 0;
  t.asm_blocks_per_sm = 0;
  t.set_blocks_per_sm = 0;
  t.measured = 0;
  return t;
}

int size_class(int n) {
  int b = 0;
  while (n > 0) {
    b++;
    n >>= 1;
  }
  return b;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, lns_tuning>& tune_cache() {
  static std::map<std::tuple<int, int, int, int>, lns_tuning> c;
  return c;
}

// the cached tuning of the model's class, unless the caller set one
void apply_cached_tuning(lns_model* m);
// lns_autotune on first use when the options ask for it and nothing decided the tuning yet
lns_status maybe_autotune(lns_model* m);
void apply_cached_tuning(lns_model* m) {
  if (m->tune_explicit) return;
  lns_tuning t;
  if (lns_tune_cache_lookup(m->device, m->o.krylov_fp32, m->o.precond, m->d.n, &t))
    m->tune = t;
  else
    m->tune = default_tuning();
}

lns_status maybe_autotune(lns_model* m) {
  if (!m->o.autotune || m->tune.measured || m->tune_explicit || m->fault_h != 0 || m->o.profile != 0 || m->d.n == 0)
    return LNS_OK;
  apply_cached_tuning(m);  // another model of this class may have measured it meanwhile
  if (m->tune.measured) return LNS_OK;
  return lns_autotune(m, nullptr);
}

lns_status check_model(const lns_model* m) {
  if (!m) return fail(LNS_EINVAL, "model is NULL");
  return LNS_OK;
}

lns_status validate_options(const lns_options* o) {
  if (!o) return fail(LNS_EINVAL, "options is NULL");
  if (o->mode < 0 || o->mode > 3) return fail(LNS_EINVAL, "mode must be 0, 1, 2 or 3");
  if (o->m_layers < 0 || o->m_layers > 100000) return fail(LNS_EINVAL, "m_layers out of range");
  if (o->max_newton < 1 || o->max_dd_outer < 1) return fail(LNS_EINVAL, "max_newton and max_dd_outer must be >= 1");
  if (o->krylov_maxit < 1) return fail(LNS_EINVAL, "krylov_maxit must be >= 1");
  if (!(o->krylov_rtol > 0.0) || !(o->eps_p >= 0.0)) return fail(LNS_EINVAL, "krylov_rtol > 0 and eps_p >= 0 required");
  if (o->precond != LNS_PRECOND_BJAC && o->precond != LNS_PRECOND_BJAC_CELL)
    return fail(LNS_EINVAL, "unknown preconditioner");
  if (o->krylov_cluster > 16 || (o->krylov_cluster > 0 && (o->krylov_cluster & (o->krylov_cluster - 1))))
    return fail(LNS_EINVAL, "krylov_cluster must be < 0, 0, or a power of two <= 16");
  if (o->dd_local_newton < 1 || o->dd_local_shrink < 0 || o->dd_local_shrink > 1)
    return fail(LNS_EINVAL, "dd_local_newton must be >= 1 and dd_local_shrink 0 or 1");
  return LNS_OK;
}

}  // namespace

namespace lns {
lns_status validate_opts(const lns_options* o) { return validate_options(o); }

// Checks of a model description (sizes, arrays, fluid, graph symmetry, wells), on the host.
lns_status validate_desc(const lns_model_desc* desc) {
  if (!desc) return fail(LNS_EINVAL, "desc is NULL");
  const int n = desc->n_cells, na = desc->n_adj;
  if (n < 0 || na < 0) return fail(LNS_EINVAL, "negative sizes");
  if (n > 0 && (!desc->row_ptr || !desc->pv_ref || !desc->depth || !desc->line_id || !desc->always_active ||
                !desc->p0 || !desc->sw0))
    return fail(LNS_EINVAL, "missing cell array");
  if (na > 0 && (!desc->nbr || !desc->trans)) return fail(LNS_EINVAL, "missing connection array");
  if (desc->n_wells < 0 || (desc->n_wells > 0 && (!desc->well_cell || !desc->well_wi || !desc->well_bhp)))
    return fail(LNS_EINVAL, "bad well arrays");
  const lns_fluid& f = desc->fluid;
  if (f.n_w < 1 || f.n_w > 8 || f.n_o < 1 || f.n_o > 8) return fail(LNS_EINVAL, "Corey exponents must be 1..8");
  if (!(f.swc + f.sor < 1.0) || !(f.mu_o > 0.0) || !(f.mu_w > 0.0)) return fail(LNS_EINVAL, "bad fluid constants");
  // graph checks: row_ptr monotone, neighbours in range, no self loops, ascending rows
  if (n > 0) {
    if (desc->row_ptr[0] != 0 || desc->row_ptr[n] != na) return fail(LNS_EINVAL, "row_ptr must run from 0 to n_adj");
    for (int i = 0; i < n; i++) {
      if (desc->row_ptr[i + 1] < desc->row_ptr[i]) return fail(LNS_EINVAL, "row_ptr not monotone");
      for (int e = desc->row_ptr[i]; e < desc->row_ptr[i + 1]; e++) {
        const int j = desc->nbr[e];
        if (j < 0 || j >= n || j == i) return fail(LNS_EINVAL, "neighbour index out of range or self loop");
        if (e > desc->row_ptr[i] && desc->nbr[e - 1] >= j) return fail(LNS_EINVAL, "row neighbours not ascending");
      }
    }
    // every connection stored at both endpoints with the same transmissibility
    for (int i = 0; i < n; i++)
      for (int e = desc->row_ptr[i]; e < desc->row_ptr[i + 1]; e++) {
        const int j = desc->nbr[e];
        const int* b = desc->nbr + desc->row_ptr[j];
        const int* t = desc->nbr + desc->row_ptr[j + 1];
        const int* f = std::lower_bound(b, t, i);
        if (f == t || *f != i || desc->trans[f - desc->nbr] != desc->trans[e])
          return fail(LNS_EINVAL, "connection graph is not symmetric (each connection must be stored at both ends)");
      }
  } else if (na != 0) {
    return fail(LNS_EINVAL, "n_adj must be 0 when n_cells is 0");
  }
  for (int w = 0; w < desc->n_wells; w++)
    if (desc->well_cell[w] < 0 || desc->well_cell[w] >= n) return fail(LNS_EINVAL, "well cell out of range");
  for (int i = 0; i < n; i++)
    if (!std::isfinite(desc->p0[i]) || !std::isfinite(desc->sw0[i]) || !(desc->pv_ref[i] > 0.0) ||
        !std::isfinite(desc->pv_ref[i]) || !std::isfinite(desc->depth[i]))
      return fail(LNS_EINVAL, "non-finite initial state or cell data (cell " + std::to_string(i) + ")");
  for (int e = 0; e < na; e++)
    if (!std::isfinite(desc->trans[e]) || desc->trans[e] < 0.0)
      return fail(LNS_EINVAL, "transmissibilities must be finite and >= 0");

  return LNS_OK;
}
}  // namespace lns

extern "C" {

const char* lns_last_error(void) { return g_err.c_str(); }

int64_t lns_launch_count(void) { return (int64_t)lns::g_launches.load(std::memory_order_relaxed); }

lns_status lns_options_default(lns_options* o) {
  if (!o) return fail(LNS_EINVAL, "options is NULL");
  const double psi = 6894.757293168;
  std::memset(o, 0, sizeof(*o));
  o->mode = LNS_MODE_LOCAL;
  o->eps_p = 0.3 * psi;
  o->eps_sw = 0.0;
  o->m_layers = 2;
  o->tol_dp = 0.3 * psi;
  o->tol_cnv = 1e-6;
  o->max_newton = 25;
  o->max_dd_outer = 25;
  o->sat_chop = 0.2;
  o->krylov_fp32 = 0;
  o->precond = LNS_PRECOND_BJAC;
  o->krylov_rtol = 1e-6;
  o->krylov_maxit = 2000;
  o->krylov_fail_rtol = 1e-3;
  o->p_scale = 0.0;
  o->profile = 0;
  o->fp64_fallback = 1;
  o->krylov_cluster = -1;
  o->autotune = 1;
  o->dd_local_newton = 1;
  o->dd_local_shrink = 0;
  return LNS_OK;
}

lns_status lns_model_create(const lns_model_desc* desc, const lns_options* opts, const lns_allocator* allocator,
                            void* cuda_stream, lns_model** out) {
  if (!desc || !out) return fail(LNS_EINVAL, "desc and out must be non-NULL");
  *out = nullptr;
  TRY(validate_options(opts));
  TRY(lns::validate_desc(desc));
  const int n = desc->n_cells, na = desc->n_adj;
  const lns_fluid& f = desc->fluid;
  lns_model* m = new lns_model();
  m->o = *opts;
  if (allocator && allocator->alloc && allocator->free) {
    m->alloc = *allocator;
    m->has_alloc = true;
  }
  m->stream = (cudaStream_t)cuda_stream;
  auto cleanup_fail = [&](lns_status s) {
    lns_model_destroy(m);
    return s;
  };
  if (cudaGetDevice(&m->device) != cudaSuccess) return cleanup_fail(fail(LNS_ECUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess)
    return cleanup_fail(fail(LNS_ECUDA, "cannot query SM count"));
  m->kgrid[0] = lns::krylov_grid(0, m->sms);
  m->kgrid[1] = lns::krylov_grid(1, m->sms);
  cluster_shape(m, 0, 0);  // function attributes and occupancy queries stay outside stream capture
  m->tune = default_tuning();
  Dev& d = m->d;
  d.n = n;
  d.n_adj = na;
  d.W = (n + 31) / 32;
  d.n_wells = desc->n_wells;
  d.fl = lns::Fluid{f.p_ref, f.c_r, f.b_o_ref, f.c_o, f.b_w_ref, f.c_w, f.rho_o_ref, f.rho_w_ref, f.mu_o, f.mu_w,
                    f.swc, f.sor, f.n_w, f.n_o, f.gravity};
  m->avg_degree = n > 0 ? (double)na / n : 0.0;
  const size_t N = std::max(n, 1), A = std::max(na, 1), W = std::max(d.W, 1), NW = std::max(desc->n_wells, 1);
  lns_status s = LNS_OK;
#define AL(ptr, cnt)                                  \
  do {                                                \
    s = dalloc_t(m, (size_t)(cnt), &ptr);             \
    if (s != LNS_OK) return cleanup_fail(s);          \
  } while (0)
  AL(d.row_ptr, N + 1);
  AL(d.nbr, A);
  AL(d.trans, A);
  AL(d.depth, N);
  AL(d.pv_ref, N);
  AL(d.line_id, N);
  AL(d.well_cell, NW);
  AL(d.well_wi, NW);
  AL(d.well_bhp, NW);
  AL(d.well_of_cell, N);
  AL(d.well_next, NW);
  AL(d.always_list, N);
  AL(d.always, W);
  AL(d.p, N);
  AL(d.sw, N);
  AL(d.pn, N);
  AL(d.swn, N);
  AL(d.p0, N);
  AL(d.sw0, N);
  AL(d.dp, N);
  AL(d.dsw, N);
  AL(d.stamp, N);
  AL(d.va, W);
  AL(d.vb, W);
  AL(d.supp, W);
  AL(d.reach, W);
  AL(d.uni, W);
  AL(d.prev, W);
  AL(d.tmp0, W);
  AL(d.tmp1, W);
  AL(d.tmp2, W);
  AL(d.act, N);
  AL(d.inv, N);
  AL(d.cprops, N * 16);
  AL(d.fr0, N);
  AL(d.fr1, N);
  AL(d.blk_sums, (W + 255) / 256 + 1);
  {
    double* t;
    AL(t, A * 4);
    d.blocks = t;
    AL(d.colA, A);
    AL(t, N * 2);
    d.rhs = t;
    AL(t, N * 4);
    d.line_dinv = t;
    AL(t, N * 4);
    d.line_a = t;
    AL(t, N * 4);
    d.line_g = t;
    AL(d.line_start, N);
    AL(d.line_len, N);
    AL(d.line_cum, N + 1);
    AL(d.lscratch, N);
    AL(d.lblk, W);
    {
      int* t2;
      AL(t2, 2 * N);
      d.lnk = (int2*)t2;
      AL(t2, 2 * N);
      d.arow = (int2*)t2;
      AL(t2, 2 * N);
      d.lsort = (int2*)t2;
    }
    AL(d.line_row_flag, N);
    double** vecs[14] = {(double**)&d.kx,  (double**)&d.kr,   (double**)&d.krh,  (double**)&d.ky0, (double**)&d.ky1,
                         (double**)&d.kv,  (double**)&d.ks,   (double**)&d.kt,   (double**)&d.kz,  (double**)&d.kvt0,
                         (double**)&d.kvt1, (double**)&d.krt, (double**)&d.kzf, (double**)&d.ktt};
    for (auto v : vecs) AL(*v, N * 2);
    AL(d.kls, N * 2);
    {
      float* t3;
      AL(t3, N * 2);
      d.kx0 = t3;
    }
    AL(d.partials, (size_t)8 * 4 * m->sms + 64);
  }
  AL(d.ctr, 1);
  AL(d.stepp, 2);
  AL(d.fault, 1);
#undef AL
  if (cudaMallocHost((void**)&d.ctr_h, sizeof(IterCounters)) != cudaSuccess) {
    d.ctr_h = nullptr;
    return cleanup_fail(fail(LNS_ENOMEM, "cudaMallocHost failed"));
  }
  if (cudaMallocHost((void**)&m->dt_host, 2 * sizeof(double)) != cudaSuccess) {
    m->dt_host = nullptr;
    return cleanup_fail(fail(LNS_ENOMEM, "cudaMallocHost failed"));
  }
  if (cudaMemsetAsync(d.fault, 0, sizeof(int), m->stream) != cudaSuccess)
    return cleanup_fail(fail(LNS_ECUDA, "cannot clear the fault flag"));
  // host-side derived tables
  std::vector<int> woc(N, -1), wnext(NW, -1), alist;
  for (int w = desc->n_wells - 1; w >= 0; w--) {
    wnext[w] = woc[desc->well_cell[w]];
    woc[desc->well_cell[w]] = w;
  }
  std::vector<uint32_t> abits(W, 0u);
  for (int i = 0; i < n; i++)
    if (desc->always_active[i]) {
      abits[i >> 5] |= 1u << (i & 31);
      alist.push_back(i);
    }
  d.n_always = (int)alist.size();
  {
    // The grid solver splits its rows by cost, a fracture-line row counting line_w half rows more
    // than another (its line solve follows its product).  Measured per case on GB300: long lines
    // (mean >= 12 cells: the 2D fracture networks' segments, solved a whole warp per block, few
    // blocks per warp round) are best at 4 in FP32 and 2 in FP64; short ones (the vertical columns
    // of 3D fracture panels, several per warp) at 0 in both, the matrix rows of those sets
    // (scattered cells beside the panels, six or more neighbours each) costing about as much as a
    // line row with its share of the line solves.
    std::vector<int> ids;
    for (int i = 0; i < n; i++)
      if (desc->line_id[i] >= 0) ids.push_back(desc->line_id[i]);
    const size_t cells = ids.size();
    std::sort(ids.begin(), ids.end());
    const size_t lines = (size_t)(std::unique(ids.begin(), ids.end()) - ids.begin());
    const bool long_lines = lines > 0 && cells >= 12 * lines;
    d.line_w[1] = long_lines ? 4 : 0;
    d.line_w[0] = long_lines ? 2 : 0;
  }
  // A 3D row's six neighbours in one gather round trip: the grid solves of the 3D case 6 % faster
  // on GB300; on 2D models (four neighbours) the wider batch executes 4 % more instructions and a
  // solve takes 3.6 % longer, so they keep batches of four.
  d.wide_rows = n > 0 && (long long)na > 5LL * n ? 1 : 0;
  auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0 || !src) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, m->stream);
  };
  cudaError_t e = cudaSuccess;
  e = e ? e : up(d.row_ptr, desc->row_ptr, sizeof(int) * (size_t)(n + 1) * (n > 0));
  e = e ? e : up(d.nbr, desc->nbr, sizeof(int) * (size_t)na);
  e = e ? e : up(d.trans, desc->trans, sizeof(double) * (size_t)na);
  e = e ? e : up(d.depth, desc->depth, sizeof(double) * (size_t)n);
  e = e ? e : up(d.pv_ref, desc->pv_ref, sizeof(double) * (size_t)n);
  e = e ? e : up(d.line_id, desc->line_id, sizeof(int) * (size_t)n);
  e = e ? e : up(d.well_cell, desc->well_cell, sizeof(int) * (size_t)desc->n_wells);
  e = e ? e : up(d.well_wi, desc->well_wi, sizeof(double) * (size_t)desc->n_wells);
  e = e ? e : up(d.well_bhp, desc->well_bhp, sizeof(double) * (size_t)desc->n_wells);
  e = e ? e : up(d.well_of_cell, woc.data(), sizeof(int) * (size_t)n);
  e = e ? e : up(d.well_next, wnext.data(), sizeof(int) * (size_t)desc->n_wells);
  e = e ? e : up(d.always_list, alist.data(), sizeof(int) * alist.size());
  e = e ? e : up(d.always, abits.data(), sizeof(uint32_t) * (size_t)d.W);
  e = e ? e : up(d.p0, desc->p0, sizeof(double) * (size_t)n);
  e = e ? e : up(d.sw0, desc->sw0, sizeof(double) * (size_t)n);
  if (n == 0 && e == cudaSuccess) e = cudaMemsetAsync(d.row_ptr, 0, sizeof(int), m->stream);
  if (e != cudaSuccess) return cleanup_fail(fail(LNS_ECUDA, std::string("upload: ") + cudaGetErrorString(e)));
  apply_cached_tuning(m);
  *out = m;
  lns_status r = lns_reset(m);
  if (r != LNS_OK) {
    *out = nullptr;
    return cleanup_fail(r);
  }
  return LNS_OK;
}

lns_status lns_model_destroy(lns_model* m) {
  if (!m) return LNS_OK;
  cudaStreamSynchronize(m->stream);
  for (void* p : m->owned) {
    if (m->has_alloc)
      m->alloc.free(m->alloc.ctx, p, (void*)m->stream);
    else
      cudaFree(p);
  }
  if (m->d.ctr_h) cudaFreeHost(m->d.ctr_h);
  if (m->dt_host) cudaFreeHost(m->dt_host);
  drop_graph(m);
  for (auto e : m->ev_pool) cudaEventDestroy(e);
  for (auto& pe : m->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  delete m;
  return LNS_OK;
}

lns_status lns_set_options(lns_model* m, const lns_options* o) {
  TRY(check_model(m));
  TRY(validate_options(o));
  if (m->step_open && o->mode != m->o.mode) return fail(LNS_ESTATE, "cannot change mode inside an open timestep");
  m->o = *o;
  drop_graph(m);  // captured with the old options
  cluster_shape(m, 0, 0);
  apply_cached_tuning(m);
  return LNS_OK;
}

lns_status lns_reset(lns_model* m) {
  TRY(check_model(m));
  Dev& d = m->d;
  const size_t nb = sizeof(double) * (size_t)d.n;
  if (d.n > 0) {
    CK(cudaMemcpyAsync(d.p, d.p0, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.sw, d.sw0, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.pn, d.p0, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.swn, d.sw0, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemsetAsync(d.prev, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  }
  m->has_prev = 0;
  m->step_open = false;
  return sync(m);
}

lns_status lns_set_state(lns_model* m, const double* p, const double* sw, const double* pn, const double* swn) {
  TRY(check_model(m));
  if (!p || !sw) return fail(LNS_EINVAL, "p and sw must be non-NULL");
  for (int i = 0; i < m->d.n; i++)
    if (!std::isfinite(p[i]) || !std::isfinite(sw[i]) || (pn && !std::isfinite(pn[i])) || (swn && !std::isfinite(swn[i])))
      return fail(LNS_EINVAL, "non-finite state value (cell " + std::to_string(i) + ")");
  Dev& d = m->d;
  const size_t nb = sizeof(double) * (size_t)d.n;
  if (d.n > 0) {
    CK(cudaMemcpyAsync(d.p, p, nb, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemcpyAsync(d.sw, sw, nb, cudaMemcpyHostToDevice, m->stream));
    if (pn)
      CK(cudaMemcpyAsync(d.pn, pn, nb, cudaMemcpyHostToDevice, m->stream));
    else
      CK(cudaMemcpyAsync(d.pn, d.p, nb, cudaMemcpyDeviceToDevice, m->stream));
    if (swn)
      CK(cudaMemcpyAsync(d.swn, swn, nb, cudaMemcpyHostToDevice, m->stream));
    else
      CK(cudaMemcpyAsync(d.swn, d.sw, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemsetAsync(d.prev, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  }
  m->has_prev = 0;
  m->step_open = false;
  return sync(m);
}

lns_status lns_set_state_device(lns_model* m, const double* p, const double* sw) {
  TRY(check_model(m));
  if (!p || !sw) return fail(LNS_EINVAL, "p and sw must be non-NULL");
  Dev& d = m->d;
  const size_t nb = sizeof(double) * (size_t)d.n;
  if (d.n > 0) {
    CK(cudaMemcpyAsync(d.p, p, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.sw, sw, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.pn, p, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.swn, sw, nb, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemsetAsync(d.prev, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
  }
  m->has_prev = 0;
  m->step_open = false;
  return sync(m);
}

lns_status lns_set_support(lns_model* m, const uint32_t* bits) {
  TRY(check_model(m));
  if (m->step_open) return fail(LNS_ESTATE, "cannot replace the support inside an open timestep");
  if (!bits) {
    if (m->d.W > 0) CK(cudaMemsetAsync(m->d.prev, 0, sizeof(uint32_t) * (size_t)m->d.W, m->stream));
    m->has_prev = 0;
    return sync(m);
  }
  TRY(bits_to_device(m, m->d.prev, bits));
  m->has_prev = 1;
  return sync(m);
}

lns_status lns_debug_fault(lns_model* m, int32_t code) {
  TRY(check_model(m));
  if (code < 0 || code > 4) return fail(LNS_EINVAL, "fault code must be 0..4");
  CK(cudaMemcpyAsync(m->d.fault, &code, sizeof(int), cudaMemcpyHostToDevice, m->stream));
  m->fault_h = code;
  return sync(m);
}

lns_status lns_set_stream(lns_model* m, void* cuda_stream) {
  TRY(check_model(m));
  cudaStream_t to = (cudaStream_t)cuda_stream;
  if (to != m->stream) {  // work queued on the old stream comes first (a device-side dependency)
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, m->stream);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(to, e, 0);
    cudaEventDestroy(e);
    CK(r);
    m->stream = to;
    // a model that moves between streams may run beside other models: its solver launches go
    // through the cross-stream chain, which a captured graph would bypass
    drop_graph(m);
    m->graph_ok = false;
  }
  return LNS_OK;
}

lns_status lns_get_state(const lns_model* cm, double* p, double* sw) {
  lns_model* m = const_cast<lns_model*>(cm);
  TRY(check_model(m));
  const size_t nb = sizeof(double) * (size_t)m->d.n;
  if (m->d.n > 0) {
    if (p) CK(cudaMemcpyAsync(p, m->d.p, nb, cudaMemcpyDeviceToHost, m->stream));
    if (sw) CK(cudaMemcpyAsync(sw, m->d.sw, nb, cudaMemcpyDeviceToHost, m->stream));
  }
  return sync(m);
}

lns_status lns_get_state_device(const lns_model* cm, double* p, double* sw) {
  lns_model* m = const_cast<lns_model*>(cm);
  TRY(check_model(m));
  const size_t nb = sizeof(double) * (size_t)m->d.n;
  if (m->d.n > 0) {
    if (p) CK(cudaMemcpyAsync(p, m->d.p, nb, cudaMemcpyDeviceToDevice, m->stream));
    if (sw) CK(cudaMemcpyAsync(sw, m->d.sw, nb, cudaMemcpyDeviceToDevice, m->stream));
  }
  return sync(m);
}

lns_status lns_get_support(const lns_model* cm, uint32_t* bits) {
  lns_model* m = const_cast<lns_model*>(cm);
  TRY(check_model(m));
  if (!bits) return fail(LNS_EINVAL, "bits is NULL");
  TRY(bits_to_host(m, bits, m->d.prev));
  return sync(m);
}

struct NvtxRange {  // a named range on the profiler's timeline (no-op without a tool attached)
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

lns_status lns_newton_iter(lns_model* m, double dt, lns_iter_stats* out) {
  TRY(check_model(m));
  NvtxRange range("lns_newton_iter");
  if (m->o.mode == LNS_MODE_DD || m->o.mode == LNS_MODE_RESIDUAL)
    return fail(LNS_ESTATE, "lns_newton_iter is not available in LNS_MODE_DD or LNS_MODE_RESIDUAL");
  if (m->d.n == 0) return fail(LNS_EINVAL, "empty model");
  if (!m->step_open) {
    TRY(maybe_autotune(m));
    TRY(open_step(m, dt));
  }
  lns_iter_stats st{};
  lns_status s = alg1_iteration(m, &st);
  if (s != LNS_OK) {
    m->step_open = false;
    if (out) *out = st;
    return s;
  }
  s = after_iteration(m, &st);
  if (out) *out = st;
  return s;
}

lns_status lns_advance(lns_model* m, double t_span, const lns_dt_control* ctl, lns_advance_stats* out) {
  TRY(check_model(m));
  if (out) std::memset(out, 0, sizeof(*out));
  if (m->step_open) return fail(LNS_ESTATE, "a timestep opened by lns_newton_iter is still open");
  if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(LNS_EINVAL, "t_span must be positive and finite");
  lns_dt_control c{t_span, t_span / 1024.0, t_span, 2.0, 0.5, 4};
  if (ctl) c = *ctl;
  if (!(c.dt_init > 0.0) || !(c.dt_min > 0.0) || !(c.dt_max >= c.dt_min) || !(c.grow >= 1.0) || !(c.cut > 0.0) ||
      !(c.cut < 1.0) || !std::isfinite(c.dt_init) || !std::isfinite(c.dt_max) || !std::isfinite(c.grow))
    return fail(LNS_EINVAL, "bad time-step controller");
  Dev& d = m->d;
  const size_t n = (size_t)d.n;
  if (!m->ck_state) TRY(dalloc_t(m, 2 * std::max<size_t>(n, 1), &m->ck_state));
  if (!m->ck_prev) TRY(dalloc_t(m, (size_t)std::max(d.W, 1), &m->ck_prev));
  lns_advance_stats a{};
  double t = 0.0, dt = std::min(c.dt_init, c.dt_max);
  lns_status s = LNS_OK;
  while (t < t_span) {
    const double h = std::min(dt, t_span - t);
    if (n > 0) {
      CK(cudaMemcpyAsync(m->ck_state, d.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(m->ck_state + n, d.sw, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(m->ck_prev, d.prev, sizeof(uint32_t) * (size_t)d.W, cudaMemcpyDeviceToDevice, m->stream));
    }
    const int had_prev = m->has_prev;
    lns_step_stats st{};
    s = lns_timestep(m, h, &st);
    a.iterations += st.iterations;
    a.krylov_iters += st.krylov_iters;
    a.cell_updates += st.cell_updates;
    if (s == LNS_OK) {
      t = (h == t_span - t) ? t_span : t + h;
      a.steps += 1;
      if (st.iterations <= c.easy_iters) dt = std::min(dt * c.grow, c.dt_max);
      continue;
    }
    if (s != LNS_ENOCONV && s != LNS_EKRYLOV) break;
    // undo the failed step
    if (n > 0) {
      CK(cudaMemcpyAsync(d.p, m->ck_state, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(d.sw, m->ck_state + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(d.prev, m->ck_prev, sizeof(uint32_t) * (size_t)d.W, cudaMemcpyDeviceToDevice, m->stream));
    }
    m->has_prev = had_prev;
    a.cuts += 1;
    dt = h * c.cut;
    if (dt < c.dt_min) {
      s = fail(LNS_ENOCONV, "time step fell below dt_min");
      break;
    }
    s = LNS_OK;
  }
  TRY(sync(m));
  a.status = s;
  a.t_done = t;
  a.dt_next = dt;
  if (out) *out = a;
  return s;
}

lns_status lns_batch_advance(lns_model* const* members, int32_t n_members, double t_span, const lns_dt_control* ctl,
                             lns_advance_stats* out, lns_batch_stats* bst) {
  if (bst) std::memset(bst, 0, sizeof(*bst));
  if (n_members < 0 || (n_members > 0 && (!members || !out)))
    return fail(LNS_EINVAL, "members and out must be non-NULL");
  if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(LNS_EINVAL, "t_span must be positive and finite");
  lns_dt_control c{t_span, t_span / 1024.0, t_span, 2.0, 0.5, 4};
  if (ctl) c = *ctl;
  if (!(c.dt_init > 0.0) || !(c.dt_min > 0.0) || !(c.dt_max >= c.dt_min) || !(c.grow >= 1.0) || !(c.cut > 0.0) ||
      !(c.cut < 1.0) || !std::isfinite(c.dt_init) || !std::isfinite(c.dt_max) || !std::isfinite(c.grow))
    return fail(LNS_EINVAL, "bad time-step controller");
  std::vector<lns_model*> ms(members, members + n_members);
  for (int i = 0; i < n_members; i++) {
    TRY(check_model(ms[i]));
    for (int j = 0; j < i; j++)
      if (ms[j] == ms[i]) return fail(LNS_EINVAL, "a model appears twice in the batch");
    if (ms[i]->o.mode != LNS_MODE_LOCAL && ms[i]->o.mode != LNS_MODE_FULL)
      return fail(LNS_EINVAL, "batched advance runs standard Newton or Algorithm 1 only");
    if (ms[i]->step_open) return fail(LNS_ESTATE, "a member has a timestep open");
  }
  struct Member {
    lns_model* m;
    double t, dt, h;
    int had_prev;
    bool live, open;
    lns_advance_stats a;
  };
  std::vector<Member> st(n_members);
  for (int i = 0; i < n_members; i++) {
    lns_model* m = ms[i];
    Dev& d = m->d;
    std::memset(&out[i], 0, sizeof(out[i]));
    st[i] = Member{m, 0.0, std::min(c.dt_init, c.dt_max), 0.0, 0, true, false, lns_advance_stats{}};
    if (d.n == 0) {  // nothing to solve: the plain controller
      lns_status s = lns_advance(m, t_span, &c, &out[i]);
      if (s != LNS_OK) return s;
      st[i].live = false;
      continue;
    }
    const size_t n = (size_t)d.n;
    if (!m->ck_state) TRY(dalloc_t(m, 2 * n, &m->ck_state));
    if (!m->ck_prev) TRY(dalloc_t(m, (size_t)std::max(d.W, 1), &m->ck_prev));
    if (m->o.krylov_fp32 && !d.raw) TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.raw));
    TRY(maybe_autotune(m));
  }
  // the end of a step attempt (lns_advance's controller)
  auto end_step = [&](Member& b, lns_status s) -> lns_status {
    lns_model* m = b.m;
    Dev& d = m->d;
    const size_t n = (size_t)d.n;
    b.a.iterations += m->cur.iterations;
    b.a.krylov_iters += m->cur.krylov_iters;
    b.a.cell_updates += m->cur.cell_updates;
    b.open = false;
    if (s == LNS_OK) {
      b.t = (b.h == t_span - b.t) ? t_span : b.t + b.h;
      b.a.steps += 1;
      if (m->cur.iterations <= c.easy_iters) b.dt = std::min(b.dt * c.grow, c.dt_max);
      if (b.t >= t_span) b.live = false;
      return LNS_OK;
    }
    if (s != LNS_ENOCONV && s != LNS_EKRYLOV) {
      b.a.status = s;
      b.live = false;
      return LNS_OK;
    }
    CK(cudaMemcpyAsync(d.p, m->ck_state, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.sw, m->ck_state + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(d.prev, m->ck_prev, sizeof(uint32_t) * (size_t)d.W, cudaMemcpyDeviceToDevice, m->stream));
    m->has_prev = b.had_prev;
    b.a.cuts += 1;
    b.dt = b.h * c.cut;
    if (b.dt < c.dt_min) {
      b.a.status = LNS_ENOCONV;
      b.live = false;
    }
    return LNS_OK;
  };
  for (;;) {
    std::vector<Member*> live;
    for (auto& b : st)
      if (b.live) live.push_back(&b);
    if (live.empty()) break;
    if (bst) bst->rounds += 1;
    for (Member* b : live) {  // open a step where none is open (checkpoint first, as lns_advance)
      if (b->open) continue;
      lns_model* m = b->m;
      Dev& d = m->d;
      const size_t n = (size_t)d.n;
      b->h = std::min(b->dt, t_span - b->t);
      CK(cudaMemcpyAsync(m->ck_state, d.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(m->ck_state + n, d.sw, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      CK(cudaMemcpyAsync(m->ck_prev, d.prev, sizeof(uint32_t) * (size_t)d.W, cudaMemcpyDeviceToDevice, m->stream));
      b->had_prev = m->has_prev;
      TRY(open_step(m, b->h));
      b->open = true;
    }
    for (Member* b : live) TRY(run_half(b->m, 0));
    for (Member* b : live) CK(cudaStreamSynchronize(b->m->stream));
    for (Member* b : live) {
      lns_model* m = b->m;
      const int which = pick_solver(m);
      if (bst) (which == 1 ? bst->cluster_solves : bst->grid_solves) += 1;
      CK(lns::launch_bicgstab_which(m->d, m->o.krylov_fp32, m->o.precond == LNS_PRECOND_BJAC, m->o.krylov_rtol,
                                    m->o.krylov_maxit, m->kgrid[m->o.krylov_fp32 ? 1 : 0], batch_shape(m), which,
                                    cfg(m)));
      TRY(run_half(m, 1));
    }
    for (Member* b : live) CK(cudaStreamSynchronize(b->m->stream));
    for (Member* b : live) {
      lns_model* m = b->m;
      m->pending.clear();
      lns_status s = finish_iteration(m, nullptr);
      if (s != LNS_OK) {
        m->step_open = false;
        TRY(end_step(*b, s));
        continue;
      }
      s = after_iteration(m, nullptr);
      if (s != LNS_OK || !m->step_open) TRY(end_step(*b, s));
    }
  }
  lns_status first_bad = LNS_OK;
  for (int i = 0; i < n_members; i++) {
    Member& b = st[i];
    if (b.m->d.n == 0) continue;
    TRY(sync(b.m));
    b.a.t_done = b.t;
    b.a.dt_next = b.dt;
    out[i] = b.a;
    if (b.a.status != LNS_OK && first_bad == LNS_OK) first_bad = (lns_status)b.a.status;
  }
  if (first_bad != LNS_OK) return fail(first_bad, "a member of the batch did not complete (see its status)");
  return LNS_OK;
}

int32_t lns_tune_pick(int32_t n, const int32_t* sizes, const double* t_cluster, const double* t_grid) {
  int32_t best = 0;
  for (int32_t k = 0; k < n && sizes && t_cluster && t_grid; k++) {
    if (!(t_cluster[k] >= 0.0) || !(t_cluster[k] < t_grid[k])) break;
    best = sizes[k];
  }
  return best;
}

int32_t lns_tune_cache_lookup(int32_t device, int32_t krylov_fp32, int32_t precond, int32_t n_cells, lns_tuning* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = tune_cache().find(std::make_tuple(device, krylov_fp32 ? 1 : 0, precond, size_class(n_cells)));
  if (it == tune_cache().end()) return 0;
  if (out) *out = it->second;
  return 1;
}

void lns_tune_cache_store(int32_t device, int32_t krylov_fp32, int32_t precond, int32_t n_cells, const lns_tuning* t) {
  if (!t) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache()[std::make_tuple(device, krylov_fp32 ? 1 : 0, precond, size_class(n_cells))] = *t;
}

void lns_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache().clear();
}

lns_status lns_get_tuning(const lns_model* m, lns_tuning* out) {
  TRY(check_model(m));
  if (!out) return fail(LNS_EINVAL, "out is NULL");
  *out = m->tune;
  return LNS_OK;
}

lns_status lns_set_tuning(lns_model* m, const lns_tuning* t) {
  TRY(check_model(m));
  if (!t) {  // back to the cache or the defaults
    m->tune_explicit = false;
    apply_cached_tuning(m);
    drop_graph(m);
    return LNS_OK;
  }
  if ((t->asm_block != 0 && t->asm_block != 64 && t->asm_block != 128 && t->asm_block != 256) ||
      t->asm_blocks_per_sm < 0 || t->asm_blocks_per_sm > 16 || t->set_blocks_per_sm < 0 || t->set_blocks_per_sm > 16)
    return fail(LNS_EINVAL, "asm_block must be 0, 64, 128 or 256 and blocks per SM 0..16");
  m->tune = *t;
  m->tune_explicit = true;
  drop_graph(m);  // captured with the old launch shapes
  return LNS_OK;
}

lns_status lns_autotune(lns_model* m, lns_tuning* out) {
  TRY(check_model(m));
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  Dev& d = m->d;
  lns_tuning best = default_tuning();
  if (d.n == 0) {
    m->tune = best;
    if (out) *out = best;
    return LNS_OK;
  }
  const int fp32 = m->o.krylov_fp32, lines = m->o.precond == LNS_PRECOND_BJAC;
  if (fp32 && !d.raw) TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.raw));
  drop_graph(m);
  const lns_tuning saved = m->tune;
  m->tune = default_tuning();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto timed = [&](auto body, int reps, double* us) -> lns_status {
    double best_us = 1e30;
    for (int r = 0; r < reps; r++) {
      CK(cudaEventRecord(e0, m->stream));
      TRY(body());
      CK(cudaEventRecord(e1, m->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      best_us = std::min(best_us, 1e3 * (double)ms);
    }
    *us = best_us;
    return LNS_OK;
  };
  const int asm_blk[3] = {64, 128, 256}, mults[3] = {2, 4, 8};
  double t_asm[3][3] = {}, t_set[3] = {};
  std::vector<int32_t> sizes;
  std::vector<double> tcl, tgr;
  const lns::ClusterShape cap_shape = cluster_shape(m, fp32, lines);  // its capacity (no threshold yet)
  TRY(set_dt(m, 10.0 * 86400.0));  // a mid-range step of the workloads (0.01-30 days)
  lns_status st = [&]() -> lns_status {
    // the always-active cells (every active set of the model contains them), or the model's initial
    // set when it has none; then 1, 2, 4, ... more rings of neighbours at each step
    if (d.n_always > 0)
      CK(lns::launch_words_op(d, lns::kCopy, d.va, d.always, nullptr, cfg(m)));
    else
      TRY(initial_set(m, d.va));
    for (int k = 0; k < 8; k++) {
      TRY(reset_iter(m));
      CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, cfg(m)));
      TRY(read_counters(m));
      const int nA = d.ctr_h->n_active;
      if (nA == 0) break;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          LaunchCfg c = cfg(m);
          c.asm_block = asm_blk[a];
          c.asm_mult = mults[b];
          double us = 0;
          TRY(timed([&]() -> lns_status {
                CK(lns::launch_assemble(d, eff_p_scale(m), fp32, lines, 0, c));
                return LNS_OK;
              }, 3, &us));
          t_asm[a][b] += us;
        }
      CK(lns::launch_assemble(d, eff_p_scale(m), fp32, lines, 0, cfg(m)));
      if (lines) CK(lns::launch_line_setup(d, fp32, cfg(m)));
      const lns::ClusterShape cl = cap_shape;
      double tc = -1.0, tg = 0.0;
      if (cl.ctas > 0 && nA <= cl.cap)
        TRY(timed([&]() -> lns_status {
              CK(lns::launch_bicgstab_which(d, fp32, lines, m->o.krylov_rtol, m->o.krylov_maxit, m->kgrid[fp32 ? 1 : 0],
                                            cl, 1, cfg(m)));
              return LNS_OK;
            }, 3, &tc));
      TRY(timed([&]() -> lns_status {
            CK(lns::launch_bicgstab_which(d, fp32, lines, m->o.krylov_rtol, m->o.krylov_maxit, m->kgrid[fp32 ? 1 : 0], cl,
                                          2, cfg(m)));
            return LNS_OK;
          }, 3, &tg));
      sizes.push_back(nA);
      tcl.push_back(tc);
      tgr.push_back(tg);
      for (int b = 0; b < 3; b++) {  // update/flag kernel (no state change; seeds the frontier with the
                                     // moved boundary cells, at most n_A) and a two-ring expansion
        LaunchCfg c = cfg(m);
        c.set_mult = mults[b];
        double us = 0;
        TRY(timed([&]() -> lns_status {
              CK(cudaMemsetAsync(d.reach, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
              CK(cudaMemsetAsync(&d.ctr->n_frontier[0], 0, 2 * sizeof(int), m->stream));
              CK(lns::launch_flag(d, d.vb, 0, 0, 0, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop, fp32, d.kx,
                                  -1.0, c));
              CK(lns::launch_dilate(d, d.reach, 2, c));
              return LNS_OK;
            }, 3, &us));
        t_set[b] += us;
      }
      if (nA >= d.n || (cl.ctas > 0 && nA > cl.cap) || (cl.ctas == 0 && k >= 2)) break;
      // next set: this one and its neighbours
      CK(cudaMemsetAsync(d.reach, 0, sizeof(uint32_t) * (size_t)d.W, m->stream));
      CK(cudaMemsetAsync(d.ctr, 0, sizeof(IterCounters), m->stream));
      CK(lns::launch_seed_frontier(d, d.act, nA, d.reach, cfg(m)));
      CK(lns::launch_dilate(d, d.reach, 1 << k, cfg(m)));
      CK(lns::launch_words_op(d, lns::kCopy, d.va, d.reach, nullptr, cfg(m)));
    }
    return LNS_OK;
  }();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LNS_OK) {
    m->tune = saved;
    return st;
  }
  int ba = 0, bb = 1;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      if (t_asm[a][b] < t_asm[ba][bb]) {
        ba = a;
        bb = b;
      }
  int bs = 1;
  for (int b = 0; b < 3; b++)
    if (t_set[b] < t_set[bs]) bs = b;
  best.cluster_max_rows = lns_tune_pick((int32_t)sizes.size(), sizes.data(), tcl.data(), tgr.data());
  best.asm_block = asm_blk[ba];
  best.asm_blocks_per_sm = mults[bb];
  best.set_blocks_per_sm = mults[bs];
  best.measured = 1;
  m->tune = best;
  m->tune_explicit = false;
  lns_tune_cache_store(m->device, fp32, m->o.precond, d.n, &best);
  TRY(sync(m));
  if (out) *out = best;
  return LNS_OK;
}

lns_status lns_timestep(lns_model* m, double dt, lns_step_stats* out) {
  TRY(check_model(m));
  NvtxRange range("lns_timestep");
  if (m->d.n == 0) {
    if (out) std::memset(out, 0, sizeof(*out));
    return LNS_OK;
  }
  if (m->step_open) return fail(LNS_ESTATE, "a timestep opened by lns_newton_iter is still open");
  TRY(maybe_autotune(m));
  if (m->o.mode == LNS_MODE_DD) return dd_timestep(m, dt, out);
  if (m->o.mode == LNS_MODE_RESIDUAL) return residual_timestep(m, dt, out);
  TRY(open_step(m, dt));
  lns_status s = LNS_OK;
  for (;;) {
    lns_iter_stats st{};
    s = lns_newton_iter(m, dt, &st);
    if (s != LNS_OK || st.step_done) break;
  }
  m->cur.status = s;
  if (out) *out = m->cur;
  return s;
}

lns_status lns_active_set(lns_model* m, const double* dp, const double* dsw, int32_t du_on_device, int32_t converged,
                          uint32_t* va_bits, uint32_t* vb_bits, int32_t* is_expand) {
  TRY(check_model(m));
  if (!dp || !va_bits) return fail(LNS_EINVAL, "dp and va_bits must be non-NULL");
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  const size_t nb = sizeof(double) * (size_t)d.n;
  if (d.n == 0) {
    if (is_expand) *is_expand = 0;
    return LNS_OK;
  }
  const cudaMemcpyKind kind = du_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(d.dp, dp, nb, kind, m->stream));
  if (dsw)
    CK(cudaMemcpyAsync(d.dsw, dsw, nb, kind, m->stream));
  else
    CK(cudaMemsetAsync(d.dsw, 0, nb, m->stream));
  TRY(bits_to_device(m, d.va, va_bits));
  TRY(reset_iter(m));
  CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, c));
  CK(lns::launch_boundary(d, d.va, d.vb, c));
  CK(lns::launch_flag(d, d.vb, 0, 0, 0, m->o.eps_p, m->o.eps_sw, 1.0, 0.0, 0, nullptr, -1.0, c));
  TRY(dilate(m, m->o.m_layers));
  // the union accumulator is scratch here
  CK(lns::launch_alg1_combine(d, m->o.tol_dp, m->o.tol_cnv, converged ? 1 : 0, c));
  CK(lns::launch_boundary(d, d.va, d.vb, c));
  TRY(bits_to_host(m, va_bits, d.va));
  if (vb_bits) TRY(bits_to_host(m, vb_bits, d.vb));
  TRY(read_counters(m));
  if (is_expand) *is_expand = d.ctr_h->is_expand;
  return LNS_OK;
}

lns_status lns_dd_expand(lns_model* m, const double* dp, const double* dsw, int32_t du_on_device, const uint32_t* vb_k,
                         uint32_t* vt, uint32_t* va_next, uint32_t* vb_next, uint32_t* vdb_next, int32_t* is_expand) {
  TRY(check_model(m));
  if (!dp || !vb_k || !vt || !va_next) return fail(LNS_EINVAL, "dp, vb_k, vt and va_next must be non-NULL");
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  const size_t nb = sizeof(double) * (size_t)d.n;
  if (d.n == 0) {
    if (is_expand) *is_expand = 0;
    return LNS_OK;
  }
  const cudaMemcpyKind kind = du_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(d.dp, dp, nb, kind, m->stream));
  if (dsw)
    CK(cudaMemcpyAsync(d.dsw, dsw, nb, kind, m->stream));
  else
    CK(cudaMemsetAsync(d.dsw, 0, nb, m->stream));
  TRY(bits_to_device(m, d.tmp1, vb_k));
  TRY(bits_to_device(m, d.tmp2, vt));
  TRY(reset_iter(m));
  // flag the cells of V_B^k: E = {i in V_B^k : |du_i| >= eps}
  CK(lns::launch_compact(d, d.tmp1, d.act, nullptr, &d.ctr->n_active, c));
  CK(lns::launch_flag(d, d.tmp1, 0, 0, 0, m->o.eps_p, m->o.eps_sw, 1.0, 0.0, 0, nullptr, -1.0, c));
  TRY(dilate(m, m->o.m_layers));
  int ie = 0;
  TRY(dd_expand_sets(m, d.tmp2, d.va, d.vb, d.supp, &ie));
  TRY(bits_to_host(m, vt, d.tmp2));
  TRY(bits_to_host(m, va_next, d.va));
  if (vb_next) TRY(bits_to_host(m, vb_next, d.vb));
  if (vdb_next) TRY(bits_to_host(m, vdb_next, d.supp));
  TRY(sync(m));
  if (is_expand) *is_expand = ie;
  return LNS_OK;
}

lns_status lns_solve_local(lns_model* m, double dt, const uint32_t* va_bits, double* dp, double* dsw,
                           lns_iter_stats* out) {
  TRY(check_model(m));
  if (!va_bits) return fail(LNS_EINVAL, "va_bits is NULL");
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  if (!(dt > 0.0)) return fail(LNS_EINVAL, "dt must be positive");
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  if (d.n == 0) return LNS_OK;
  TRY(set_dt(m, dt));
  const size_t nb = sizeof(double) * (size_t)d.n;
  TRY(bits_to_device(m, d.va, va_bits));
  TRY(reset_iter(m));
  TRY(local_solve(m, 0));
  CK(cudaMemsetAsync(d.dp, 0, nb, m->stream));
  CK(cudaMemsetAsync(d.dsw, 0, nb, m->stream));
  CK(lns::launch_flag(d, nullptr, 0, 0, 0, m->o.eps_p, m->o.eps_sw, eff_p_scale(m), m->o.sat_chop, m->o.krylov_fp32,
                      d.kx, -1.0, c));
  if (dp) CK(cudaMemcpyAsync(dp, d.dp, nb, cudaMemcpyDeviceToHost, m->stream));
  if (dsw) CK(cudaMemcpyAsync(dsw, d.dsw, nb, cudaMemcpyDeviceToHost, m->stream));
  TRY(read_counters(m));
  const IterCounters& h = *d.ctr_h;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->n_active = h.n_active;
    out->krylov_iters = h.krylov_iters;
    out->krylov_status = h.krylov_status;
    out->krylov_relres = h.krylov_relres;
    out->max_dp = bits2d(h.max_dp_bits);
    out->max_dsw = bits2d(h.max_dsw_bits);
    out->cnv = bits2d(h.cnv_bits);
    out->krylov_solver = h.krylov_solver;
  }
  return krylov_outcome(m);
}

lns_status lns_compact(lns_model* m, const uint32_t* va_bits, int32_t* act, int32_t* inv, int32_t* n_active) {
  TRY(check_model(m));
  if (!va_bits || !n_active) return fail(LNS_EINVAL, "va_bits and n_active must not be NULL");
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  Dev& d = m->d;
  *n_active = 0;
  if (d.n == 0) return LNS_OK;
  TRY(bits_to_device(m, d.va, va_bits));
  TRY(reset_iter(m));
  CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, cfg(m)));
  TRY(read_counters(m));
  const int na = d.ctr_h->n_active;
  *n_active = na;
  if (act && na > 0) CK(cudaMemcpyAsync(act, d.act, sizeof(int32_t) * (size_t)na, cudaMemcpyDeviceToHost, m->stream));
  if (inv) CK(cudaMemcpyAsync(inv, d.inv, sizeof(int32_t) * (size_t)d.n, cudaMemcpyDeviceToHost, m->stream));
  TRY(sync(m));
  if (inv) {  // the device map is defined on V_A only; report -1 elsewhere
    const std::vector<uint32_t>& w = m->stage;  // V_A as uploaded (bits past n cleared)
    for (int i = 0; i < d.n; i++)
      if (!((w[i >> 5] >> (i & 31)) & 1u)) inv[i] = -1;
  }
  return LNS_OK;
}

lns_status lns_assemble(lns_model* m, double dt, const uint32_t* va_bits, double* F, double* Jd, double* Jo) {
  TRY(check_model(m));
  if (!va_bits) return fail(LNS_EINVAL, "va_bits is NULL");
  if (m->step_open) return fail(LNS_ESTATE, "a timestep is open");
  if (!(dt > 0.0)) return fail(LNS_EINVAL, "dt must be positive");
  Dev& d = m->d;
  LaunchCfg c = cfg(m);
  if (d.n == 0) return LNS_OK;
  if (!d.resid) {
    TRY(dalloc_t(m, (size_t)d.n * 2, &d.resid));
    TRY(dalloc_t(m, (size_t)d.n * 4, &d.dbg_diag));
    TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.dbg_off));
  }
  CK(cudaMemsetAsync(d.resid, 0, sizeof(double) * 2 * (size_t)d.n, m->stream));
  CK(cudaMemsetAsync(d.dbg_diag, 0, sizeof(double) * 4 * (size_t)d.n, m->stream));
  CK(cudaMemsetAsync(d.dbg_off, 0, sizeof(double) * 4 * (size_t)std::max(d.n_adj, 1), m->stream));
  TRY(set_dt(m, dt));
  TRY(bits_to_device(m, d.va, va_bits));
  TRY(reset_iter(m));
  CK(lns::launch_compact(d, d.va, d.act, d.inv, &d.ctr->n_active, c));
  if (m->o.krylov_fp32 && !d.raw) TRY(dalloc_t(m, (size_t)std::max(d.n_adj, 1) * 4, &d.raw));
  CK(lns::launch_assemble(d, eff_p_scale(m), m->o.krylov_fp32, 0, 1, c));
  if (F) CK(cudaMemcpyAsync(F, d.resid, sizeof(double) * 2 * (size_t)d.n, cudaMemcpyDeviceToHost, m->stream));
  if (Jd) CK(cudaMemcpyAsync(Jd, d.dbg_diag, sizeof(double) * 4 * (size_t)d.n, cudaMemcpyDeviceToHost, m->stream));
  if (Jo && d.n_adj > 0)
    CK(cudaMemcpyAsync(Jo, d.dbg_off, sizeof(double) * 4 * (size_t)d.n_adj, cudaMemcpyDeviceToHost, m->stream));
  return sync(m);
}

lns_status lns_kernel_times(const lns_model* m, lns_kernel_time* out, int32_t cap, int32_t* count) {
  TRY(check_model(m));
  int k = 0;
  for (int c = 0; c < KC_COUNT && k < cap; c++) {
    if (!out) break;
    out[k] = m->kt[c];
    std::snprintf(out[k].name, sizeof(out[k].name), "%s", kClassName[c]);
    k++;
  }
  if (count) *count = k;
  return LNS_OK;
}

lns_status lns_reset_kernel_times(lns_model* m) {
  TRY(check_model(m));
  std::memset(m->kt, 0, sizeof(m->kt));
  return LNS_OK;
}

}  // extern "C"
