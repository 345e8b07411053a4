/*
 * lns.h -- C ABI of the GB300 localized Newton solver (liblns.so).
 *
 * The library advances an oil-water fully implicit finite-volume model on a matrix +
 * discrete-fracture-network connection graph by Newton's method, with the localized
 * variants of Jiang, "Localized Nonlinear Solution Strategies for Efficient Simulation
 * of Unconventional Reservoirs" (arXiv 2008.01539):
 *   - standard Newton (Section 4.1),
 *   - localized Newton, Algorithm 1 (Section 4.3),
 *   - adaptive nonlinear domain decomposition, Algorithm 2 (Section 4.4).
 * Every step of a Newton iteration runs in the library's CUDA kernels for sm_103a: the
 * a-priori active-set estimate, compaction of the active cells, masked residual and
 * Jacobian assembly (Appendix A), the BiCGStab solve of J_A du_A = -F_A and the scatter
 * of the update.  For the three-phase black-oil model, the residual and Jacobian assembly and
 * the update with the primary-variable switch are available on caller-owned device arrays
 * (lns_bo_assemble, lns_bo_update).
 *
 * Conventions (all entry points):
 *   - Every call returns lns_status; no exception crosses the ABI.  On failure
 *     lns_last_error() returns a message for the calling thread.
 *   - Array arguments are plain pointers.  They are HOST pointers unless the argument
 *     list says otherwise (a *_on_device flag).  Inputs are read during the call and
 *     not retained; outputs are caller-allocated.
 *   - Units are SI: Pa, m, m^2, m^3, Pa s, s.
 *   - Bitsets are arrays of ceil(n/32) little-endian uint32 words, bit (i & 31) of word
 *     (i >> 5) standing for cell i.
 *   - Work is enqueued on the model's CUDA stream; every call below returns after that
 *     work has completed (it synchronizes the stream).
 *   - A model may be used by one host thread at a time.
 */
#ifndef LNS_H
#define LNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lns_model lns_model; /* opaque, owned by the library */

typedef enum {
  LNS_OK = 0,
  LNS_EINVAL = -1,   /* invalid argument (null pointer, size out of range, bad option) */
  LNS_ENOMEM = -2,   /* device allocation failed */
  LNS_ECUDA = -3,    /* a CUDA runtime call or kernel failed (message in lns_last_error) */
  LNS_ENOCONV = -4,  /* Newton loop reached max_newton (or Algorithm 2 max_dd_outer) */
  LNS_EKRYLOV = -5,  /* BiCGStab broke down or reached krylov_maxit above krylov_fail_rtol */
  LNS_ETIMEOUT = -6, /* a bounded device-side wait gave up (the solver grid barrier, 2 s) */
  LNS_ESTATE = -7    /* call not valid in the model's current state */
} lns_status;

/* LNS_MODE_RESIDUAL: residual-based active sets, the alternative a-priori estimate the paper
 * cites (Section 1, Section 4.2): each iteration evaluates the full-domain residual and solves on
 * the cells whose scaled residual CNV_i = max_l |R_l,i| dt / (PV_i b_l,i) >= tol_cnv, inflated by
 * m_layers of neighbours (an empty unconverged set before convergence keeps the previous set);
 * converged when no cell is unconverged and the last update's max |dp| < tol_dp.  For
 * comparison with Algorithm 1; lns_timestep only. */
enum { LNS_MODE_FULL = 0, LNS_MODE_LOCAL = 1, LNS_MODE_DD = 2, LNS_MODE_RESIDUAL = 3 };
enum {
  LNS_PRECOND_BJAC = 0,     /* block Jacobi whose blocks are single cells and whole fracture segments
                               (block tridiagonal along each segment) */
  LNS_PRECOND_BJAC_CELL = 1 /* block Jacobi with 2x2 single-cell blocks only */
};

/* Fluid and rock.  b_l(p) = b_l_ref (1 + c_l (p - p_ref)) (inverse formation volume
 * factor), rho_l = rho_l_ref b_l, pore volume PV_ref (1 + c_r (p - p_ref)), Corey
 * relative permeabilities k_rw = Se^n_w, k_ro = (1 - Se)^n_o, Se = (Sw - Swc)/(1 - Swc - Sor)
 * clamped to [0, 1], integer exponents 1..8.  (Appendix A reduced to two phases.) */
typedef struct {
  double p_ref, c_r, b_o_ref, c_o, b_w_ref, c_w, rho_o_ref, rho_w_ref, mu_o, mu_w, swc, sor;
  int32_t n_w, n_o;
  double gravity;
} lns_fluid;

/* Model description (Section 5 models; Appendix A TPFA).  The connection graph is CSR:
 * row i lists the neighbours of cell i in ascending order, and every connection is stored
 * at both endpoints with the same transmissibility.  Cells of one fracture segment are
 * numbered consecutively along the segment and carry the same line_id (>= 0; -1 for
 * matrix cells).  always_active marks cells never dropped from the active set (the paper
 * keeps fractures active, Section 5.2.3; wells too).  All arrays are host, copied at create. */
typedef struct {
  int32_t n_cells;
  int32_t n_adj;              /* number of CSR entries (twice the connections) */
  const int32_t* row_ptr;     /* [n_cells + 1] */
  const int32_t* nbr;         /* [n_adj] */
  const double* trans;        /* [n_adj] transmissibility T_ij (m^3) */
  const double* pv_ref;       /* [n_cells] pore volume at p_ref (m^3) */
  const double* depth;        /* [n_cells] cell-centre depth, positive down (m) */
  const int32_t* line_id;     /* [n_cells] fracture segment id or -1 */
  const uint8_t* always_active; /* [n_cells] 0/1 */
  int32_t n_wells;
  const int32_t* well_cell;   /* [n_wells] producer perforation cell */
  const double* well_wi;      /* [n_wells] well index (m^3) */
  const double* well_bhp;     /* [n_wells] bottom-hole pressure (Pa) */
  lns_fluid fluid;
  const double* p0;           /* [n_cells] initial pressure */
  const double* sw0;          /* [n_cells] initial water saturation */
} lns_model_desc;

/* Solver options.  Convergence of an iteration (Section 5: pressure increment; plus the
 * scaled mass residual): max |dp| < tol_dp and CNV = max_{i,l} |R_l,i| dt / (PV_i b_l,i)
 * < tol_cnv over the rows solved.  eps_p / eps_sw: the cutoff epsilon of the support set
 * supp du = {i : |du_i| >= eps} (Section 4.1) on pressure and (if > 0) saturation. */
typedef struct {
  int32_t mode;          /* LNS_MODE_* */
  double eps_p;          /* Pa */
  double eps_sw;         /* <= 0 disables the saturation cutoff */
  int32_t m_layers;      /* m of the neighbour set V_nbr^{i,m} (connection hops) */
  double tol_dp;         /* Pa */
  double tol_cnv;
  int32_t max_newton;    /* iterations per timestep (Algorithm 2: expansion solves) */
  int32_t max_dd_outer;  /* Algorithm 2 outer passes */
  double sat_chop;       /* |dSw| limit per update; <= 0: none */
  int32_t krylov_fp32;   /* 1: BiCGStab and Jacobian blocks in FP32 (inexact Newton) */
  int32_t precond;       /* LNS_PRECOND_* */
  double krylov_rtol;    /* stop when ||r|| <= krylov_rtol ||b|| (scaled system) */
  int32_t krylov_maxit;
  double krylov_fail_rtol; /* at krylov_maxit, fail with LNS_EKRYLOV if ||r||/||b|| is above this */
  double p_scale;        /* pressure unknown scaling for the Krylov norm (1/Pa); <= 0: c_r + c_o */
  int32_t profile;       /* 1: time every kernel class with CUDA events (lns_kernel_times); 2: the
                          * BiCGStab solves only (one event pair per Newton iteration) */
  int32_t fp64_fallback; /* with krylov_fp32: an FP32 solve that breaks down or stops above
                          * krylov_fail_rtol is redone in FP64 within the same Newton iteration
                          * (a failed solve changes neither the state nor V_A).  Default 1. */
  int32_t krylov_cluster; /* local systems small enough for one thread-block cluster (up to 16 SMs,
                           * vectors in distributed shared memory) are solved there, larger ones by
                           * the grid solver over every SM: the largest cluster in CTAs (2, 4, 8 or
                           * 16); 0: the grid solver only; < 0: the default (16).  Default -1. */
  int32_t autotune;       /* 1: the first timestep of a model whose size class has no cached tuning
                           * runs lns_autotune first (a one-time cost per device, precision,
                           * preconditioner and size class); 0: the cache or the defaults.  Default 1. */
  /* Algorithm 2 variants (Section 4.4 after Algorithm 2, and Section 6: solving a subproblem
   * further, exploiting the solution's locality inside a subdomain).  A subdomain visit takes up to
   * dd_local_newton Newton steps on its subdomain (>= 1; default 1, the plain visit), stopping at the
   * first step that passes the convergence test; the outer pass converges when every subdomain it
   * visited passed the test at its first step.  With dd_local_shrink = 1 each step of a visit after
   * the first solves only the support of the previous step's update within the subdomain plus the
   * subdomain's always-active cells (an empty set ends the visit).  Default 0. */
  int32_t dd_local_newton;
  int32_t dd_local_shrink;
} lns_options;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns a
 * device pointer of at least `bytes` bytes (256-byte aligned) or NULL; free releases it.
 * `stream` is the model's stream.  A NULL allocator means cudaMalloc / cudaFree. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} lns_allocator;

typedef struct {
  int32_t n_active;      /* n_A of the iteration just done */
  int32_t is_expand;     /* Algorithm 1 mode after the iteration */
  int32_t converged;     /* convergence test of the iteration */
  int32_t step_done;     /* the timestep closed after this iteration */
  int32_t krylov_iters;
  int32_t krylov_status; /* 0 ok, 1 max iterations, 2 breakdown, 3 grid barrier wait timed out */
  int32_t fp64_retry;    /* 1: the FP32 solve failed and this iteration's solve was redone in FP64
                          * (krylov_iters counts both solves; status/relres are the FP64 solve's) */
  double max_dp, max_dsw, cnv, krylov_relres;
  int32_t krylov_solver; /* solver of the (last) solve: 1 cluster, 2 grid (options.krylov_cluster) */
} lns_iter_stats;

typedef struct {
  int32_t status;        /* lns_status of the step */
  int32_t iterations;    /* Newton iterations (Algorithm 2: local solves) */
  int32_t krylov_iters;  /* summed over iterations */
  int32_t n_subdomains;  /* Algorithm 2: N */
  int32_t dd_outer;      /* Algorithm 2: outer passes */
  int32_t fp64_retries;  /* iterations whose FP32 solve was redone in FP64 (fp64_fallback) */
  int64_t cell_updates;  /* sum of n_A over iterations */
  double last_max_dp, last_cnv;
} lns_step_stats;

typedef struct {
  char name[24];
  int64_t launches;
  double total_ms;       /* summed CUDA-event durations */
  double bytes;          /* algorithmic bytes moved, summed over launches */
  double flops;          /* algorithmic FP64/FP32 flops, summed over launches */
} lns_kernel_time;

/* Default options: Algorithm 1, eps_p = tol_dp = 0.3 psi, m = 2, tol_cnv = 1e-6, FP64, BiCGStab to
 * krylov_rtol = 1e-6 (an inexact Newton step; the Newton loop reaches the same FP64 tolerance). */
lns_status lns_options_default(lns_options* out);

/* Copy the model to the device, set u = (p0, sw0).  cuda_stream: a cudaStream_t to run
 * on (NULL: the legacy default stream).  allocator may be NULL.  The problem statement is
 * Section 4.1: advance F(u^{n+1}) = 0 from u^n. */
lns_status lns_model_create(const lns_model_desc* desc, const lns_options* opts,
                            const lns_allocator* allocator, void* cuda_stream, lns_model** out);
lns_status lns_model_destroy(lns_model* model);
lns_status lns_set_options(lns_model* model, const lns_options* opts);

/* One timestep u^n -> u^{n+1} of size dt (seconds) by the model's mode (Section 4.1;
 * Algorithm 1 or 2).  On LNS_ENOCONV the state is left at the last iterate. */
lns_status lns_timestep(lns_model* model, double dt, lns_step_stats* out);

/* Adaptive time stepping over an interval.  The paper advances with simple time stepping
 * (Section 5); this is the usual controller around lns_timestep: a step that fails to converge
 * (LNS_ENOCONV, or LNS_EKRYLOV from the local solve) is undone -- state and the support set that
 * seeds the next step's active set are restored -- and retried with dt * cut; a step that
 * converges in at most easy_iters Newton iterations lets the next one grow to dt * grow (at most
 * dt_max).  The last step is shortened to end exactly at t_span. */
typedef struct {
  double dt_init;        /* first step (s) */
  double dt_min;         /* give up (LNS_ENOCONV, state at the last accepted step) below this (s) */
  double dt_max;         /* largest step (s) */
  double grow;           /* >= 1 */
  double cut;            /* in (0, 1) */
  int32_t easy_iters;    /* Newton iterations (Algorithm 2: local solves) of an easy step */
} lns_dt_control;

typedef struct {
  int32_t status;        /* lns_status of the call */
  int32_t steps;         /* accepted steps */
  int32_t cuts;          /* failed (undone) steps */
  int32_t iterations;    /* Newton iterations over all steps, failed ones included */
  int64_t krylov_iters;
  int64_t cell_updates;
  double t_done;         /* time advanced (s) */
  double dt_next;        /* the controller's next step (s), for a following call */
} lns_advance_stats;

/* Advance the model by t_span seconds with the controller above.  Errors other than LNS_ENOCONV /
 * LNS_EKRYLOV return at once (the state is then that of the failed step).  ctl NULL: dt_init =
 * t_span, dt_min = t_span / 1024, dt_max = t_span, grow 2, cut 0.5, easy_iters 4. */
lns_status lns_advance(lns_model* model, double t_span, const lns_dt_control* ctl, lns_advance_stats* out);

/* Batched ensembles: many independent models (e.g. DFN realizations of uneven size) advanced
 * together.  The paper advances one model (Section 4.3); this runs its method on every member at
 * once.  Each member keeps its own state, active sets, convergence test and time-step controller
 * (lns_advance's rule with ctl, applied per member: a member whose step fails is cut and retried
 * while the others go on).  A round advances every live member by one Newton iteration: the work
 * before the solve (compaction, assembly, line factors) of all members, then each member's solve
 * and update; the members' work runs on their own streams and overlaps on the device.  Every
 * system the cluster solver can hold goes to it (it occupies up to 16 SMs, so the members' solves
 * run side by side), larger ones to the grid solver, one at a time; so each member ends exactly,
 * bit for bit, as lns_advance(member, t_span, ctl) leaves it alone with the tuning's
 * cluster_max_rows < 0 (every system that fits in the cluster).  Give every member a stream of its
 * own (lns_set_stream) for overlap.
 * Members: standard Newton or Algorithm 1, no timestep open, each model at most once.  out
 * [n_members] gets each member's statistics (status per member); the call returns the first
 * member's failure status, if any, after all members are done. */
typedef struct {
  int32_t rounds;         /* batch Newton rounds */
  int64_t cluster_solves; /* solves run by the cluster solver */
  int64_t grid_solves;    /* solves run by the grid solver */
} lns_batch_stats;
lns_status lns_batch_advance(lns_model* const* members, int32_t n_members, double t_span, const lns_dt_control* ctl,
                             lns_advance_stats* out, lns_batch_stats* stats);

/* One Newton iteration of Algorithm 1 (or standard Newton): opens a timestep of size dt
 * if none is open, runs lines 4-21 once, and closes the timestep once the loop condition
 * (is_expand or not converged) is false.  Not available in LNS_MODE_DD or LNS_MODE_RESIDUAL. */
lns_status lns_newton_iter(lns_model* model, double dt, lns_iter_stats* out);

/* Algorithm 1, lines 8-20 (steps 3-4 of Section 4.3) on a caller-given update: with
 * V_A = va_bits (in) and its boundary V_B, expand V_A by V_nbr^{i,m} of every boundary
 * cell with |du_i| >= eps, or shrink it to supp du_A (fractures/wells kept; an empty
 * support before convergence keeps V_A).  dp, dsw: [n_cells] update (entries outside V_A
 * are ignored), host or device per du_on_device.  Outputs the new V_A (va_bits, in place),
 * its boundary (vb_bits) and is_expand.  Bit-exact: pure integer/compare logic. */
lns_status lns_active_set(lns_model* model, const double* dp, const double* dsw, int32_t du_on_device,
                          int32_t converged, uint32_t* va_bits, uint32_t* vb_bits, int32_t* is_expand);

/* Algorithm 2, lines 8-22: one expansion step of the dynamic partition build.  vb_k is the
 * boundary set of the subdomain just solved, vt the total active set V_T (in/out).
 * Outputs the next subdomain V_A^{k+1} = (union of V_nbr^{i,m}) minus the old V_T, its
 * boundary set V_B^{k+1} = V_B(V_T) intersect V_A^{k+1}, its outer halo V_dB^{k+1}, and
 * is_expand (0 when no boundary update is >= eps or no new cell was reached). */
lns_status lns_dd_expand(lns_model* model, const double* dp, const double* dsw, int32_t du_on_device,
                         const uint32_t* vb_k, uint32_t* vt, uint32_t* va_next, uint32_t* vb_next,
                         uint32_t* vdb_next, int32_t* is_expand);

/* One localized Newton step without changing the state: solve J_A du_A = -F_A
 * (J_A = R_A J R_A^T, Section 4.3) at the current state u over V_A = va_bits, with the
 * time level u^n set by lns_set_state, and return du (dp, dsw: [n_cells] host, zero
 * outside V_A, saturation chop applied). */
lns_status lns_solve_local(lns_model* model, double dt, const uint32_t* va_bits, double* dp, double* dsw,
                           lns_iter_stats* out);

/* Compaction of the active set (step a2 of an iteration; Section 4.3: R_A restricts to V_A, and
 * F_A, J_A = R_A J R_A^T are built directly on the active rows): the ascending list of the cells
 * of V_A = va_bits (host bitset), act [n_A] (host, capacity n_cells; may be NULL), and the inverse
 * map inv [n_cells] (host; may be NULL): inv[act[k]] = k, -1 for cells outside V_A.  *n_active
 * gets n_A.  The compacted system of lns_solve_local and every Newton iteration numbers its rows
 * in this order.  Bit-exact: integer work only. */
lns_status lns_compact(lns_model* model, const uint32_t* va_bits, int32_t* act, int32_t* inv, int32_t* n_active);

/* The residual F_A and Jacobian blocks of the active rows at the current state
 * (Appendix A).  F: [2 n_cells] (oil, water), Jd: [4 n_cells] diagonal blocks,
 * Jo: [4 n_adj] off-diagonal blocks (row i, column nbr[e]); blocks row-major
 * [dRo/dp, dRo/dSw, dRw/dp, dRw/dSw], FP64, unscaled.  Rows outside V_A and blocks of
 * inactive columns are left untouched.  Any output may be NULL. */
lns_status lns_assemble(lns_model* model, double dt, const uint32_t* va_bits, double* F, double* Jd,
                        double* Jo);

/* State transfer (host arrays of n_cells).  set_state sets u and the time level u^n
 * (pn/swn NULL: u^n = u) and forgets the previous timestep's support. */
lns_status lns_get_state(const lns_model* model, double* p, double* sw);
lns_status lns_set_state(lns_model* model, const double* p, const double* sw, const double* pn,
                         const double* swn);
/* Device-to-device variants for device-resident callers (pointers are device memory).
 * set_state_device sets u = (p, sw) and u^n = u, and forgets the support, like lns_set_state. */
lns_status lns_get_state_device(const lns_model* model, double* p, double* sw);
lns_status lns_set_state_device(lns_model* model, const double* p, const double* sw);
/* Replace the previous timestep's support set (host bitset of n_cells bits; NULL: none), e.g.
 * to restore a model saved with lns_get_support/lns_get_state so that its next timestep starts
 * from the same active set as it would have. */
lns_status lns_set_support(lns_model* model, const uint32_t* bits);
/* Failure injection for tests of the device-side error paths (no GPU fault is involved):
 * code 1 makes the solver's first grid barrier miss one block's arrival, so every bounded wait of
 * that barrier runs out (2 s) and the next solve returns LNS_ETIMEOUT with the context intact;
 * code 2 starts BiCGStab with rho = 0, a breakdown (LNS_EKRYLOV); code 3 does so in FP32 solves
 * only (exercises fp64_fallback); code 4 stops FP32 solves after their first iteration as if
 * they had stalled (exercises the FP64 redo that starts from the FP32 iterate); 0 clears it. */
lns_status lns_debug_fault(lns_model* model, int32_t code);
/* Move the model to another CUDA stream (after the work queued on the current one finishes). */
lns_status lns_set_stream(lns_model* model, void* cuda_stream);
/* Return to the initial state (p0, sw0) without host transfers; forget the support. */
lns_status lns_reset(lns_model* model);
/* The previous timestep's support set (the next step's initial active set before the
 * always-active cells are added). */
lns_status lns_get_support(const lns_model* model, uint32_t* bits);

/* ---------------------------------------------------------------------------------------
 * Autotuning.  The paper has no counterpart (its method is independent of the hardware); these
 * choices only change how the kernels are laid out over the GPU, never what they compute:
 *   - cluster_max_rows: local systems of at most this many rows are solved by the thread-block
 *     cluster solver, larger ones by the grid solver (clamped to the cluster solver's capacity;
 *     < 0: its capacity; 0: never).  The two solvers reach the same Krylov tolerance with a
 *     different reduction order, so this choice moves results by rounding only;
 *   - asm_block, asm_blocks_per_sm: block size (64, 128 or 256 threads, two lanes per row) and
 *     blocks per SM of the assembly (0: defaults 64 and 4);
 *   - set_blocks_per_sm: blocks per SM of the update/flag and frontier-expansion kernels
 *     (0: default 4).
 * Launch shapes leave every result bit-identical (each row is computed by its own lanes and every
 * set operation is order-independent).
 *
 * lns_autotune measures on the model's own data and device: it builds active sets of growing size
 * (the always-active cells, then 1, 2, 4, ... more rings of neighbours), assembles each system, and
 * times both solvers and each launch shape with CUDA events; cluster_max_rows is the largest size
 * up to which the cluster solver was faster at every measured size.  It applies the choice to the
 * model, stores it in a process-wide cache keyed by device, Krylov precision, preconditioner and
 * model size class (the bit length of n_cells), and returns it.  Models created later (or given new
 * options) in the same class take the cached choice unless lns_set_tuning set one.  The model's
 * state is not changed; no timestep may be open.  Work runs on the model's stream. */
typedef struct {
  int32_t cluster_max_rows;
  int32_t asm_block;
  int32_t asm_blocks_per_sm;
  int32_t set_blocks_per_sm;
  int32_t measured;       /* 1: chosen by lns_autotune (here or from the cache), 0: defaults or caller's */
} lns_tuning;
lns_status lns_autotune(lns_model* model, lns_tuning* out);
lns_status lns_get_tuning(const lns_model* model, lns_tuning* out);
lns_status lns_set_tuning(lns_model* model, const lns_tuning* tuning);
/* The autotuner's solver rule on its measurements (exported so it can be checked without a GPU):
 * sizes ascending; t_cluster[k] < 0 where the system did not fit the cluster solver.  Returns the
 * largest sizes[k] such that the cluster solver was faster at sizes[0..k], else 0. */
int32_t lns_tune_pick(int32_t n, const int32_t* sizes, const double* t_cluster, const double* t_grid);
/* The cache (exported for the same reason): lookup returns 1 and fills *out when an entry exists. */
int32_t lns_tune_cache_lookup(int32_t device, int32_t krylov_fp32, int32_t precond, int32_t n_cells, lns_tuning* out);
void lns_tune_cache_store(int32_t device, int32_t krylov_fp32, int32_t precond, int32_t n_cells, const lns_tuning* t);
void lns_tune_cache_clear(void);

/* Kernel timing (options.profile = 1 or 2): up to cap entries, *count gets the number. */
lns_status lns_kernel_times(const lns_model* model, lns_kernel_time* out, int32_t cap, int32_t* count);
lns_status lns_reset_kernel_times(lns_model* model);

/* Allocation-free variant of lns_active_set.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- their memory is owned by a host
 * framework's pool or a fixed budget, or they run where cudaMalloc (which may synchronize the
 * whole device) would stall other work -- and therefore cannot create a model.
 *
 * Computes exactly what lns_active_set computes, on the caller's arrays:
 *   row_ptr [n_cells+1], nbr [row_ptr[n_cells]]: the connection graph as in lns_model_desc;
 *   always_bits: bitset of always-active cells, or NULL for none;
 *   dp, dsw [n_cells]: the update (dsw may be NULL: zero); entries outside V_A are ignored;
 *   va_bits (in/out): V_A, replaced by the new V_A;  vb_bits (out): the new V_B.
 * All of these are DEVICE pointers owned by the caller; is_expand is a host pointer.  Work runs
 * on cuda_stream (NULL: legacy default stream) and the call returns after it has finished.
 *
 * The call allocates nothing: its working storage (frontier lists, bitsets, counters; about
 * 8.4 MB for the limit below) is one file-scope __device__ array that every GPU loading the
 * library keeps until the process exits.  Limits: n_cells <= LNS_NOALLOC_MAX_CELLS and
 * m_layers <= LNS_NOALLOC_MAX_LAYERS; larger values return LNS_EINVAL.  The call reads its result
 * flag back and waits for its stream, so it must never be made while a stream is being captured
 * (it then returns LNS_EINVAL).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of the process, so do
 * not use this call on a device after resetting it (cudaDeviceReset) in the same process.  All
 * calls share the array and each clears what it needs, so calls that overlap on the GPU (two
 * streams or two threads on one device) race: serialize them. */
#define LNS_NOALLOC_MAX_CELLS (1 << 20)
#define LNS_NOALLOC_MAX_LAYERS 1024
lns_status lns_active_set_noalloc(int32_t n_cells, const int32_t* row_ptr, const int32_t* nbr,
                                  const uint32_t* always_bits, const double* dp, const double* dsw, double eps_p,
                                  double eps_sw, int32_t m_layers, int32_t converged, uint32_t* va_bits,
                                  uint32_t* vb_bits, int32_t* is_expand, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Serving: many resident models on one GPU.  The paper has no counterpart (its method advances
 * one model); this is the request loop of a deployment that advances many.
 *
 * Requests "advance model k by dt" (lns_server_submit, any thread, any time) are served by
 * `workers` threads, each with its own CUDA stream: a worker takes the oldest queued request
 * whose model is idle and runs lns_timestep on it, so the requests of different models overlap on
 * the device; the requests of one model run in submission order.  Models stay on the device; they
 * are created when first needed and admitted against hbm_budget_bytes (0: no limit) -- when a
 * model does not fit, idle models are evicted least recently used first, their state and support
 * saved to the host and restored exactly on their next request; a model that does not fit even
 * then waits for the running requests, and runs alone if it exceeds the budget by itself.  A request
 * runs lns_advance over its interval (first step dt; a step that does not converge is undone and
 * halved, steps grow back after easy ones, down to dt * dt_min_fraction); a request that fails
 * even there leaves its model unchanged.  Served models send every system that fits to the cluster
 * solver (their tuning's cluster_max_rows < 0), so solves of different models run side by side.
 * Results are the same as those of lns_advance on a model alone with that tuning (the kernels are
 * deterministic).
 * --------------------------------------------------------------------------------------- */
typedef struct lns_server lns_server; /* opaque */

typedef struct {
  int32_t workers;           /* requests run at once (1..64) */
  int64_t hbm_budget_bytes;  /* device bytes the resident models may hold; 0: no limit */
  double dt_min_fraction;    /* a request's steps may be cut down to dt * this; 0: 2^-16 */
} lns_server_options;

typedef struct {
  int64_t request_id;        /* as submitted */
  int32_t model;
  int32_t status;            /* lns_status of the request */
  double dt;
  double t_submit, t_start, t_done;  /* seconds on the server clock (lns_server_now) */
  lns_step_stats stats;      /* summed over the request's steps (failed ones included); dd_outer = cuts */
} lns_completion;

typedef struct {
  int32_t models, resident_models, queued, in_flight;
  int64_t submitted, completed, failed, cancelled, admissions, evictions;
  int64_t resident_bytes;    /* device bytes counted for the resident models */
  int64_t cell_updates;      /* summed over completed requests */
} lns_server_stats;

lns_status lns_server_create(const lns_server_options* options, lns_server** out);
/* Stops the workers after the requests they are running; queued requests are dropped. */
lns_status lns_server_destroy(lns_server* server);
/* Registers a model (arrays copied to the host side of the server; validated now, created on
 * the device at its first request).  opts NULL: lns_options_default. */
lns_status lns_server_add_model(lns_server* server, const lns_model_desc* desc, const lns_options* opts,
                                int32_t* model_id);
lns_status lns_server_submit(lns_server* server, int32_t model_id, double dt, int64_t request_id);
/* Cancel a queued request: it completes at once with status LNS_ESTATE and its model is unchanged.
 * LNS_ESTATE if the request is not queued (unknown, already running or finished). */
lns_status lns_server_cancel(lns_server* server, int64_t request_id);
/* Up to cap completions, waiting up to timeout_s for the first one; *count gets the number. */
lns_status lns_server_poll(lns_server* server, lns_completion* out, int32_t cap, double timeout_s,
                           int32_t* count);
/* Waits until no request is queued or running (LNS_ESTATE after timeout_s). */
lns_status lns_server_drain(lns_server* server, double timeout_s);
/* Fields of an idle model (host arrays of n_cells). */
lns_status lns_server_get_state(lns_server* server, int32_t model_id, double* p, double* sw);
lns_status lns_server_get_stats(lns_server* server, lns_server_stats* out);
double lns_server_now(lns_server* server);

/* ---- Three-phase black-oil physics (the 3D workload's model) -----------------------------------
 * Components water, oil and gas in surface volumes, gas dissolving in oil; Appendix A's
 * backward-Euler TPFA residual with phase-potential upwinding (the lower cell index on a tie):
 *   R_c,i = [M_c(u_i) - M_c(u_i^n)] / dt + sum_j F_c,ij + q_c,i,   c = oil, water, gas
 *   M_o = PV b_o So, M_w = PV b_w Sw, M_g = PV (b_g Sg + Rs b_o So), So = 1 - Sw - Sg;
 *   F_l,ij = T_ij (lambda_l b_l)_up dPhi_l,ij, and the dissolved gas (Rs lambda_o b_o) upwinded
 *   with the oil; dPhi_l,ij = (p_i - p_j) - g (rho_l,i + rho_l,j) / 2 (z_i - z_j);
 *   producers q_c = WI (lambda_c b_c) max(p - BHP, 0), q_g += Rs q_o.
 * Fluid functions: PV = PV_ref (1 + c_r (p - p_ref)), b_w = b_w_ref (1 + c_w (p - p_ref)),
 * b_o = b_o_ref (1 + c_o (p - p_ref)) / (1 + kappa Rs), b_g = b_g_per_pa p, rho_w = rho_w_sc b_w,
 * rho_o = b_o (rho_o_sc + Rs rho_g_sc), rho_g = rho_g_sc b_g, Rs_sat(p) = rs_max p / p_bubble,
 * Corey kr_w((Sw - swc) / span), kr_o((So - sor) / span), kr_g(Sg / span), span = 1 - swc - sor,
 * exponents n_w, n_o, n_g, clamped to [0, 1].  Gas-oil ratios in surface m^3 per surface m^3.
 * Primary variables per cell (p, Sw, X): X = Sg where sat = 1 (free gas; Rs = Rs_sat(p)), X = Rs
 * where sat = 0 (no free gas; Sg = 0).  Section 3.1's variable substitution in black-oil form
 * (after an update): Sg < 0 -> sat = 0, Sg = 0, Rs = Rs_sat(p); Rs > Rs_sat(p) with sat = 0 ->
 * sat = 1, Sg = 0, Rs = Rs_sat(p). */
typedef struct {
  double p_ref, c_r;
  double b_w_ref, c_w, rho_w_sc, mu_w;
  double b_o_ref, c_o, kappa, rho_o_sc, mu_o;
  double b_g_per_pa, rho_g_sc, mu_g;
  double rs_max, p_bubble;
  double swc, sor, gravity;
  int32_t n_w, n_o, n_g;
} lns_bo_fluid;

/* Residual, Jacobian and scaled residual of every cell at the state (p, sw, sg, rs, sat) against
 * the time level (p_old, ...), over the time step dt > 0.  The graph (row_ptr [n_cells+1], nbr and
 * trans [n_adj], pv_ref and depth [n_cells], wells [n_wells]) is the model description's
 * (lns_model_desc); states are [n_cells] (sat: 0 or 1).  Outputs: F [3 n_cells] (oil, water, gas
 * per cell), Jd [9 n_cells] diagonal blocks and Jo [9 n_adj] off-diagonal blocks (row i, column
 * nbr[e]), row-major d(oil, water, gas)/d(p, Sw, X), FP64; cnv [n_cells] = max over components
 * of |R_c| dt / (PV b_c), b of the phase carrying c.  Any output may be NULL.  Every array is a
 * DEVICE pointer owned by the caller (fluid: host).  Work runs on cuda_stream (NULL: legacy
 * default stream); the call returns after it has finished.  LNS_EINVAL on a NULL input, negative
 * sizes, dt <= 0 or a fluid with p_bubble <= 0, swc + sor >= 1 or a Corey exponent < 1; LNS_ECUDA
 * if the kernel fails. */
lns_status lns_bo_assemble(const lns_bo_fluid* fluid, int32_t n_cells, const int32_t* row_ptr, const int32_t* nbr,
                           const double* trans, const double* pv_ref, const double* depth, int32_t n_wells,
                           const int32_t* well_cell, const double* well_wi, const double* well_bhp,
                           const double* p, const double* sw, const double* sg, const double* rs,
                           const uint8_t* sat, const double* p_old, const double* sw_old, const double* sg_old,
                           const double* rs_old, const uint8_t* sat_old, double dt, double* F, double* Jd,
                           double* Jo, double* cnv, void* cuda_stream);

/* u <- u + du on the cells of va_bits (device bitset; NULL: every cell), du [3 n_cells] in
 * (p, Sw, X) per cell, with the saturation chop (|dSw|, and |dSg| where sat = 1, at most sat_chop
 * when sat_chop > 0) and then the variable switch above.  switched [n_cells] (may be NULL) gets 1
 * where a cell's variable set changed, else 0.  Every array is a DEVICE pointer owned by the
 * caller (fluid: host); stream and errors as lns_bo_assemble. */
lns_status lns_bo_update(const lns_bo_fluid* fluid, int32_t n_cells, double sat_chop, const double* du,
                         const uint32_t* va_bits, double* p, double* sw, double* sg, double* rs, uint8_t* sat,
                         uint8_t* switched, void* cuda_stream);

/* Number of CUDA kernels the library has launched in this process (all models). */
int64_t lns_launch_count(void);

/* Message of the last failed call on this thread ("" if none). */
const char* lns_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LNS_H */
