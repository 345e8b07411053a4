// lns_internal.cuh -- device data layout and kernel launchers of liblns (sm_103a).
//
// Layout in HBM (n cells, E2 = CSR entries, W = ceil(n/32) bitset words):
//   static graph : row_ptr[n+1], nbr[E2] (int32), trans[E2] (f64), depth/pv_ref[n] (f64),
//                  line_id[n] (int32), always bitset[W], well table
//   state        : p, sw (iterate u^nu), pn, swn (time level u^n), p0, sw0 (initial), f64[n]
//   sets         : va, vb, supp, reach, step union, previous-step support  (bitsets[W])
//   compaction   : act[n] ascending active cells, inv[n] cell -> compact row (valid where
//                  va is set), frontier lists fr0/fr1[n]; cprops[n][2][8] phase properties of
//                  the active rows (f64)
//   system       : blocks[E2] 2x2 off-diagonal blocks stored at the CSR entry of their
//                  row (f64 or f32), colA[E2] compact column or -1, rhs[2n]; the diagonal
//                  blocks are scaled to the identity and not stored
//   Krylov       : x, r, rhat, y[2], v, s, t, z, v~[2], r~, z~, t~ [2n] (f64 or f32), partial sums
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lns.h"

namespace lns {

constexpr int kMaxLinesPerRow = 1;
// Fracture lines are cut into preconditioner blocks of at most this many rows (a multiple of 32:
// one warp holds a block in registers, 32 rows per chunk).
#ifndef LNS_LINE_BLOCK_ROWS
#define LNS_LINE_BLOCK_ROWS 128
#endif
constexpr int kLineBlockRows = LNS_LINE_BLOCK_ROWS;
static_assert(kLineBlockRows % 32 == 0 && kLineBlockRows >= 32, "line blocks are whole 32-row chunks");

struct Fluid {
  double p_ref, c_r, b_o_ref, c_o, b_w_ref, c_w, rho_o_ref, rho_w_ref, mu_o, mu_w, swc, sor;
  int n_w, n_o;
  double gravity;
};

// Device scalars written by kernels and read back to the host once per iteration.
struct IterCounters {
  int n_active;        // compaction output
  int n_frontier[2];   // frontier list sizes (ping-pong)
  int any_e;           // some boundary cell had a non-negligible update
  int any_s;           // the support of du_A is non-empty
  int any_new;         // Algorithm 2: the next subdomain is non-empty
  int n_lines;         // fracture line blocks in the compacted system (after cutting long lines)
  int n_line_starts;   // fracture lines found by the marking pass (before cutting)
  int krylov_iters;
  int krylov_status;   // 0 ok, 1 maxit, 2 breakdown, 3 grid barrier wait timed out
  int converged;
  int is_expand;
  int halo_flag;       // Algorithm 2 halo test result
  unsigned long long max_dp_bits;   // max |dp| as the bit pattern of a non-negative double
  unsigned long long max_dsw_bits;
  unsigned long long cnv_bits;
  double krylov_relres;
  unsigned bar_count;  // grid barrier of the Krylov kernel (its top bit flips at each barrier)
  unsigned bar_pad;
  int bar_timeout;     // set when a barrier wait gave up (the kernel then stops)
  int solve_failed;    // the update kernel found the Krylov solve failed and applied nothing
  int krylov_solver;   // which solver ran the last solve: 1 cluster, 2 grid
  int pad_i;
  double pad[1];
};

struct Dev {
  int n, n_adj, W, n_wells, n_always;
  Fluid fl;
  // static graph
  int *row_ptr, *nbr, *line_id, *well_cell, *well_of_cell, *well_next, *always_list;
  double *trans, *depth, *pv_ref, *well_wi, *well_bhp;
  uint32_t* always;
  // state
  double *p, *sw, *pn, *swn, *p0, *sw0, *dp, *dsw;
  int* stamp;  // Algorithm 2: solve id of the last non-negligible update of each cell
  // sets
  uint32_t *va, *vb, *supp, *reach, *uni, *prev, *tmp0, *tmp1, *tmp2;
  // compaction
  int *act, *inv, *fr0, *fr1, *blk_sums;
  // per compact row and phase, FP64 properties of the current iterate (8 doubles: b, rho,
  // lambda b, db/dp, drho/dp, d(lambda b)/dp, d(lambda b)/dSw, unused), written once per iteration
  // before the assembly reads them for the row itself and for its active neighbours
  double* cprops;
  // system
  void* blocks;  // E2 * 4 * sizeof(T)
  double* raw;   // E2 * 4: unscaled FP64 blocks (FP32 path only; the FP64 path scales in place)
  int* colA;
  void* rhs;     // 2n * sizeof(T)
  double* resid; // 2n (diagnostics), f64
  double* dbg_diag;  // 4n (diagnostics), f64
  double* dbg_off;   // 4 E2 (diagnostics), f64
  // fracture-line blocks of the preconditioner (per compact row, T)
  void *line_dinv, *line_a, *line_g;
  // line_start: the marking pass's line starts (any order), then the ascending list of line-block
  // starts (after cutting); line_len[k]: rows of the line block starting at compact row k;
  // lblk: bitset of line-block starts; lscratch: compaction scratch; line_cum[l]: rows of the line
  // blocks before block l of the ascending list (l = 0 .. n_lines)
  int *line_start, *line_len, *line_row_flag, *lscratch, *line_cum;
  int2* lsort;  // the grid solver's line blocks listed by length class, per chunk at its blocks' range
  // extra cost of a fracture-line row in the grid solver's row split, in half rows, for FP64 [0] and
  // FP32 [1] solves (chosen per model from its fracture lines' mean length)
  int line_w[2];
  // 1: the grid solver's FP32 products gather 6 neighbours of a row per round trip (models whose
  // cells have more than 5 neighbours on average, the 3D ones), else 4
  int wide_rows;
  int2* lnk;  // per compact row: CSR entries of its couplings to the previous / next row of its line (-1)
  int2* arow;  // per compact row: first CSR entry, and degree | line flag << 24 (written by the assembly)
  uint32_t* lblk;
  // Krylov vectors
  void *kx, *kr, *krh, *ky0, *ky1, *kv, *ks, *kt, *kz, *kvt0, *kvt1, *krt, *kzf, *ktt;
  double* kls;  // 2n: line-solve inputs of chunks too long for shared memory
  // the FP32 iterate of a failed solve (float2 per compact row), which the FP64 redo starts from
  // when krylov_warm is set (0: every solve starts from x = 0)
  void* kx0;
  int krylov_warm;
  double* partials;
  IterCounters* ctr;   // device
  IterCounters* ctr_h; // pinned host mirror
  double* stepp;       // device [2]: dt and 1/dt of the current solve (read by the assembly, so a
                       // captured Newton iteration needs no parameter change between timesteps)
  int* fault;          // device: injected fault of the solver for failure tests (0: none)
};

// Process-wide count of kernels launched by the library (lns_launch_count).
void count_launches(int k);
// Message returned by lns_last_error() on the calling thread.
void set_last_error(const char* msg);
// Host checks of a model description and of options (lns_model_create runs them first).
lns_status validate_desc(const lns_model_desc* desc);
lns_status validate_opts(const lns_options* o);

// ---- launchers (defined in the .cu files) ----
struct LaunchCfg {
  int sms;
  cudaStream_t stream;
  // launch shapes chosen by the autotuner (0: the defaults); results do not depend on them
  int asm_block = 0;  // assembly threads per block (64, 128, 256)
  int asm_mult = 0;   // assembly blocks per SM
  int set_mult = 0;   // blocks per SM of the update/flag and frontier-expansion kernels
};

// k_sets.cu
cudaError_t launch_compact(const Dev& d, const uint32_t* bits, int* list, int* inv, int* count_out,
                           LaunchCfg c);
cudaError_t launch_boundary(const Dev& d, const uint32_t* set, uint32_t* out, LaunchCfg c);
cudaError_t launch_outer_halo(const Dev& d, const uint32_t* set, const int* list, const int* count,
                              uint32_t* out, LaunchCfg c);
cudaError_t launch_flag(const Dev& d, const uint32_t* vb, int apply, int record_stamp, int solve_id,
                        double eps_p, double eps_sw, double p_scale, double sat_chop, int fp32,
                        const void* x, double fail_rtol, LaunchCfg c);
cudaError_t launch_dilate(const Dev& d, uint32_t* reach, int layers, LaunchCfg c);
cudaError_t launch_seed_frontier(const Dev& d, const int* list, int count_host, uint32_t* reach,
                                 LaunchCfg c);
cudaError_t launch_alg1_combine(const Dev& d, double tol_dp, double tol_cnv, int converged_override,
                                LaunchCfg c);
cudaError_t launch_dd_combine(const Dev& d, const uint32_t* reach, uint32_t* vt, uint32_t* va_next,
                              LaunchCfg c);
cudaError_t launch_words_op(const Dev& d, int op, uint32_t* out, const uint32_t* a, const uint32_t* b,
                            LaunchCfg c);
cudaError_t launch_step_support(const Dev& d, double eps_p, double eps_sw, LaunchCfg c);
cudaError_t launch_halo_check(const Dev& d, const uint32_t* vdb, int since, LaunchCfg c);

enum WordsOp { kCopy = 0, kOr = 1, kAnd = 2, kAndNot = 3, kAll = 5 };

// k_assemble.cu
cudaError_t launch_assemble(const Dev& d, double p_scale, int fp32, int lines, int debug, LaunchCfg c);
cudaError_t launch_line_setup(const Dev& d, int fp32, LaunchCfg c);

// k_krylov.cu
cudaError_t launch_residual_flags(const Dev& d, double tol_cnv, LaunchCfg c);
// Cluster solver shape: ctas per cluster (0: none) and the largest n_A it takes (-1: none).
struct ClusterShape {
  int ctas, cap;
};
cudaError_t launch_bicgstab(const Dev& d, int fp32, int lines, double rtol, int maxit, int grid, ClusterShape cl,
                            LaunchCfg c);
cudaError_t launch_bicgstab_which(const Dev& d, int fp32, int lines, double rtol, int maxit, int grid, ClusterShape cl,
                                  int which, LaunchCfg c);
int krylov_grid(int fp32, int sms);
// The largest cluster (<= max_ctas, a power of two) the device co-schedules for the cluster solver.
ClusterShape krylov_cluster_shape(int fp32, int lines, int max_ctas);

}  // namespace lns
