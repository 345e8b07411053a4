/*
 * lns_oracle.h -- CPU FP64 oracle for the localized fully implicit Newton solver
 * (Jiang, "Localized Nonlinear Solution Strategies for Efficient Simulation of
 * Unconventional Reservoirs", arXiv 2008.01539).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may call it; the
 * library's product path never links or loads it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Everything is plain, serial, double precision, written for a reader who checks
 * it against the paper by eye:
 *   - Appendix A: backward-Euler TPFA finite-volume residual with
 *     phase-potential upwinding, reduced to oil-water (two phases, no
 *     capillarity, no mass exchange between phases).
 *   - Section 4.1: Newton's method J du = -F, support set supp du = {i : |du_i| >= eps}.
 *   - Section 4.3, Algorithm 1: localized Newton (expand / shrink active set).
 *   - Section 4.4, Algorithm 2: adaptive nonlinear domain decomposition.
 *   - Section 1 / Section 4.2: the residual-based active set the paper compares against
 *     (unconverged cells plus layers of neighbours), as mode 3.
 * The linear step is a hand-written block sparse LU (nested-dissection ordering,
 * symbolic factorization by elimination tree, row-by-row Doolittle elimination
 * with 2x2 block pivots), or on request BiCGStab with a block ILU(0) preconditioner
 * (for models too large for the LU; the CPU baseline of the million-cell case).
 *
 * Parity pins (tests/test_oracle_pins.py): closed-form erfc solution for 1D
 * slightly compressible flow into a constant-pressure fracture; cumulative mass
 * balance; central-difference Jacobian; dense LU on small systems; brute-force
 * graph distances for the neighbour sets; hydrostatic column; special cases of
 * Algorithms 1 and 2; for mode 3 (tests/test_oracle_residual_sets.py) the first set against
 * scipy graph distances from the unconverged cells, full inflation against standard Newton's
 * iterates, an equilibrium, and the converged fields against standard Newton.
 * Two-phase terms (tests/test_oracle_two_phase_pins.py): face fluxes at interior saturations
 * against Corey relative permeabilities written out as fractions (fractional-flow ratio,
 * endpoints, saturation-independent total flux for linear Corey); the scaled residual (CNV) of
 * a pure-accumulation cell equals its saturation change, plus a worked example.  Planted
 * mistakes in those terms (tests/test_oracle_mutants.py) each fail one of these pins.
 */
#ifndef LNS_ORACLE_H
#define LNS_ORACLE_H
#include <stdint.h>

typedef struct {
  double p_ref, c_r, b_o_ref, c_o, b_w_ref, c_w, rho_o_ref, rho_w_ref, mu_o, mu_w, swc, sor;
  int32_t n_w, n_o;
  double gravity;
} orc_fluid;

typedef struct {
  int32_t n, n_adj;
  const int32_t* row_ptr;   /* [n+1] */
  const int32_t* nbr;       /* [n_adj] */
  const double* trans;      /* [n_adj] */
  const double* pv_ref;     /* [n] */
  const double* depth;      /* [n] */
  const uint8_t* always;    /* [n] cells never dropped from the active set */
  int32_t n_wells;
  const int32_t* well_cell;
  const double* well_wi;
  const double* well_bhp;
  orc_fluid fl;
} orc_model;

typedef struct {
  int32_t mode;        /* 0 full Newton, 1 Algorithm 1, 2 Algorithm 2, 3 residual-based sets */
  double eps_p;        /* cutoff on |dp| (Pa) */
  double eps_sw;       /* cutoff on |dSw|; <= 0 disables */
  int32_t m_layers;    /* m of the neighbour set */
  double tol_dp;       /* convergence: max |dp| < tol_dp ... */
  double tol_cnv;      /* ... and CNV < tol_cnv */
  int32_t max_newton;
  double sat_chop;     /* |dSw| limit per update (<= 0: none) */
  int32_t max_dd_outer;
  /* Algorithm 2 variants (the paper's Section 4.4 closing remarks and Section 6): a subdomain
   * visit takes up to dd_local_newton Newton steps on its subdomain, stopping at local convergence
   * (1: the plain one-step visit); with dd_local_shrink, each step after the first solves only the
   * support of the previous step's update within the subdomain, plus its always-active cells. */
  int32_t dd_local_newton;
  int32_t dd_local_shrink;
  /* linear step: 0 the block sparse LU (default), 1 BiCGStab preconditioned by block ILU(0) in the
   * natural (ascending cell) order, stopped at ||r|| <= lin_rtol ||b|| or lin_maxit iterations */
  int32_t linear;
  double lin_rtol;
  int32_t lin_maxit;
} orc_opts;

typedef struct {
  int32_t status;          /* 0 ok, -4 no convergence */
  int32_t iterations;      /* Newton iterations (inner local solves for Algorithm 2) */
  int64_t cell_updates;    /* sum over iterations of the active-set size */
  int32_t n_subdomains;    /* Algorithm 2: N */
  int32_t dd_outer;        /* Algorithm 2: outer passes */
  double last_max_dp, last_cnv;
} orc_step_stats;

#ifdef __cplusplus
extern "C" {
#endif

/* Full-domain residual F[2n] (oil, water per cell) and Jacobian: diagonal blocks
 * Jd[4n] and off-diagonal blocks Jo[4 n_adj] (row i, column nbr[e]); blocks are
 * row-major [dRo/dp, dRo/dSw, dRw/dp, dRw/dSw].  Any output pointer may be NULL. */
void orc_assemble(const orc_model* m, const double* p, const double* sw, const double* pn,
                  const double* swn, double dt, double* F, double* Jd, double* Jo);

/* CNV_i = max_l |R_l,i| dt / (PV_i b_l,i) per cell. */
void orc_cnv(const orc_model* m, const double* p, const double* F, double dt, double* cnv);

/* Solve the block system A x = rhs (2x2 blocks, structurally symmetric pattern given by
 * row_ptr/col without the diagonal).  Returns 0, or -1 on a singular pivot. *fill gets
 * the number of stored off-diagonal blocks of L+U. */
/* BiCGStab on the block system (diag, off as for orc_lu_solve), right-preconditioned by block
 * ILU(0) (no fill beyond the pattern of the matrix; rows eliminated in index order).  Returns 0 on
 * convergence, 1 at maxit, 2 on breakdown or a singular pivot; *iters gets the iterations. */
int orc_ilu0_bicgstab(int32_t nb, const int32_t* row_ptr, const int32_t* col, const double* diag,
                      const double* off, const double* rhs, double* x, double rtol, int32_t maxit, int32_t* iters);
int orc_lu_solve(int32_t nb, const int32_t* row_ptr, const int32_t* col, const double* diag,
                 const double* off, const double* rhs, double* x, int64_t* fill);

/* Set logic on byte masks of length n. */
void orc_dilate(const orc_model* m, const uint8_t* seed, int32_t layers, uint8_t* out);
void orc_boundary(const orc_model* m, const uint8_t* va, uint8_t* vb);
void orc_outer_halo(const orc_model* m, const uint8_t* va, uint8_t* vdb);

/* Algorithm 1, steps 3-4, on a given update (dp, dsw over all cells; entries outside
 * va are ignored).  va is updated in place; vb gets the boundary of the new set. */
void orc_active_set_update(const orc_model* m, const orc_opts* o, uint8_t* va, const double* dp,
                           const double* dsw, int32_t converged, uint8_t* vb, int32_t* is_expand);

/* Algorithm 2, lines 8-22: one expansion step.  vt (in/out) is the total active set,
 * vb_k the boundary set of the subdomain just solved.  Outputs the next subdomain
 * va_next, its boundary set vb_next and its outer halo vdb_next, and is_expand. */
void orc_dd_expand(const orc_model* m, const orc_opts* o, const uint8_t* vb_k, const double* dp,
                   const double* dsw, uint8_t* vt, uint8_t* va_next, uint8_t* vb_next,
                   uint8_t* vdb_next, int32_t* is_expand);

/* One Newton step restricted to va (J_A du_A = -F_A, Section 4.3): returns du (zero
 * outside va, saturation chop applied), the maximum CNV over va at the input state and
 * the maximum |dp| over va.  Returns 0 or -1 on a singular pivot. */
int orc_local_solve(const orc_model* m, const orc_opts* o, const double* p, const double* sw,
                    const double* pn, const double* swn, double dt, const uint8_t* va,
                    double* dp, double* dsw, double* cnv_max, double* dp_max);

/* Simulation state: p, sw (in/out), the previous timestep's support (in/out, byte mask)
 * and whether a previous step exists.  One timestep u^n -> u^{n+1} by the chosen mode.
 * trace (optional, may be NULL): per iteration the active-set size, written up to
 * trace_cap entries.  union_out (optional): union of the sets solved during the step. */
int orc_timestep(const orc_model* m, const orc_opts* o, double* p, double* sw, uint8_t* prev_supp,
                 int32_t* has_prev, double dt, orc_step_stats* st, int32_t* trace, int32_t trace_cap,
                 uint8_t* union_out);

/* The initial active set of a timestep (Section 4.3 and Section 5.2): the previous
 * timestep's support united with the always-active cells, or on the first step the
 * always-active cells and their m-layer neighbours. */
void orc_initial_set(const orc_model* m, const orc_opts* o, const uint8_t* prev_supp,
                     int32_t has_prev, uint8_t* va);

#ifdef __cplusplus
}
#endif
#endif
