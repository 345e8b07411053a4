// k_assemble.cu -- masked residual and Jacobian assembly of the active rows, and the
// factorization of the fracture-line blocks of the preconditioner.
//
// Residual (Appendix A, two phases, no capillarity), cell i, phase l (0 oil, 1 water):
//   R_l,i = [M_l(u_i) - M_l(u_i^n)] / dt + sum_j T_ij (lambda_l b_l)_up dPhi_l,ij + q_l,i
//   dPhi_l,ij = (p_i - p_j) - g rho_l,ij (z_i - z_j),  rho_l,ij = (rho_l,i + rho_l,j) / 2,
//   phase-potential upwinding (tie: the smaller cell index), producer q = WI lambda b max(p - BHP, 0).
// Only the rows of V_A are assembled; their columns outside V_A are dropped, so inactive
// cells act as Dirichlet values (J_A = R_A J R_A^T, Section 4.3).
//
// Each row is written already multiplied by S D_i^{-1} (D_i its diagonal block,
// S = diag(p_scale, 1)), i.e. block-Jacobi left scaling fused into the assembly epilogue:
// the stored diagonal is the identity and is not stored.  The unknowns are
// (p_scale dp, dSw).  All residual, flux and accumulation arithmetic is FP64; the scaled
// blocks and right-hand side are stored in T (FP64, or FP32 for the inexact-Newton path).
//
// Mapping: a pass over the active rows evaluates each row's phase properties once (k_cell_props,
// two lanes per row); the assembly then takes a lane pair per active row, one lane per phase, and
// reads the properties of the row and of its active neighbours from that pass -- only an inactive
// neighbour (a Dirichlet value) is evaluated in place.  FP64 issues at a small fraction of the FP32
// rate on this GPU, so the FP64 instruction chain of a row is what bounds the kernel.  The boundary
// set V_B of the solved set (rows with an inactive neighbour) falls out of the column scan and is
// written here too.
#include <cuda_runtime.h>

#include <algorithm>

#include "lns_internal.cuh"

namespace lns {

namespace {

constexpr int kAsmBlk = 64;  // small blocks spread the few thousand active rows over all SMs

struct FluidK {
  Fluid f;
  double inv_span, inv_mu[2];
};

__device__ __forceinline__ double ipow(double x, int k) {
  double r = 1.0;
  for (int t = 0; t < k; t++) r *= x;
  return r;
}

__device__ __forceinline__ bool bit(const uint32_t* s, int i) { return (s[i >> 5] >> (i & 31)) & 1u; }

template <typename T>
struct alignas(4 * sizeof(T)) Blk4 {
  T a, b, c, d;
};

// Properties of one phase l of a cell and their derivatives, FP64.  (The Jacobian stays FP64 until
// it is scaled: the diagonal of a pressure row nearly cancels against its off-diagonals, so
// rounding them separately to FP32 would erase the accumulation term.)
struct PhaseProps {
  double b, rho, mob, db, drho, dmob_dp, dmob_ds;
};

__device__ __forceinline__ PhaseProps phase_props(const FluidK& F, double p, double sw, int l) {
  const Fluid& f = F.f;
  const double dpr = p - f.p_ref;
  const double bref = l ? f.b_w_ref : f.b_o_ref, c = l ? f.c_w : f.c_o, rref = l ? f.rho_w_ref : f.rho_o_ref;
  PhaseProps q;
  q.b = bref * (1.0 + c * dpr);
  const double db = bref * c;
  q.rho = rref * q.b;
  q.db = db;
  q.drho = rref * db;
  double se = (sw - f.swc) * F.inv_span, dse = F.inv_span;
  if (se <= 0.0) {
    se = 0.0;
    dse = 0.0;
  } else if (se >= 1.0) {
    se = 1.0;
    dse = 0.0;
  }
  const int n = l ? f.n_w : f.n_o;
  const double x = l ? se : 1.0 - se;  // k_rw = Se^n_w, k_ro = (1 - Se)^n_o
  const double kr = ipow(x, n), dkr = (double)n * ipow(x, n - 1) * (l ? dse : -dse);
  const double im = F.inv_mu[l];
  q.mob = kr * im * q.b;
  q.dmob_dp = kr * im * db;
  q.dmob_ds = dkr * im * q.b;
  return q;
}

// Phase properties of every active row, once per iteration: lane pair per row, lane l = phase l.
// The assembly reads them for the row itself and for each active neighbour, instead of evaluating
// them again per connection (a cell's properties would otherwise be computed 1 + degree times).
__global__ void __launch_bounds__(128) k_cell_props(Dev d, FluidK F) {
  const int nA = d.ctr->n_active;
  const int l = threadIdx.x & 1;
  const int pairs = (gridDim.x * blockDim.x) >> 1;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 1; k < nA; k += pairs) {
    const int i = d.act[k];
    const PhaseProps q = phase_props(F, d.p[i], d.sw[i], l);
    double4_32a* o = (double4_32a*)(d.cprops + 16 * (size_t)k + 8 * l);
    o[0] = make_double4_32a(q.b, q.rho, q.mob, q.db);
    o[1] = make_double4_32a(q.drho, q.dmob_dp, q.dmob_ds, 0.0);
  }
}

__device__ __forceinline__ PhaseProps load_props(const double* cprops, int k, int l) {
  const double4_32a* o = (const double4_32a*)(cprops + 16 * (size_t)k + 8 * l);
  const double4_32a a = o[0], b = o[1];
  PhaseProps q;
  q.b = a.x;
  q.rho = a.y;
  q.mob = a.z;
  q.db = a.w;
  q.drho = b.x;
  q.dmob_dp = b.y;
  q.dmob_ds = b.z;
  return q;
}

// Two lanes per active row, one per phase (l = lane parity: 0 oil, 1 water): each lane evaluates
// its phase's accumulation, fluxes and well terms (FP64), the pair
// exchanges its residual and diagonal rows, and both lanes form D^{-1}.  Pass 1 writes each
// lane's row of the raw off-diagonal blocks (FP64) and marks the row as a boundary cell (V_B: an
// inactive neighbour); pass 2 scales the blocks by S D^{-1} in place, each lane its own row, the
// other row coming from its partner by shuffle.  Splitting the phases halves the chain of
// dependent FP64 instructions a warp issues per row (one FP64 warp instruction per ~64 cycles at
// most on this GPU), and the rows spread over all SMs.
template <typename T, int BLK>
__global__ void __launch_bounds__(BLK) k_assemble(Dev d, FluidK F, double p_scale, double inv_p_scale, int lines,
                                                 int debug) {
  const int nA = d.ctr->n_active;
  const double dt = d.stepp[0], inv_dt = d.stepp[1];
  const double g = F.f.gravity;
  const Fluid& f = F.f;
  T* blocks = (T*)d.blocks;
  double* raw = sizeof(T) == sizeof(double) ? (double*)d.blocks : d.raw;
  T* rhs = (T*)d.rhs;
  const int lane = threadIdx.x & 31, l = lane & 1;
  const unsigned pm = 3u << (lane & 30);  // this lane pair
  double cnv_max = 0.0;
  const int pairs = (gridDim.x * blockDim.x) >> 1;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 1; k < nA; k += pairs) {
    const int i = d.act[k];
    const int e0 = d.row_ptr[i], e1 = d.row_ptr[i + 1];
    const double p_i = d.p[i], sw_i = d.sw[i], z_i = d.depth[i], pvr = d.pv_ref[i];
    const PhaseProps qi = load_props(d.cprops, k, l);
    const double pv = pvr * (1.0 + f.c_r * (p_i - f.p_ref)), dpv = pvr * f.c_r;
    double R, Dp, Ds;  // residual of phase l and row l of the diagonal block (d/dp_i, d/dSw_i)
    {  // accumulation
      const double pn_i = d.pn[i], swn = d.swn[i];
      const double pvn = pvr * (1.0 + f.c_r * (pn_i - f.p_ref));
      const double bn = (l ? f.b_w_ref : f.b_o_ref) * (1.0 + (l ? f.c_w : f.c_o) * (pn_i - f.p_ref));
      const double S = l ? sw_i : 1.0 - sw_i, Sn = l ? swn : 1.0 - swn;
      R = (pv * qi.b * S - pvn * bn * Sn) * inv_dt;
      Dp = (dpv * qi.b + pv * qi.db) * S * inv_dt;
      Ds = (l ? pv : -pv) * qi.b * inv_dt;
    }
    bool edge = false;
    // fracture-line links: the couplings to the previous / next cell of the same segment, when that
    // cell is active too (it is then the previous / next compact row)
    const int lid_i = lines ? d.line_id[i] : -1;
    int eprev = -1, enext = -1;
    // connections in batches of kNb: every load of a batch (neighbour, its state, its set bit and
    // compact row, then its properties) is issued before any is used, so a batch costs about two
    // dependent L2 round trips instead of two per connection; the flux sums run in CSR order
    constexpr int kNb = 8;
    for (int eb = e0; eb < e1; eb += kNb) {
      int jj[kNb], kj[kNb];
      double T_e[kNb], p_j[kNb], z_j[kNb], sw_j[kNb];
      bool in[kNb];
#pragma unroll
      for (int q = 0; q < kNb; q++) {
        jj[q] = eb + q < e1 ? d.nbr[eb + q] : i;
        T_e[q] = eb + q < e1 ? d.trans[eb + q] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kNb; q++) {
        p_j[q] = d.p[jj[q]];
        z_j[q] = d.depth[jj[q]];
        sw_j[q] = d.sw[jj[q]];
        in[q] = bit(d.va, jj[q]);
      }
#pragma unroll
      for (int q = 0; q < kNb; q++) kj[q] = in[q] ? d.inv[jj[q]] : -1;
      PhaseProps qn[kNb];
#pragma unroll
      for (int q = 0; q < kNb; q++)
        if (in[q]) qn[q] = load_props(d.cprops, kj[q], l);
#pragma unroll
      for (int q = 0; q < kNb; q++) {
        const int e = eb + q;
        if (e >= e1) break;
        const int j = jj[q];
        // an active neighbour's properties were computed once this iteration; an inactive one
        // (frozen at its current state, a Dirichlet value) is evaluated here
        const PhaseProps qj = in[q] ? qn[q] : phase_props(F, p_j[q], sw_j[q], l);
        const double dz = z_i - z_j[q];
        const double rho_avg = 0.5 * (qi.rho + qj.rho);
        const double dphi = (p_i - p_j[q]) - (g * rho_avg) * dz;
        const bool up_i = dphi > 0.0 || (dphi == 0.0 && i < j);
        const double tm = T_e[q] * (up_i ? qi.mob : qj.mob);
        R += tm * dphi;
        const double hgdz = g * dz * 0.5;
        double o0 = tm * (-1.0 - hgdz * qj.drho), o1 = 0.0;
        const double dl0 = tm * (1.0 - hgdz * qi.drho);
        double dl0u = 0.0, dl1 = 0.0;
        if (up_i) {
          dl0u = T_e[q] * qi.dmob_dp * dphi;
          dl1 = T_e[q] * qi.dmob_ds * dphi;
        } else {
          o0 += T_e[q] * qj.dmob_dp * dphi;
          o1 = T_e[q] * qj.dmob_ds * dphi;
        }
        Dp += dl0 + dl0u;
        Ds += dl1;
        edge |= !in[q];
        if (l == 0) d.colA[e] = kj[q];
        if (lid_i >= 0 && in[q] && (j == i - 1 || j == i + 1) && d.line_id[j] == lid_i) {
          if (j < i)
            eprev = e;
          else
            enext = e;
        }
        if (debug) {
          d.dbg_off[4 * (size_t)e + 2 * l] = o0;
          d.dbg_off[4 * (size_t)e + 2 * l + 1] = o1;
        }
        if (in[q]) {  // raw row in FP64 until it is scaled
          raw[4 * (size_t)e + 2 * l] = o0;
          raw[4 * (size_t)e + 2 * l + 1] = o1;
        }
      }
    }
    if (edge && l == 0) atomicOr(&d.vb[i >> 5], 1u << (i & 31));
    if (l == 0) {  // line rows: 2 continues a line, 1 starts one; starts listed in any order
      const int fl = lines ? (eprev >= 0 ? 2 : (enext >= 0 ? 1 : 0)) : 0;
      if (lines) {
        d.lnk[k] = make_int2(eprev, enext);
        d.line_row_flag[k] = fl;
        if (fl == 1) d.line_start[atomicAdd(&d.ctr->n_line_starts, 1)] = k;
      }
      d.arow[k] = make_int2(e0, (e1 - e0) | (fl << 24));  // the solver's row reference, one load
    }
    // producers
    for (int w = d.well_of_cell[i]; w >= 0; w = d.well_next[w]) {
      const double dpw = p_i - d.well_bhp[w];
      if (dpw > 0.0) {
        const double wi = d.well_wi[w];
        R += wi * qi.mob * dpw;
        Dp += wi * (qi.dmob_dp * dpw + qi.mob);
        Ds += wi * qi.dmob_ds * dpw;
      }
    }
    // the pair's rows: (R0, D00, D01) from lane 0, (R1, D10, D11) from lane 1
    const double Ro = __shfl_xor_sync(pm, R, 1), bo = __shfl_xor_sync(pm, qi.b, 1);
    const double Dpo = __shfl_xor_sync(pm, Dp, 1), Dso = __shfl_xor_sync(pm, Ds, 1);
    const double R0 = l ? Ro : R, R1 = l ? R : Ro;
    const double D00 = l ? Dpo : Dp, D01 = l ? Dso : Ds;
    const double D10 = l ? Dp : Dpo, D11 = l ? Ds : Dso;
    const double id = 1.0 / (D00 * D11 - D01 * D10);
    const double I00 = D11 * id, I01 = -D01 * id, I10 = -D10 * id, I11 = D00 * id;
    rhs[2 * (size_t)k + l] = l ? (T)(-(I10 * R0 + I11 * R1)) : (T)(-p_scale * (I00 * R0 + I01 * R1));
    if (l == 0) {  // CNV with one FP64 division: 1/(PV b_l) = b_other / (PV b_o b_w)
      const double ipbb = dt / (pv * qi.b * bo);
      cnv_max = fmax(cnv_max, fmax(fabs(R0) * bo * ipbb, fabs(R1) * qi.b * ipbb));
    }
    if (debug) {
      d.resid[2 * (size_t)i + l] = R;
      d.dbg_diag[4 * (size_t)i + 2 * l] = Dp;
      d.dbg_diag[4 * (size_t)i + 2 * l + 1] = Ds;
    }
    // pass 2: row l of S D^{-1} O S^{-1} on the blocks of active columns (colA of this row was
    // written by lane 0 of the pair)
    __syncwarp(pm);
    const double Il0 = l ? I10 : I00, Il1 = l ? I11 : I01;
    for (int e = e0; e < e1; e++) {
      if (d.colA[e] < 0) continue;  // same for both lanes
      const double r0 = raw[4 * (size_t)e + 2 * l], r1 = raw[4 * (size_t)e + 2 * l + 1];  // own row
      const double q0 = __shfl_xor_sync(pm, r0, 1), q1 = __shfl_xor_sync(pm, r1, 1);  // partner's row
      const double o00 = l ? q0 : r0, o01 = l ? q1 : r1, o10 = l ? r0 : q0, o11 = l ? r1 : q1;
      const double m0 = Il0 * o00 + Il1 * o10, m1 = Il0 * o01 + Il1 * o11;
      blocks[4 * (size_t)e + 2 * l] = l ? (T)(m0 * inv_p_scale) : (T)m0;
      blocks[4 * (size_t)e + 2 * l + 1] = l ? (T)m1 : (T)(m1 * p_scale);
    }
  }
  // CNV maximum over the block, one atomic per block that had rows
  if ((int)(blockIdx.x * (BLK / 2)) >= nA) return;
  __shared__ double sh[BLK / 32];
  for (int o = 16; o > 0; o >>= 1) cnv_max = fmax(cnv_max, __shfl_xor_sync(0xffffffffu, cnv_max, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnv_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < BLK / 32; w++) m = fmax(m, sh[w]);
    if (m > 0.0) atomicMax(&d.ctr->cnv_bits, (unsigned long long)__double_as_longlong(m));
  }
}

// ---------------------------------------------------------------------------------------
// Residual-based active sets (the estimate the paper compares against, Section 1 / 4.2): the
// full-domain residual at the current iterate, one thread per cell (both phases), and the cells
// whose CNV_i = max_l |R_l,i| dt / (PV_i b_l,i) >= tol_cnv go to the `reach` bitset and frontier
// list 0 (the seed of the m-layer inflation).  Max CNV over all cells to the counters.  The same
// residual terms as k_assemble, without the Jacobian.
// ---------------------------------------------------------------------------------------
constexpr int kResBlk = 128;

__global__ void __launch_bounds__(kResBlk) k_residual_flags(Dev d, FluidK F, double tol_cnv) {
  const double dt = d.stepp[0], inv_dt = d.stepp[1];
  const Fluid& f = F.f;
  const double g = f.gravity;
  double cmax = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
    const double p_i = d.p[i], sw_i = d.sw[i], z_i = d.depth[i], pvr = d.pv_ref[i];
    const PhaseProps qo = phase_props(F, p_i, sw_i, 0), qw = phase_props(F, p_i, sw_i, 1);
    const double pv = pvr * (1.0 + f.c_r * (p_i - f.p_ref));
    const double pn_i = d.pn[i], swn = d.swn[i];
    const double pvn = pvr * (1.0 + f.c_r * (pn_i - f.p_ref));
    const double bno = f.b_o_ref * (1.0 + f.c_o * (pn_i - f.p_ref));
    const double bnw = f.b_w_ref * (1.0 + f.c_w * (pn_i - f.p_ref));
    double Ro = (pv * qo.b * (1.0 - sw_i) - pvn * bno * (1.0 - swn)) * inv_dt;
    double Rw = (pv * qw.b * sw_i - pvn * bnw * swn) * inv_dt;
    for (int e = d.row_ptr[i]; e < d.row_ptr[i + 1]; e++) {
      const int j = d.nbr[e];
      const double T_e = d.trans[e], p_j = d.p[j], sw_j = d.sw[j];
      const PhaseProps jo = phase_props(F, p_j, sw_j, 0), jw = phase_props(F, p_j, sw_j, 1);
      const double dz = z_i - d.depth[j];
      {
        const double dphi = (p_i - p_j) - (g * (0.5 * (qo.rho + jo.rho))) * dz;
        const bool up_i = dphi > 0.0 || (dphi == 0.0 && i < j);
        Ro += T_e * (up_i ? qo.mob : jo.mob) * dphi;
      }
      {
        const double dphi = (p_i - p_j) - (g * (0.5 * (qw.rho + jw.rho))) * dz;
        const bool up_i = dphi > 0.0 || (dphi == 0.0 && i < j);
        Rw += T_e * (up_i ? qw.mob : jw.mob) * dphi;
      }
    }
    for (int w = d.well_of_cell[i]; w >= 0; w = d.well_next[w]) {
      const double dpw = p_i - d.well_bhp[w];
      if (dpw > 0.0) {
        const double wi = d.well_wi[w];
        Ro += wi * qo.mob * dpw;
        Rw += wi * qw.mob * dpw;
      }
    }
    const double c0 = fabs(Ro) * dt / (pv * qo.b), c1 = fabs(Rw) * dt / (pv * qw.b);
    const double c = c0 > c1 ? c0 : c1;
    if (c >= tol_cnv) {
      atomicOr(&d.reach[i >> 5], 1u << (i & 31));
      d.fr0[atomicAdd(&d.ctr->n_frontier[0], 1)] = i;  // list order does not change the dilation
    }
    cmax = fmax(cmax, c);
  }
  __shared__ double sh[kResBlk / 32];
  for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < kResBlk / 32; w++) mx = fmax(mx, sh[w]);
    atomicMax(&d.ctr->cnv_bits, (unsigned long long)__double_as_longlong(mx));
  }
}

// ---------------------------------------------------------------------------------------
// Fracture-line blocks: consecutive compact rows that are consecutive cells of one fracture
// segment form a block-tridiagonal block of the preconditioner (block Jacobi whose blocks
// are single cells or whole fracture segments).  The assembly marks the line rows, links each
// to its neighbours in the line (CSR entries) and lists the line starts; the factor pass factors
// each line in FP32 (block Thomas algorithm; a preconditioner's rounding changes the Krylov
// convergence rate, not the accuracy of the solution):
//   D'_0 = I, D'_t = I - L_t D'_{t-1}^{-1} U_{t-1},  A_t = -D'_t^{-1} L_t,  G_t = D'_t^{-1} U_t
// so that M^{-1} r is  w_t = D'_t^{-1} r_t + A_t w_{t-1},  z_t = w_t - G_t z_{t+1}.
// ---------------------------------------------------------------------------------------
// One warp per line.  The lanes load the coupling blocks of a whole line block (up to
// kMaxLineRows rows, four rows per lane, all loads in flight together) into shared memory, in
// FP32; lane 0 runs the block Thomas recurrence over the staged rows; the warp stores D'^{-1}, A
// and G (FP32) per row.
constexpr int kLineWarps = 4;
constexpr int kMaxLineRows = kLineBlockRows;

template <typename T>
__global__ void __launch_bounds__(32 * kLineWarps, 1) k_line_factor(Dev d) {
  constexpr int kQ = kMaxLineRows / 32;  // rows per lane in one block
  __shared__ float s_in[kLineWarps][kMaxLineRows][8];
  __shared__ float s_out[kLineWarps][kMaxLineRows][12];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nl = d.ctr->n_line_starts;
  const int nA = d.ctr->n_active;
  const T* blocks = (const T*)d.blocks;
  float* ldinv = (float*)d.line_dinv;
  float* la = (float*)d.line_a;
  float* lg = (float*)d.line_g;
  for (int l = gwarp; l < nl; l += nwarps) {
    const int k0 = d.line_start[l];
    // line length: the start row plus the continuation rows that follow it (kMaxLineRows rows per
    // round of loads)
    int len = 1;
    for (int base = k0 + 1;; base += kMaxLineRows) {
      bool cont[kQ];
#pragma unroll
      for (int q = 0; q < kQ; q++) {
        const int k = base + 32 * q + lane;
        cont[q] = k < nA && d.line_row_flag[k] == 2;
      }
      bool ended = false;
#pragma unroll
      for (int q = 0; q < kQ; q++) {
        if (ended) break;  // uniform
        const unsigned m = __ballot_sync(0xffffffffu, cont[q]);
        if (m == 0xffffffffu) {
          len += 32;
        } else {
          len += __ffs(~m) - 1;
          ended = true;
        }
      }
      if (ended) break;
    }
    // each block of up to kMaxLineRows rows: its couplings (U_t: row t -> t+1, L_t: row t -> t-1)
    // are staged in FP32 (all loads of the block issued together), lane 0 runs the recurrence, the
    // lanes store D'^{-1}, A and G.  Couplings across a cut are left out, so a block starts from
    // D'_0 = I.
    for (int b0 = 0; b0 < len; b0 += kMaxLineRows) {
      const int blen = min(kMaxLineRows, len - b0);
#pragma unroll
      for (int q = 0; q < kQ; q++) {
        const int j = 32 * q + lane;
        float U[4] = {0.f, 0.f, 0.f, 0.f}, L[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < blen) {
          const int2 lk = d.lnk[k0 + b0 + j];
          if (j + 1 < blen) {
            const Blk4<T> b = *(const Blk4<T>*)&blocks[4 * (size_t)lk.y];
            U[0] = (float)b.a, U[1] = (float)b.b, U[2] = (float)b.c, U[3] = (float)b.d;
          }
          if (j >= 1) {
            const Blk4<T> b = *(const Blk4<T>*)&blocks[4 * (size_t)lk.x];
            L[0] = (float)b.a, L[1] = (float)b.b, L[2] = (float)b.c, L[3] = (float)b.d;
          }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
          s_in[wib][j][c] = U[c];
          s_in[wib][j][4 + c] = L[c];
        }
      }
      __syncwarp();
      if (lane == 0) {
        float Gp[4] = {0.f, 0.f, 0.f, 0.f};  // G of the previous row
        for (int j = 0; j < blen; j++) {
          float Di[4], A[4];
          if (j == 0) {
            Di[0] = 1.f, Di[1] = 0.f, Di[2] = 0.f, Di[3] = 1.f;
            A[0] = A[1] = A[2] = A[3] = 0.f;
          } else {
            const float* Lt = &s_in[wib][j][4];
            // D' = I - L G_{t-1}
            const float p0 = 1.f - (Lt[0] * Gp[0] + Lt[1] * Gp[2]);
            const float p1 = -(Lt[0] * Gp[1] + Lt[1] * Gp[3]);
            const float p2 = -(Lt[2] * Gp[0] + Lt[3] * Gp[2]);
            const float p3 = 1.f - (Lt[2] * Gp[1] + Lt[3] * Gp[3]);
            const float id = 1.f / (p0 * p3 - p1 * p2);
            Di[0] = p3 * id, Di[1] = -p1 * id, Di[2] = -p2 * id, Di[3] = p0 * id;
            A[0] = -(Di[0] * Lt[0] + Di[1] * Lt[2]);
            A[1] = -(Di[0] * Lt[1] + Di[1] * Lt[3]);
            A[2] = -(Di[2] * Lt[0] + Di[3] * Lt[2]);
            A[3] = -(Di[2] * Lt[1] + Di[3] * Lt[3]);
          }
          const float* Ut = &s_in[wib][j][0];
          float G[4];
          G[0] = Di[0] * Ut[0] + Di[1] * Ut[2];
          G[1] = Di[0] * Ut[1] + Di[1] * Ut[3];
          G[2] = Di[2] * Ut[0] + Di[3] * Ut[2];
          G[3] = Di[2] * Ut[1] + Di[3] * Ut[3];
#pragma unroll
          for (int c = 0; c < 4; c++) {
            s_out[wib][j][c] = Di[c];
            s_out[wib][j][4 + c] = A[c];
            s_out[wib][j][8 + c] = G[c];
            Gp[c] = G[c];
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kQ; q++) {
        const int j = 32 * q + lane;
        if (j < blen) {
          const size_t k = (size_t)(k0 + b0 + j);
          const float* o = s_out[wib][j];
          *(float4*)&ldinv[4 * k] = make_float4(o[0], o[1], o[2], o[3]);
          *(float4*)&la[4 * k] = make_float4(o[4], o[5], o[6], o[7]);
          *(float4*)&lg[4 * k] = make_float4(o[8], o[9], o[10], o[11]);
        }
      }
      __syncwarp();
    }
    // lines longer than kMaxLineRows are cut into blocks of kMaxLineRows rows (the couplings at the
    // cuts were left out of the factors above); each block start is marked in lblk with its length
    // at line_len[start], and the ascending list of block starts is compacted afterwards, so that
    // the blocks are numbered the same way in every run
    if (lane == 0)
      for (int q = 0; q < len; q += kMaxLineRows) {
        const int k = k0 + q;
        atomicOr(&d.lblk[k >> 5], 1u << (k & 31));
        d.line_len[k] = min(kMaxLineRows, len - q);
      }
  }
}

// line_cum[l] = rows of the line blocks before block l of the ascending list, for l = 0 .. n_lines
// (the grid solver weighs its row chunks by it).  One block: each thread sums a run of consecutive
// blocks, an exclusive scan over the threads gives the runs' offsets, then each run is written.
constexpr int kCumThreads = 1024;
__global__ void __launch_bounds__(kCumThreads, 1) k_line_cum(Dev d) {
  __shared__ int s_w[32];
  __shared__ int s_tot;
  const int nl = d.ctr->n_lines;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int per = (nl + kCumThreads - 1) / kCumThreads;
  const int l0 = min(nl, (int)threadIdx.x * per), l1 = min(nl, l0 + per);
  int sum = 0;
#pragma unroll 4
  for (int l = l0; l < l1; l++) sum += __ldg(&d.line_len[__ldg(&d.line_start[l])]);
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int v = s_w[lane];
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, iv, o);
      if (lane >= o) iv += u;
    }
    s_w[lane] = iv - v;
    if (lane == 31) s_tot = iv;
  }
  __syncthreads();
  int run = s_w[w] + incl - sum;
  for (int l = l0; l < l1; l++) {
    d.line_cum[l] = run;
    run += __ldg(&d.line_len[__ldg(&d.line_start[l])]);
  }
  if (threadIdx.x == 0) d.line_cum[nl] = s_tot;
}

}  // namespace

cudaError_t launch_assemble(const Dev& d, double p_scale, int fp32, int lines, int debug, LaunchCfg c) {
  if (lines) {  // the assembly lists the line starts; the factor pass marks the line blocks
    cudaError_t e = cudaMemsetAsync(&d.ctr->n_lines, 0, 2 * sizeof(int), c.stream);  // n_lines, n_line_starts
    if (e == cudaSuccess) e = cudaMemsetAsync(d.lblk, 0, sizeof(uint32_t) * (size_t)d.W, c.stream);
    if (e != cudaSuccess) return e;
  }
  FluidK F;
  F.f = d.fl;
  F.inv_span = 1.0 / (1.0 - d.fl.swc - d.fl.sor);
  F.inv_mu[0] = 1.0 / d.fl.mu_o;
  F.inv_mu[1] = 1.0 / d.fl.mu_w;
  // launch shape (results do not depend on it: every row is computed by its own lane pair)
  const int blk = c.asm_block == 128 || c.asm_block == 256 ? c.asm_block : kAsmBlk;
  const int grid = (c.asm_mult >= 1 && c.asm_mult <= 16 ? c.asm_mult : 4) * c.sms;
  count_launches(2);
  k_cell_props<<<grid / 2 > 0 ? grid / 2 : 1, 128, 0, c.stream>>>(d, F);
  const double ips = 1.0 / p_scale;
  if (fp32) {
    if (blk == 256)
      k_assemble<float, 256><<<grid, 256, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
    else if (blk == 128)
      k_assemble<float, 128><<<grid, 128, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
    else
      k_assemble<float, kAsmBlk><<<grid, kAsmBlk, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
  } else {
    if (blk == 256)
      k_assemble<double, 256><<<grid, 256, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
    else if (blk == 128)
      k_assemble<double, 128><<<grid, 128, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
    else
      k_assemble<double, kAsmBlk><<<grid, kAsmBlk, 0, c.stream>>>(d, F, p_scale, ips, lines, debug);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual_flags(const Dev& d, double tol_cnv, LaunchCfg c) {
  if (d.n == 0) return cudaSuccess;
  FluidK F;
  F.f = d.fl;
  F.inv_span = 1.0 / (1.0 - d.fl.swc - d.fl.sor);
  F.inv_mu[0] = 1.0 / d.fl.mu_o;
  F.inv_mu[1] = 1.0 / d.fl.mu_w;
  const int grid = std::min((d.n + kResBlk - 1) / kResBlk, 16 * c.sms);
  count_launches(1);
  k_residual_flags<<<grid, kResBlk, 0, c.stream>>>(d, F, tol_cnv);
  return cudaGetLastError();
}

cudaError_t launch_line_setup(const Dev& d, int fp32, LaunchCfg c) {
  count_launches(1);
  if (fp32)
    k_line_factor<float><<<c.sms, 32 * kLineWarps, 0, c.stream>>>(d);
  else
    k_line_factor<double><<<c.sms, 32 * kLineWarps, 0, c.stream>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // ascending line-block starts (compact rows < n_active <= n, so the n-bit bitset covers them)
  e = launch_compact(d, d.lblk, d.line_start, d.lscratch, &d.ctr->n_lines, c);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_line_cum<<<1, kCumThreads, 0, c.stream>>>(d);
  return cudaGetLastError();
}

}  // namespace lns
