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
// Mapping: one thread per active row (each cell's properties evaluated once per use, no
// redundant FP64 work: FP64 issues at a small fraction of the FP32 rate on this GPU).  The
// boundary set V_B of the solved set (rows with an inactive neighbour) falls out of the
// column scan and is written here too.
#include <cuda_runtime.h>

#include "lns_internal.cuh"

namespace lns {

namespace {

constexpr int kAsmBlk = 256;

struct FluidK {
  Fluid f;
  double inv_span, inv_mu[2];
};

struct Props {
  double pv, dpv, b[2], db[2], rho[2], drho[2], mob[2], dmob_dp[2], dmob_ds[2];
};

__device__ __forceinline__ double ipow(double x, int k) {
  double r = 1.0;
  for (int t = 0; t < k; t++) r *= x;
  return r;
}

__device__ __forceinline__ void cell_props(const FluidK& F, double pv_ref, double p, double sw, Props& q) {
  const Fluid& f = F.f;
  const double dpr = p - f.p_ref;
  q.pv = pv_ref * (1.0 + f.c_r * dpr);
  q.dpv = pv_ref * f.c_r;
  q.b[0] = f.b_o_ref * (1.0 + f.c_o * dpr);
  q.db[0] = f.b_o_ref * f.c_o;
  q.b[1] = f.b_w_ref * (1.0 + f.c_w * dpr);
  q.db[1] = f.b_w_ref * f.c_w;
  q.rho[0] = f.rho_o_ref * q.b[0];
  q.drho[0] = f.rho_o_ref * q.db[0];
  q.rho[1] = f.rho_w_ref * q.b[1];
  q.drho[1] = f.rho_w_ref * q.db[1];
  double se = (sw - f.swc) * F.inv_span, dse = F.inv_span;
  if (se <= 0.0) {
    se = 0.0;
    dse = 0.0;
  } else if (se >= 1.0) {
    se = 1.0;
    dse = 0.0;
  }
  const double kro = ipow(1.0 - se, f.n_o), dkro = -(double)f.n_o * ipow(1.0 - se, f.n_o - 1) * dse;
  const double krw = ipow(se, f.n_w), dkrw = (double)f.n_w * ipow(se, f.n_w - 1) * dse;
  q.mob[0] = kro * F.inv_mu[0] * q.b[0];
  q.dmob_dp[0] = kro * F.inv_mu[0] * q.db[0];
  q.dmob_ds[0] = dkro * F.inv_mu[0] * q.b[0];
  q.mob[1] = krw * F.inv_mu[1] * q.b[1];
  q.dmob_dp[1] = krw * F.inv_mu[1] * q.db[1];
  q.dmob_ds[1] = dkrw * F.inv_mu[1] * q.b[1];
}

__device__ __forceinline__ bool bit(const uint32_t* s, int i) { return (s[i >> 5] >> (i & 31)) & 1u; }

template <typename T>
struct alignas(4 * sizeof(T)) Blk4 {
  T a, b, c, d;
};

// One thread per active row.  Pass 1 evaluates the row's fluxes, accumulation and wells in
// FP64, writes the raw off-diagonal blocks and marks the row as a boundary cell (V_B: an
// inactive neighbour); pass 2 scales the row by S D^{-1} in place.
template <typename T>
__global__ void __launch_bounds__(kAsmBlk) k_assemble(Dev d, FluidK F, double dt, double inv_dt, double p_scale,
                                                     double inv_p_scale, int debug) {
  const int nA = d.ctr->n_active;
  const double g = F.f.gravity;
  T* blocks = (T*)d.blocks;
  double* raw = sizeof(T) == sizeof(double) ? (double*)d.blocks : d.raw;
  T* rhs = (T*)d.rhs;
  double cnv_max = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nA; k += gridDim.x * blockDim.x) {
    const int i = d.act[k];
    const int e0 = d.row_ptr[i], e1 = d.row_ptr[i + 1];
    const double p_i = d.p[i], sw_i = d.sw[i], z_i = d.depth[i];
    Props qi;
    cell_props(F, d.pv_ref[i], p_i, sw_i, qi);
    double R0, R1, D00, D01, D10, D11;
    {  // accumulation
      Props qn;
      const double swn = d.swn[i];
      cell_props(F, d.pv_ref[i], d.pn[i], swn, qn);
      const double so = 1.0 - sw_i, son = 1.0 - swn;
      R0 = (qi.pv * qi.b[0] * so - qn.pv * qn.b[0] * son) * inv_dt;
      R1 = (qi.pv * qi.b[1] * sw_i - qn.pv * qn.b[1] * swn) * inv_dt;
      D00 = (qi.dpv * qi.b[0] + qi.pv * qi.db[0]) * so * inv_dt;
      D01 = -qi.pv * qi.b[0] * inv_dt;
      D10 = (qi.dpv * qi.b[1] + qi.pv * qi.db[1]) * sw_i * inv_dt;
      D11 = qi.pv * qi.b[1] * inv_dt;
    }
    bool edge = false;
    for (int e = e0; e < e1; e++) {
      const int j = d.nbr[e];
      const double T_e = d.trans[e];
      const double p_j = d.p[j];
      Props qj;
      cell_props(F, d.pv_ref[j], p_j, d.sw[j], qj);
      const double dz = z_i - d.depth[j];
      const double dpp = p_i - p_j;
      double o[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int l = 0; l < 2; l++) {
        const double rho_avg = 0.5 * (qi.rho[l] + qj.rho[l]);
        const double dphi = dpp - (g * rho_avg) * dz;
        const bool up_i = dphi > 0.0 || (dphi == 0.0 && i < j);
        const double tm = T_e * (up_i ? qi.mob[l] : qj.mob[l]);
        const double rl = tm * dphi;
        const double dl0 = tm * (1.0 - g * dz * 0.5 * qi.drho[l]);
        o[2 * l] = tm * (-1.0 - g * dz * 0.5 * qj.drho[l]);
        double dl0u = 0.0, dl1 = 0.0;
        if (up_i) {
          dl0u = T_e * qi.dmob_dp[l] * dphi;
          dl1 = T_e * qi.dmob_ds[l] * dphi;
        } else {
          o[2 * l] += T_e * qj.dmob_dp[l] * dphi;
          o[2 * l + 1] = T_e * qj.dmob_ds[l] * dphi;
        }
        if (l == 0) {
          R0 += rl;
          D00 += dl0 + dl0u;
          D01 += dl1;
        } else {
          R1 += rl;
          D10 += dl0 + dl0u;
          D11 += dl1;
        }
      }
      const bool in = bit(d.va, j);
      edge |= !in;
      d.colA[e] = in ? d.inv[j] : -1;
      if (debug) {
        d.dbg_off[4 * (size_t)e + 0] = o[0];
        d.dbg_off[4 * (size_t)e + 1] = o[1];
        d.dbg_off[4 * (size_t)e + 2] = o[2];
        d.dbg_off[4 * (size_t)e + 3] = o[3];
      }
      if (in) {  // raw block in FP64 until it is scaled (FP32 rounding before D^{-1} could cancel)
        Blk4<double> bk = {o[0], o[1], o[2], o[3]};
        *(Blk4<double>*)&raw[4 * (size_t)e] = bk;
      }
    }
    if (edge) atomicOr(&d.vb[i >> 5], 1u << (i & 31));
    // producers
    for (int w = d.well_of_cell[i]; w >= 0; w = d.well_next[w]) {
      const double dpw = p_i - d.well_bhp[w];
      if (dpw > 0.0) {
        const double wi = d.well_wi[w];
        R0 += wi * qi.mob[0] * dpw;
        R1 += wi * qi.mob[1] * dpw;
        D00 += wi * (qi.dmob_dp[0] * dpw + qi.mob[0]);
        D01 += wi * qi.dmob_ds[0] * dpw;
        D10 += wi * (qi.dmob_dp[1] * dpw + qi.mob[1]);
        D11 += wi * qi.dmob_ds[1] * dpw;
      }
    }
    const double id = 1.0 / (D00 * D11 - D01 * D10);
    const double I00 = D11 * id, I01 = -D01 * id, I10 = -D10 * id, I11 = D00 * id;
    rhs[2 * (size_t)k] = (T)(-p_scale * (I00 * R0 + I01 * R1));
    rhs[2 * (size_t)k + 1] = (T)(-(I10 * R0 + I11 * R1));
    {  // CNV with one FP64 division: 1/(PV b_l) = b_other / (PV b_o b_w)
      const double ipbb = dt / (qi.pv * qi.b[0] * qi.b[1]);
      cnv_max = fmax(cnv_max, fmax(fabs(R0) * qi.b[1] * ipbb, fabs(R1) * qi.b[0] * ipbb));
    }
    if (debug) {
      d.resid[2 * (size_t)i] = R0;
      d.resid[2 * (size_t)i + 1] = R1;
      d.dbg_diag[4 * (size_t)i + 0] = D00;
      d.dbg_diag[4 * (size_t)i + 1] = D01;
      d.dbg_diag[4 * (size_t)i + 2] = D10;
      d.dbg_diag[4 * (size_t)i + 3] = D11;
    }
    // pass 2: S D^{-1} O S^{-1} on the blocks of active columns
    const double sp = p_scale, isp = inv_p_scale;
    for (int e = e0; e < e1; e++) {
      if (d.colA[e] < 0) continue;
      const Blk4<double> bk = *(const Blk4<double>*)&raw[4 * (size_t)e];
      const double o0 = bk.a, o1 = bk.b, o2 = bk.c, o3 = bk.d;
      const double m00 = I00 * o0 + I01 * o2, m01 = I00 * o1 + I01 * o3;
      const double m10 = I10 * o0 + I11 * o2, m11 = I10 * o1 + I11 * o3;
      Blk4<T> sk = {(T)m00, (T)(m01 * sp), (T)(m10 * isp), (T)m11};
      *(Blk4<T>*)&blocks[4 * (size_t)e] = sk;
    }
  }
  // CNV maximum over the block, one atomic per block
  __shared__ double sh[kAsmBlk / 32];
  for (int o = 16; o > 0; o >>= 1) cnv_max = fmax(cnv_max, __shfl_xor_sync(0xffffffffu, cnv_max, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnv_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kAsmBlk / 32; w++) m = fmax(m, sh[w]);
    atomicMax(&d.ctr->cnv_bits, (unsigned long long)__double_as_longlong(m));
  }
}

// ---------------------------------------------------------------------------------------
// Fracture-line blocks: consecutive compact rows that are consecutive cells of one fracture
// segment form a block-tridiagonal block of the preconditioner (block Jacobi whose blocks
// are single cells or whole fracture segments).  Pass 1 marks line rows and lists line
// starts; pass 2 factors each line in FP32 (block Thomas algorithm; a preconditioner's
// rounding changes the Krylov convergence rate, not the accuracy of the solution):
//   D'_0 = I, D'_t = I - L_t D'_{t-1}^{-1} U_{t-1},  A_t = -D'_t^{-1} L_t,  G_t = D'_t^{-1} U_t
// so that M^{-1} r is  w_t = D'_t^{-1} r_t + A_t w_{t-1},  z_t = w_t - G_t z_{t+1}.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int find_entry(const int* row_ptr, const int* nbr, int i, int j) {
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++)
    if (nbr[e] == j) return e;
  return -1;
}

__global__ void k_line_mark(Dev d) {
  const int nA = d.ctr->n_active;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nA; k += gridDim.x * blockDim.x) {
    const int i = d.act[k];
    const int lid = d.line_id[i];
    bool cont = false, next = false;
    if (lid >= 0) {
      if (k > 0 && d.act[k - 1] == i - 1 && d.line_id[i - 1] == lid)
        cont = find_entry(d.row_ptr, d.nbr, i, i - 1) >= 0 && find_entry(d.row_ptr, d.nbr, i - 1, i) >= 0;
      if (k + 1 < nA && d.act[k + 1] == i + 1 && d.line_id[i + 1] == lid)
        next = find_entry(d.row_ptr, d.nbr, i, i + 1) >= 0 && find_entry(d.row_ptr, d.nbr, i + 1, i) >= 0;
    }
    d.line_row_flag[k] = cont ? 2 : (next ? 1 : 0);
    if (next && !cont) {
      int pos = atomicAdd(&d.ctr->n_line_starts, 1);
      d.line_start[pos] = k;
    }
  }
}

// One warp per line.  The lanes find and load the line's coupling blocks (U_t: row t -> t+1,
// L_t: row t -> t-1) 32 rows at a time into shared memory, in FP32; lane 0 runs the block
// Thomas recurrence over the staged rows; the warp stores D'^{-1}, A and G (FP32) per row.
constexpr int kLineWarps = 4;
constexpr int kMaxLineRows = kLineBlockRows;

template <typename T>
__global__ void __launch_bounds__(32 * kLineWarps, 1) k_line_factor(Dev d) {
  __shared__ float s_in[kLineWarps][32][8];
  __shared__ float s_out[kLineWarps][32][12];
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
    // line length: the start row plus the continuation rows that follow it
    int len = 1;
    for (int base = k0 + 1;; base += 32) {
      const int k = base + lane;
      const bool cont = k < nA && d.line_row_flag[k] == 2;
      const unsigned m = __ballot_sync(0xffffffffu, cont);
      if (m == 0xffffffffu) {
        len += 32;
        continue;
      }
      len += __ffs(~m) - 1;
      break;
    }
    float Gp[4] = {0.f, 0.f, 0.f, 0.f};  // G of the previous row (lane 0)
    for (int base = 0; base < len; base += 32) {
      const int t = base + lane;
      float U[4] = {0.f, 0.f, 0.f, 0.f}, L[4] = {0.f, 0.f, 0.f, 0.f};
      if (t < len) {
        const int i = d.act[k0 + t];
        if (t + 1 < len && (t + 1) % kMaxLineRows != 0) {
          const Blk4<T> b = *(const Blk4<T>*)&blocks[4 * (size_t)find_entry(d.row_ptr, d.nbr, i, i + 1)];
          U[0] = (float)b.a, U[1] = (float)b.b, U[2] = (float)b.c, U[3] = (float)b.d;
        }
        if (t >= 1 && t % kMaxLineRows != 0) {
          const Blk4<T> b = *(const Blk4<T>*)&blocks[4 * (size_t)find_entry(d.row_ptr, d.nbr, i, i - 1)];
          L[0] = (float)b.a, L[1] = (float)b.b, L[2] = (float)b.c, L[3] = (float)b.d;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        s_in[wib][lane][q] = U[q];
        s_in[wib][lane][4 + q] = L[q];
      }
      __syncwarp();
      if (lane == 0) {
        const int cnt = min(32, len - base);
        for (int j = 0; j < cnt; j++) {
          const int tt = base + j;
          float Di[4], A[4];
          if (tt == 0) {
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
          for (int q = 0; q < 4; q++) {
            s_out[wib][j][q] = Di[q];
            s_out[wib][j][4 + q] = A[q];
            s_out[wib][j][8 + q] = G[q];
            Gp[q] = G[q];
          }
        }
      }
      __syncwarp();
      if (t < len) {
        const size_t k = (size_t)(k0 + t);
        *(float4*)&ldinv[4 * k] = make_float4(s_out[wib][lane][0], s_out[wib][lane][1], s_out[wib][lane][2],
                                               s_out[wib][lane][3]);
        *(float4*)&la[4 * k] = make_float4(s_out[wib][lane][4], s_out[wib][lane][5], s_out[wib][lane][6],
                                            s_out[wib][lane][7]);
        *(float4*)&lg[4 * k] = make_float4(s_out[wib][lane][8], s_out[wib][lane][9], s_out[wib][lane][10],
                                            s_out[wib][lane][11]);
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

}  // namespace

cudaError_t launch_assemble(const Dev& d, double dt, double p_scale, int fp32, int debug, LaunchCfg c) {
  FluidK F;
  F.f = d.fl;
  F.inv_span = 1.0 / (1.0 - d.fl.swc - d.fl.sor);
  F.inv_mu[0] = 1.0 / d.fl.mu_o;
  F.inv_mu[1] = 1.0 / d.fl.mu_w;
  const int grid = 4 * c.sms;
  count_launches(1);
  if (fp32)
    k_assemble<float><<<grid, kAsmBlk, 0, c.stream>>>(d, F, dt, 1.0 / dt, p_scale, 1.0 / p_scale, debug);
  else
    k_assemble<double><<<grid, kAsmBlk, 0, c.stream>>>(d, F, dt, 1.0 / dt, p_scale, 1.0 / p_scale, debug);
  return cudaGetLastError();
}

cudaError_t launch_line_setup(const Dev& d, int fp32, LaunchCfg c) {
  cudaError_t e = cudaMemsetAsync(&d.ctr->n_lines, 0, 2 * sizeof(int), c.stream);  // n_lines, n_line_starts
  if (e == cudaSuccess) e = cudaMemsetAsync(d.lblk, 0, sizeof(uint32_t) * (size_t)d.W, c.stream);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_line_mark<<<4 * c.sms, 256, 0, c.stream>>>(d);
  count_launches(1);
  if (fp32)
    k_line_factor<float><<<c.sms, 32 * kLineWarps, 0, c.stream>>>(d);
  else
    k_line_factor<double><<<c.sms, 32 * kLineWarps, 0, c.stream>>>(d);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // ascending line-block starts (compact rows < n_active <= n, so the n-bit bitset covers them)
  return launch_compact(d, d.lblk, d.line_start, d.lscratch, &d.ctr->n_lines, c);
}

}  // namespace lns
