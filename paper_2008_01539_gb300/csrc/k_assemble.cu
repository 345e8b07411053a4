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
// Mapping: LPR lanes per row (one lane per connection of the row), warp-uniform loops so the
// lane groups can reduce with shuffles.
#include <cuda_runtime.h>

#include "lns_internal.cuh"

namespace lns {

namespace {

constexpr int kLPR = 8;   // lanes per row
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
struct Blk4 {
  T a, b, c, d;
};

template <typename T, int LPR>
__global__ void __launch_bounds__(kAsmBlk) k_assemble(Dev d, FluidK F, double dt, double p_scale, int debug) {
  const int nA = d.ctr->n_active;
  const int lane = threadIdx.x & 31;
  const int q = lane % LPR;                       // lane within the row group
  const int grp = lane / LPR;                     // row group within the warp
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const double inv_dt = 1.0 / dt;
  const double g = F.f.gravity;
  T* blocks = (T*)d.blocks;
  T* rhs = (T*)d.rhs;
  double cnv_max = 0.0;
  for (int base = gwarp * (32 / LPR); base < nA; base += warps * (32 / LPR)) {
    const int k = base + grp;
    const bool valid = k < nA;
    double R0 = 0.0, R1 = 0.0, D00 = 0.0, D01 = 0.0, D10 = 0.0, D11 = 0.0;
    double O00 = 0.0, O01 = 0.0, O10 = 0.0, O11 = 0.0;
    int i = 0, e0 = 0, e1 = 0;
    Props qi;
    if (valid) {
      i = d.act[k];
      e0 = d.row_ptr[i];
      e1 = d.row_ptr[i + 1];
      const double p_i = d.p[i], sw_i = d.sw[i], z_i = d.depth[i];
      cell_props(F, d.pv_ref[i], p_i, sw_i, qi);
      for (int e = e0 + q, round = 0; e < e1; e += LPR, round++) {
        const int j = d.nbr[e];
        const double T_e = d.trans[e];
        Props qj;
        const double p_j = d.p[j];
        cell_props(F, d.pv_ref[j], p_j, d.sw[j], qj);
        const double dz = z_i - d.depth[j];
        const double dpp = p_i - p_j;
        double o[4] = {0.0, 0.0, 0.0, 0.0};
        double Rl[2] = {0.0, 0.0}, Dl[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
        for (int l = 0; l < 2; l++) {
          const double rho_avg = 0.5 * (qi.rho[l] + qj.rho[l]);
          const double dphi = dpp - (g * rho_avg) * dz;
          const bool up_i = dphi > 0.0 || (dphi == 0.0 && i < j);
          const double tm = T_e * (up_i ? qi.mob[l] : qj.mob[l]);
          Rl[l] = tm * dphi;
          Dl[l][0] = tm * (1.0 - g * dz * 0.5 * qi.drho[l]);
          o[2 * l] = tm * (-1.0 - g * dz * 0.5 * qj.drho[l]);
          if (up_i) {
            Dl[l][0] += T_e * qi.dmob_dp[l] * dphi;
            Dl[l][1] = T_e * qi.dmob_ds[l] * dphi;
          } else {
            o[2 * l] += T_e * qj.dmob_dp[l] * dphi;
            o[2 * l + 1] = T_e * qj.dmob_ds[l] * dphi;
          }
        }
        R0 += Rl[0];
        R1 += Rl[1];
        D00 += Dl[0][0];
        D01 += Dl[0][1];
        D10 += Dl[1][0];
        D11 += Dl[1][1];
        d.colA[e] = bit(d.va, j) ? d.inv[j] : -1;
        if (debug) {
          d.dbg_off[4 * (size_t)e + 0] = o[0];
          d.dbg_off[4 * (size_t)e + 1] = o[1];
          d.dbg_off[4 * (size_t)e + 2] = o[2];
          d.dbg_off[4 * (size_t)e + 3] = o[3];
        }
        if (round == 0) {
          O00 = o[0];
          O01 = o[1];
          O10 = o[2];
          O11 = o[3];
        } else {  // rows with more than LPR connections: park the raw block, scale it below
          Blk4<T> bk = {(T)o[0], (T)o[1], (T)o[2], (T)o[3]};
          *(Blk4<T>*)&blocks[4 * (size_t)e] = bk;
        }
      }
      if (q == 0) {
        // accumulation
        Props qn;
        const double sw_i2 = d.sw[i], swn = d.swn[i];
        cell_props(F, d.pv_ref[i], d.pn[i], swn, qn);
        const double so = 1.0 - sw_i2, son = 1.0 - swn;
        R0 += (qi.pv * qi.b[0] * so - qn.pv * qn.b[0] * son) * inv_dt;
        R1 += (qi.pv * qi.b[1] * sw_i2 - qn.pv * qn.b[1] * swn) * inv_dt;
        D00 += (qi.dpv * qi.b[0] + qi.pv * qi.db[0]) * so * inv_dt;
        D01 += -qi.pv * qi.b[0] * inv_dt;
        D10 += (qi.dpv * qi.b[1] + qi.pv * qi.db[1]) * sw_i2 * inv_dt;
        D11 += qi.pv * qi.b[1] * inv_dt;
        // producers
        for (int w = d.well_of_cell[i]; w >= 0; w = d.well_next[w]) {
          const double dpw = d.p[i] - d.well_bhp[w];
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
      }
    }
    // sum the row over its lane group
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
      R0 += __shfl_xor_sync(0xffffffffu, R0, o, LPR);
      R1 += __shfl_xor_sync(0xffffffffu, R1, o, LPR);
      D00 += __shfl_xor_sync(0xffffffffu, D00, o, LPR);
      D01 += __shfl_xor_sync(0xffffffffu, D01, o, LPR);
      D10 += __shfl_xor_sync(0xffffffffu, D10, o, LPR);
      D11 += __shfl_xor_sync(0xffffffffu, D11, o, LPR);
    }
    if (!valid) continue;
    const double det = D00 * D11 - D01 * D10;
    const double id = 1.0 / det;
    const double I00 = D11 * id, I01 = -D01 * id, I10 = -D10 * id, I11 = D00 * id;
    if (q == 0) {
      rhs[2 * (size_t)k] = (T)(-p_scale * (I00 * R0 + I01 * R1));
      rhs[2 * (size_t)k + 1] = (T)(-(I10 * R0 + I11 * R1));
      const double c0 = fabs(R0) * dt / (qi.pv * qi.b[0]);
      const double c1 = fabs(R1) * dt / (qi.pv * qi.b[1]);
      cnv_max = fmax(cnv_max, fmax(c0, c1));
      if (debug) {
        d.resid[2 * (size_t)i] = R0;
        d.resid[2 * (size_t)i + 1] = R1;
        d.dbg_diag[4 * (size_t)i + 0] = D00;
        d.dbg_diag[4 * (size_t)i + 1] = D01;
        d.dbg_diag[4 * (size_t)i + 2] = D10;
        d.dbg_diag[4 * (size_t)i + 3] = D11;
      }
    }
    const double sp = p_scale, isp = 1.0 / p_scale;
    for (int e = e0 + q, round = 0; e < e1; e += LPR, round++) {
      double o0, o1, o2, o3;
      if (round == 0) {
        o0 = O00;
        o1 = O01;
        o2 = O10;
        o3 = O11;
      } else {
        Blk4<T> bk = *(const Blk4<T>*)&blocks[4 * (size_t)e];
        o0 = bk.a;
        o1 = bk.b;
        o2 = bk.c;
        o3 = bk.d;
      }
      // S D^{-1} O S^{-1}
      const double m00 = I00 * o0 + I01 * o2, m01 = I00 * o1 + I01 * o3;
      const double m10 = I10 * o0 + I11 * o2, m11 = I10 * o1 + I11 * o3;
      Blk4<T> bk = {(T)m00, (T)(m01 * sp), (T)(m10 * isp), (T)m11};
      *(Blk4<T>*)&blocks[4 * (size_t)e] = bk;
    }
  }
  // CNV maximum over the block, one atomic per block
  __shared__ double sh[kAsmBlk / 32];
  for (int o = 16; o > 0; o >>= 1) cnv_max = fmax(cnv_max, __shfl_xor_sync(0xffffffffu, cnv_max, o));
  if (lane == 0) sh[threadIdx.x >> 5] = cnv_max;
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
// starts; pass 2 factors each line (block Thomas algorithm):
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
      int pos = atomicAdd(&d.ctr->n_lines, 1);
      d.line_start[pos] = k;
    }
  }
}

template <typename T>
__device__ __forceinline__ void inv2(const double* a, double* r) {
  const double id = 1.0 / (a[0] * a[3] - a[1] * a[2]);
  r[0] = a[3] * id;
  r[1] = -a[1] * id;
  r[2] = -a[2] * id;
  r[3] = a[0] * id;
}

__device__ __forceinline__ void mul2(const double* a, const double* b, double* c) {
  c[0] = a[0] * b[0] + a[1] * b[2];
  c[1] = a[0] * b[1] + a[1] * b[3];
  c[2] = a[2] * b[0] + a[3] * b[2];
  c[3] = a[2] * b[1] + a[3] * b[3];
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, double* v) {
  Blk4<T> b = *(const Blk4<T>*)p;
  v[0] = b.a;
  v[1] = b.b;
  v[2] = b.c;
  v[3] = b.d;
}

template <typename T>
__device__ __forceinline__ void store4(T* p, const double* v) {
  Blk4<T> b = {(T)v[0], (T)v[1], (T)v[2], (T)v[3]};
  *(Blk4<T>*)p = b;
}

template <typename T>
__global__ void k_line_factor(Dev d) {
  const int nl = d.ctr->n_lines;
  const int nA = d.ctr->n_active;
  const T* blocks = (const T*)d.blocks;
  T* ldinv = (T*)d.line_dinv;
  T* la = (T*)d.line_a;
  T* lg = (T*)d.line_g;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    int k = d.line_start[l];
    double dinv[4] = {1.0, 0.0, 0.0, 1.0};
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    store4<T>(&ldinv[4 * (size_t)k], dinv);
    store4<T>(&la[4 * (size_t)k], zero);
    int len = 1;
    while (k + 1 < nA && d.line_row_flag[k + 1] == 2) {
      const int i = d.act[k], i1 = d.act[k + 1];
      double U[4], L[4], G[4], LG[4], Dp[4], Dn[4], A[4];
      load4<T>(&blocks[4 * (size_t)find_entry(d.row_ptr, d.nbr, i, i1)], U);
      load4<T>(&blocks[4 * (size_t)find_entry(d.row_ptr, d.nbr, i1, i)], L);
      mul2(dinv, U, G);
      store4<T>(&lg[4 * (size_t)k], G);
      mul2(L, G, LG);
      Dp[0] = 1.0 - LG[0];
      Dp[1] = -LG[1];
      Dp[2] = -LG[2];
      Dp[3] = 1.0 - LG[3];
      inv2<T>(Dp, Dn);
      mul2(Dn, L, A);
      A[0] = -A[0];
      A[1] = -A[1];
      A[2] = -A[2];
      A[3] = -A[3];
      k++;
      store4<T>(&ldinv[4 * (size_t)k], Dn);
      store4<T>(&la[4 * (size_t)k], A);
      dinv[0] = Dn[0];
      dinv[1] = Dn[1];
      dinv[2] = Dn[2];
      dinv[3] = Dn[3];
      len++;
    }
    store4<T>(&lg[4 * (size_t)k], zero);
    d.line_len[l] = len;
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
  if (fp32)
    k_assemble<float, kLPR><<<grid, kAsmBlk, 0, c.stream>>>(d, F, dt, p_scale, debug);
  else
    k_assemble<double, kLPR><<<grid, kAsmBlk, 0, c.stream>>>(d, F, dt, p_scale, debug);
  return cudaGetLastError();
}

cudaError_t launch_line_setup(const Dev& d, int fp32, LaunchCfg c) {
  cudaError_t e = cudaMemsetAsync(&d.ctr->n_lines, 0, sizeof(int), c.stream);
  if (e != cudaSuccess) return e;
  k_line_mark<<<4 * c.sms, 256, 0, c.stream>>>(d);
  if (fp32)
    k_line_factor<float><<<c.sms, 128, 0, c.stream>>>(d);
  else
    k_line_factor<double><<<c.sms, 128, 0, c.stream>>>(d);
  return cudaGetLastError();
}

}  // namespace lns
