// k_krylov.cu -- BiCGStab on the compacted local system J_A du_A = -F_A (Section 4.3),
// right-preconditioned by block Jacobi whose blocks are single cells (already the identity
// after the assembly's row scaling) and whole fracture segments (block tridiagonal).
//
// One persistent cooperative launch runs the whole Krylov loop; grid-wide barriers
// separate the phases of an iteration (5 per iteration).  Dot products are reduced per
// block into fixed slots and every block sums the slots in the same order, so all blocks
// hold identical scalars and the result does not depend on scheduling.
//
// Matrix-vector product: one thread per compact row, the row's 2x2 blocks are contiguous
// at its CSR entries; columns outside V_A carry colA = -1 and are skipped.
// Line solves: one warp per fracture segment, the two recurrences of the block Thomas
// algorithm evaluated as inclusive scans of 2x2 affine maps (log2(32) shuffle steps per
// 32 rows, carried across chunks of 32).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "lns_internal.cuh"

namespace cg = cooperative_groups;

namespace lns {

namespace {

constexpr int kKryBlk = 512;

template <typename T>
struct V2;
template <>
struct V2<float> {
  using t = float2;
};
template <>
struct V2<double> {
  using t = double2;
};

template <typename T>
struct alignas(4 * sizeof(T)) B4 {
  T a, b, c, d;
};

// Vectors are rewritten by other blocks between grid barriers: read them through L2.
__device__ __forceinline__ float2 ldv(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldv(const double2* p) { return __ldcg(p); }

template <typename T>
__device__ __forceinline__ typename V2<T>::t mk(T x, T y) {
  typename V2<T>::t v;
  v.x = x;
  v.y = y;
  return v;
}

// Block-reduce up to two doubles into partial slots (slot, slot+1) of this block.  Only the
// first `nw` warps hold rows; the others skip the FP64 shuffles (FP64 issues slowly here).
__device__ __forceinline__ void block_store2(double a, double b, double* sh, double* part, int slot, int nb, int nw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < nw) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      sh[2 * w] = a;
      sh[2 * w + 1] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < nw; k++) {
      sa += sh[2 * k];
      sb += sh[2 * k + 1];
    }
    part[(size_t)slot * nb + blockIdx.x] = sa;
    part[(size_t)(slot + 1) * nb + blockIdx.x] = sb;
  }
  __syncthreads();
}

// Sum partial slots (slot, slot+1) over all blocks in a fixed order; every block gets the
// same two numbers.
__device__ __forceinline__ void grid_sum2(const double* part, int slot, int nb, double* sh, double& ra, double& rb) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += 32) {
      a += __ldcg(&part[(size_t)slot * nb + k]);
      b += __ldcg(&part[(size_t)(slot + 1) * nb + k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      sh[64] = a;
      sh[65] = b;
    }
  }
  __syncthreads();
  ra = sh[64];
  rb = sh[65];
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ typename V2<T>::t spmv_row(const Dev& d, int k, const typename V2<T>::t* __restrict__ xv,
                                                      const T* __restrict__ blocks) {
  using V = typename V2<T>::t;
  const int i = d.act[k];
  V y = ldv(&xv[k]);  // identity diagonal
  const int e1 = d.row_ptr[i + 1];
  for (int e = d.row_ptr[i]; e < e1; e++) {
    const int c = d.colA[e];
    if (c < 0) continue;
    const B4<T> bk = *(const B4<T>*)&blocks[4 * (size_t)e];
    const V xc = ldv(&xv[c]);
    y.x += bk.a * xc.x + bk.b * xc.y;
    y.y += bk.c * xc.x + bk.d * xc.y;
  }
  return y;
}

// 2x2 helpers in T
template <typename T>
struct M2 {
  T a, b, c, d;
};
template <typename T>
__device__ __forceinline__ M2<T> mm(const M2<T>& x, const M2<T>& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
template <typename T>
__device__ __forceinline__ typename V2<T>::t mv(const M2<T>& x, const typename V2<T>::t& v) {
  return mk<T>(x.a * v.x + x.b * v.y, x.c * v.x + x.d * v.y);
}
template <typename T>
__device__ __forceinline__ M2<T> ld2(const T* p) {
  const B4<T> b = *(const B4<T>*)p;
  return {b.a, b.b, b.c, b.d};
}

// Apply M^{-1} to one fracture line (rows k0 .. k0+len-1) by one warp, in FP32.  The input
// vector is produced per row by `make(k)` (the warp also stores it); the result goes to dst.
// Forward: w_t = Dinv_t src_t + A_t w_{t-1}; backward: z_t = w_t - G_t z_{t+1}; both as
// inclusive scans of 2x2 affine maps, carried across chunks of 32 rows.
__device__ __forceinline__ float4 ldf4(const float* p) { return *(const float4*)p; }

template <typename T, typename MakeF>
__device__ __forceinline__ void line_apply(const Dev& d, int k0, int len, typename V2<T>::t* __restrict__ dst,
                                           MakeF make) {
  using V = typename V2<T>::t;
  const int lane = threadIdx.x & 31;
  const float* ldinv = (const float*)d.line_dinv;
  const float* la = (const float*)d.line_a;
  const float* lg = (const float*)d.line_g;
  float2 carry = make_float2(0.f, 0.f);
  for (int base = 0; base < len; base += 32) {
    const int t = base + lane;
    const bool valid = t < len;
    M2<float> A = {0.f, 0.f, 0.f, 0.f};
    float2 c = make_float2(0.f, 0.f);
    if (valid) {
      const int k = k0 + t;
      const V s = make(k);
      const float4 Di = ldf4(&ldinv[4 * (size_t)k]);
      const float sx = (float)s.x, sy = (float)s.y;
      c = make_float2(Di.x * sx + Di.y * sy, Di.z * sx + Di.w * sy);
      const float4 a4 = ldf4(&la[4 * (size_t)k]);
      A = {a4.x, a4.y, a4.z, a4.w};
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      M2<float> Ap;
      float2 cp;
      Ap.a = __shfl_up_sync(0xffffffffu, A.a, o);
      Ap.b = __shfl_up_sync(0xffffffffu, A.b, o);
      Ap.c = __shfl_up_sync(0xffffffffu, A.c, o);
      Ap.d = __shfl_up_sync(0xffffffffu, A.d, o);
      cp.x = __shfl_up_sync(0xffffffffu, c.x, o);
      cp.y = __shfl_up_sync(0xffffffffu, c.y, o);
      if (lane >= o) {
        c.x += A.a * cp.x + A.b * cp.y;
        c.y += A.c * cp.x + A.d * cp.y;
        A = mm(A, Ap);
      }
    }
    const float2 w = make_float2(c.x + A.a * carry.x + A.b * carry.y, c.y + A.c * carry.x + A.d * carry.y);
    if (valid) dst[k0 + t] = mk<T>((T)w.x, (T)w.y);
    const int last = min(31, len - 1 - base);
    carry.x = __shfl_sync(0xffffffffu, w.x, last);
    carry.y = __shfl_sync(0xffffffffu, w.y, last);
  }
  __syncwarp();
  carry = make_float2(0.f, 0.f);
  const int nchunk = (len + 31) / 32;
  for (int ch = nchunk - 1; ch >= 0; ch--) {
    const int t = ch * 32 + lane;
    const bool valid = t < len;
    M2<float> B = {0.f, 0.f, 0.f, 0.f};
    float2 c = make_float2(0.f, 0.f);
    if (valid) {
      const int k = k0 + t;
      const V wv = ldv(&dst[k]);
      c = make_float2((float)wv.x, (float)wv.y);
      const float4 g4 = ldf4(&lg[4 * (size_t)k]);
      B = {-g4.x, -g4.y, -g4.z, -g4.w};
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      M2<float> Bp;
      float2 cp;
      Bp.a = __shfl_down_sync(0xffffffffu, B.a, o);
      Bp.b = __shfl_down_sync(0xffffffffu, B.b, o);
      Bp.c = __shfl_down_sync(0xffffffffu, B.c, o);
      Bp.d = __shfl_down_sync(0xffffffffu, B.d, o);
      cp.x = __shfl_down_sync(0xffffffffu, c.x, o);
      cp.y = __shfl_down_sync(0xffffffffu, c.y, o);
      if (lane + o < 32) {
        c.x += B.a * cp.x + B.b * cp.y;
        c.y += B.c * cp.x + B.d * cp.y;
        B = mm(B, Bp);
      }
    }
    const float2 z = make_float2(c.x + B.a * carry.x + B.b * carry.y, c.y + B.c * carry.x + B.d * carry.y);
    if (valid) dst[k0 + t] = mk<T>((T)z.x, (T)z.y);
    carry.x = __shfl_sync(0xffffffffu, z.x, 0);
    carry.y = __shfl_sync(0xffffffffu, z.y, 0);
  }
  __syncwarp();
}

template <typename T, bool LINES>
__global__ void __launch_bounds__(kKryBlk, 1) k_bicgstab(Dev d, double rtol, int maxit) {
  using V = typename V2<T>::t;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[72];
  const int nA = d.ctr->n_active;
  const int nb = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int gwarp = tid >> 5, nwarps = nth >> 5;
  // rows: a contiguous chunk per block, spread over all SMs (FP64 throughput is per SM)
  const int rpb = (nA + nb - 1) / nb;
  const int r0 = min(nA, blockIdx.x * rpb), r1 = min(nA, r0 + rpb);
  const int kbeg = r0 + (int)threadIdx.x, kstep = blockDim.x;
  const int nw = min((int)(blockDim.x >> 5), (r1 - r0 + 31) / 32);
  const int nlines = LINES ? d.ctr->n_lines : 0;
  // (s, s) also collects the line rows' contributions from the line warps: every warp may hold some
  const int nw_ss = LINES ? (int)(blockDim.x >> 5) : nw;
  V* x = (V*)d.kx;
  V* r = (V*)d.kr;
  V* rh = (V*)d.krh;
  V* p = (V*)d.kp;
  V* v = (V*)d.kv;
  V* s = (V*)d.ks;
  V* t = (V*)d.kt;
  V* ph = LINES ? (V*)d.kph : p;
  V* shv = LINES ? (V*)d.ksh : s;
  const V* b = (const V*)d.rhs;
  const T* blocks = (const T*)d.blocks;
  const int* lflag = d.line_row_flag;
  double* part = d.partials;

  double l_bb = 0.0;
  for (int k = kbeg; k < r1; k += kstep) {
    const V bk = b[k];
    x[k] = mk<T>(0, 0);
    r[k] = bk;
    rh[k] = bk;
    p[k] = mk<T>(0, 0);
    v[k] = mk<T>(0, 0);
    l_bb += (double)bk.x * bk.x + (double)bk.y * bk.y;
  }
  block_store2(l_bb, 0.0, sh, part, 0, nb, nw);
  grid.sync();
  double bb, dummy;
  grid_sum2(part, 0, nb, sh, bb, dummy);
  int status = 0, it = 0;
  double relres = 0.0;
  if (bb > 0.0) {
    const double stop2 = rtol * rtol * bb;
    double rho = bb, rho_old = 1.0, alpha = 1.0, omega = 1.0;
    status = 1;
    for (it = 1; it <= maxit; it++) {
      const T beta = (T)(it == 1 ? 0.0 : (rho / rho_old) * (alpha / omega));
      const T om = (T)omega;
      // Phase A: p = r + beta (p - omega v);  ph = M^{-1} p
      for (int k = kbeg; k < r1; k += kstep) {
        if (LINES && lflag[k]) continue;
        const V rk = ldv(&r[k]), pk = ldv(&p[k]), vk = ldv(&v[k]);
        const V np = mk<T>(rk.x + beta * (pk.x - om * vk.x), rk.y + beta * (pk.y - om * vk.y));
        p[k] = np;
        if (LINES) ph[k] = np;
      }
      if (LINES)
        for (int l = gwarp; l < nlines; l += nwarps) {
          line_apply<T>(d, d.line_start[l], d.line_len[l], ph, [&](int k) {
            const V rk = ldv(&r[k]), pk = ldv(&p[k]), vk = ldv(&v[k]);
            const V np = mk<T>(rk.x + beta * (pk.x - om * vk.x), rk.y + beta * (pk.y - om * vk.y));
            p[k] = np;
            return np;
          });
        }
      grid.sync();
      // Phase B: v = A ph, (rh, v)
      double l_rv = 0.0;
      for (int k = kbeg; k < r1; k += kstep) {
        const V vk = spmv_row<T>(d, k, ph, blocks);
        v[k] = vk;
        const V rk = ldv(&rh[k]);
        l_rv += (double)rk.x * vk.x + (double)rk.y * vk.y;
      }
      block_store2(l_rv, 0.0, sh, part, 2, nb, nw);
      grid.sync();
      double rv;
      grid_sum2(part, 2, nb, sh, rv, dummy);
      if (rv == 0.0 || !isfinite(rv)) {
        status = 2;
        break;
      }
      alpha = rho / rv;
      const T al = (T)alpha;
      // Phase C: s = r - alpha v; shv = M^{-1} s; (s, s)
      double l_ss = 0.0;
      for (int k = kbeg; k < r1; k += kstep) {
        if (LINES && lflag[k]) continue;
        const V rk = ldv(&r[k]), vk = ldv(&v[k]);
        const V sk = mk<T>(rk.x - al * vk.x, rk.y - al * vk.y);
        s[k] = sk;
        if (LINES) shv[k] = sk;
        l_ss += (double)sk.x * sk.x + (double)sk.y * sk.y;
      }
      if (LINES)
        for (int l = gwarp; l < nlines; l += nwarps) {
          double acc = 0.0;
          line_apply<T>(d, d.line_start[l], d.line_len[l], shv, [&](int k) {
            const V rk = ldv(&r[k]), vk = ldv(&v[k]);
            const V sk = mk<T>(rk.x - al * vk.x, rk.y - al * vk.y);
            s[k] = sk;
            acc += (double)sk.x * sk.x + (double)sk.y * sk.y;
            return sk;
          });
          l_ss += acc;
        }
      block_store2(l_ss, 0.0, sh, part, 4, nb, nw_ss);
      grid.sync();
      double ss;
      grid_sum2(part, 4, nb, sh, ss, dummy);
      if (ss <= stop2) {
        for (int k = kbeg; k < r1; k += kstep) {
          const V xk = ldv(&x[k]), pk = ldv(&ph[k]);
          x[k] = mk<T>(xk.x + al * pk.x, xk.y + al * pk.y);
        }
        relres = sqrt(ss / bb);
        status = 0;
        break;
      }
      // Phase D: t = A shv; (t, s), (t, t)
      double l_ts = 0.0, l_tt = 0.0;
      for (int k = kbeg; k < r1; k += kstep) {
        const V tk = spmv_row<T>(d, k, shv, blocks);
        t[k] = tk;
        const V sk = ldv(&s[k]);
        l_ts += (double)tk.x * sk.x + (double)tk.y * sk.y;
        l_tt += (double)tk.x * tk.x + (double)tk.y * tk.y;
      }
      block_store2(l_ts, l_tt, sh, part, 6, nb, nw);
      grid.sync();
      double ts, tt;
      grid_sum2(part, 6, nb, sh, ts, tt);
      if (tt == 0.0 || !isfinite(tt)) {
        status = 2;
        break;
      }
      omega = ts / tt;
      const T omg = (T)omega;
      // Phase E: x += alpha ph + omega shv; r = s - omega t; (rh, r), (r, r)
      double l_rr = 0.0, l_rhr = 0.0;
      for (int k = kbeg; k < r1; k += kstep) {
        const V xk = ldv(&x[k]), pk = ldv(&ph[k]), sk2 = ldv(&shv[k]), sk = ldv(&s[k]), tk = ldv(&t[k]), rhk = ldv(&rh[k]);
        x[k] = mk<T>(xk.x + al * pk.x + omg * sk2.x, xk.y + al * pk.y + omg * sk2.y);
        const V rk = mk<T>(sk.x - omg * tk.x, sk.y - omg * tk.y);
        r[k] = rk;
        l_rr += (double)rk.x * rk.x + (double)rk.y * rk.y;
        l_rhr += (double)rhk.x * rk.x + (double)rhk.y * rk.y;
      }
      block_store2(l_rhr, l_rr, sh, part, 0, nb, nw);
      grid.sync();
      double rr;
      rho_old = rho;
      grid_sum2(part, 0, nb, sh, rho, rr);
      relres = sqrt(rr / bb);
      if (rr <= stop2) {
        status = 0;
        break;
      }
      if (rho == 0.0 || omega == 0.0 || !isfinite(rho)) {
        status = 2;
        break;
      }
    }
    if (it > maxit) it = maxit;
  } else {
    for (int k = kbeg; k < r1; k += kstep) x[k] = mk<T>(0, 0);
  }
  if (tid == 0) {
    d.ctr->krylov_iters = it;
    d.ctr->krylov_status = status;
    d.ctr->krylov_relres = relres;
  }
}

template <typename T, bool L>
int max_blocks(int sms) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab<T, L>, kKryBlk, 0);
  if (nb > 2) nb = 2;
  if (nb < 1) nb = 1;
  return nb * sms;
}

}  // namespace

int krylov_grid(int fp32, int sms) {
  int a = fp32 ? max_blocks<float, true>(sms) : max_blocks<double, true>(sms);
  int b = fp32 ? max_blocks<float, false>(sms) : max_blocks<double, false>(sms);
  return a < b ? a : b;
}

cudaError_t launch_bicgstab(const Dev& d, int fp32, int lines, double rtol, int maxit, int grid, LaunchCfg c) {
  Dev dd = d;
  void* args[] = {&dd, &rtol, &maxit};
  count_launches(1);
  void* fn = fp32 ? (lines ? (void*)k_bicgstab<float, true> : (void*)k_bicgstab<float, false>)
                  : (lines ? (void*)k_bicgstab<double, true> : (void*)k_bicgstab<double, false>);
  return cudaLaunchCooperativeKernel(fn, grid, kKryBlk, args, 0, c.stream);
}

}  // namespace lns
