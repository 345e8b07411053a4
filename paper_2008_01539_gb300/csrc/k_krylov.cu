// k_krylov.cu -- BiCGStab on the compacted local system J_A du_A = -F_A (Section 4.3),
// right-preconditioned by block Jacobi whose blocks are single cells (already the identity
// after the assembly's row scaling) and whole fracture segments (block tridiagonal).
//
// One persistent cooperative launch runs the whole Krylov loop; grid-wide barriers separate
// the five phases of an iteration.  Dot products are reduced per block into fixed slots and
// every block sums the slots in the same order, so all blocks hold identical scalars, take
// the same branches, and the result does not depend on scheduling.
//
// The local systems of the localized method are small (thousands of rows), so an iteration
// is bound by latency, not bandwidth.  Each phase is kept to one level of L2 round trips:
//  - rows are contiguous chunks spread over all SMs; the columns and blocks of a block's rows,
//    and the factors of its fracture lines (line l lives in block l mod gridDim), are staged
//    in shared memory once per solve (read-only data does not survive in L1 across grid
//    barriers); the partial sums of a reduction are loaded all at once;
//  - the product's gathers of the preconditioned vector are issued several at a time;
//  - a fracture line (one warp) loads all of its rows at once, runs the forward and backward
//    block-Thomas recurrences as FP32 scans of 2x2 affine maps in registers, and stores once.
// Vectors written by other blocks between barriers are read through L2 (__ldcg).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "lns_internal.cuh"

namespace cg = cooperative_groups;

namespace lns {

namespace {

constexpr int kKryBlk = 512;
constexpr int kRowsCached = 2;   // rows per thread whose CSR bounds stay in registers
constexpr int kLineChunks = 4;   // 32-row chunks a line warp holds in registers (longer lines: chunked path)

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

__device__ __forceinline__ float2 ldv(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldv(const double2* p) { return __ldcg(p); }

__device__ __forceinline__ float4 ldf4(const float* p) { return __ldg((const float4*)p); }

template <typename T>
__device__ __forceinline__ typename V2<T>::t mk(T x, T y) {
  typename V2<T>::t v;
  v.x = x;
  v.y = y;
  return v;
}

template <typename T>
struct M2 {
  T a, b, c, d;
};
template <typename T>
__device__ __forceinline__ M2<T> mm(const M2<T>& x, const M2<T>& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}

// Block-reduce up to two doubles into partial slots (slot, slot+1) of this block.  Only the
// first `nw` warps hold values; the others skip the FP64 shuffles (FP64 issues slowly here).
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

// Sum partial slots (slot, slot+1) over all blocks in a fixed order (warp 0; the sums are
// valid in thread 0).  Every block computes the same two numbers.  All of a lane's partial
// loads are issued before any is used.
__device__ __forceinline__ void grid_sum2(const double* part, int slot, int nb, double& ra, double& rb) {
  ra = rb = 0.0;
  if (threadIdx.x < 32) {
    constexpr int kU = 8;
    double a = 0.0, b = 0.0;
    for (int base = 0; base < nb; base += 32 * kU) {
      double va[kU], vb[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int k = base + u * 32 + (int)threadIdx.x;
        va[u] = k < nb ? __ldcg(&part[(size_t)slot * nb + k]) : 0.0;
        vb[u] = k < nb ? __ldcg(&part[(size_t)(slot + 1) * nb + k]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; u++) {
        a += va[u];
        b += vb[u];
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    ra = a;
    rb = b;
  }
}

// Reductions inside the iteration are carried in double-float: an unevaluated sum hi + lo of
// two FP32 words, added with Knuth's TwoSum and renormalized (about 48 significant bits).
// Dependent FP64 operations have a long latency on this GPU; the FP32 pipe does the same tree
// several times faster.  Values are first multiplied by an exact power of two near 1/||b||^2 so
// that no partial sum leaves the FP32 range.  Per-row products, vectors and the recurrence
// scalars stay FP64; the summation order is fixed (deterministic).
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float av = __fsub_rn(s, bv);
  const float e = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(b.hi, bv));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Block partials of two scaled values into slots (slot, slot+1), as (hi, lo) pairs.
__device__ __forceinline__ void block_store_df(double a, double b, double scale, float4* sh4, double* part, int slot,
                                               int nb, int nw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < nw) {
    DF da = df_from(a * scale), db = df_from(b * scale);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      da = df_add(da, df_shfl_xor(da, o));
      db = df_add(db, df_shfl_xor(db, o));
    }
    if (lane == 0) sh4[w] = make_float4(da.hi, da.lo, db.hi, db.lo);
  }
  __syncthreads();
  if (w == 0) {
    const float4 v = lane < nw ? sh4[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    DF da = {v.x, v.y}, db = {v.z, v.w};
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {  // nw <= 16 warps per block
      da = df_add(da, df_shfl_xor(da, o));
      db = df_add(db, df_shfl_xor(db, o));
    }
    if (lane == 0) {
      ((float2*)part)[(size_t)slot * nb + blockIdx.x] = make_float2(da.hi, da.lo);
      ((float2*)part)[(size_t)(slot + 1) * nb + blockIdx.x] = make_float2(db.hi, db.lo);
    }
  }
}

// Sum of the block partials of slots (slot, slot+1), unscaled, valid in warp 0.
__device__ __forceinline__ void grid_sum_df(const double* part, int slot, int nb, double inv_scale, double& ra,
                                            double& rb) {
  ra = rb = 0.0;
  if (threadIdx.x < 32) {
    constexpr int kU = 8;
    DF a = {0.f, 0.f}, b = {0.f, 0.f};
    for (int base = 0; base < nb; base += 32 * kU) {
      DF va[kU], vb[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int k = base + u * 32 + (int)threadIdx.x;
        const float2 x = k < nb ? __ldcg(&((const float2*)part)[(size_t)slot * nb + k]) : make_float2(0.f, 0.f);
        const float2 y = k < nb ? __ldcg(&((const float2*)part)[(size_t)(slot + 1) * nb + k]) : make_float2(0.f, 0.f);
        va[u] = {x.x, x.y};
        vb[u] = {y.x, y.y};
      }
#pragma unroll
      for (int h = 1; h < kU; h <<= 1)
#pragma unroll
        for (int u = 0; u + h < kU; u += 2 * h) {
          va[u] = df_add(va[u], va[u + h]);
          vb[u] = df_add(vb[u], vb[u + h]);
        }
      a = df_add(a, va[0]);
      b = df_add(b, vb[0]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = df_add(a, df_shfl_xor(a, o));
      b = df_add(b, df_shfl_xor(b, o));
    }
    ra = ((double)a.hi + (double)a.lo) * inv_scale;
    rb = ((double)b.hi + (double)b.lo) * inv_scale;
  }
}

// y_k = x_k + sum over active columns of the row's scaled blocks (identity diagonal).  The
// row's columns and blocks come from shared memory (staged once per solve) or from global
// memory.  The gathers are issued U at a time (U = 4 for FP32 blocks, 2 for FP64 to stay within
// registers).
template <typename T>
__device__ __forceinline__ typename V2<T>::t spmv_row(const int* col, const B4<T>* blk, int deg, int k,
                                                      const typename V2<T>::t* xv) {
  using V = typename V2<T>::t;
  constexpr int U = sizeof(T) == 8 ? 2 : 4;
  V y = ldv(&xv[k]);
  for (int j = 0; j < deg; j += U) {
    int c[U];
#pragma unroll
    for (int q = 0; q < U; q++) c[q] = (j + q < deg) ? col[j + q] : -1;
    V xc[U];
    B4<T> b[U];
#pragma unroll
    for (int q = 0; q < U; q++)
      if (c[q] >= 0) {
        xc[q] = ldv(&xv[c[q]]);
        b[q] = blk[j + q];
      }
#pragma unroll
    for (int q = 0; q < U; q++)
      if (c[q] >= 0) {
        y.x += b[q].a * xc[q].x + b[q].b * xc[q].y;
        y.y += b[q].c * xc[q].x + b[q].d * xc[q].y;
      }
  }
  return y;
}

// Forward and backward block-Thomas recurrences of one 32-row chunk as FP32 inclusive scans of
// 2x2 affine maps.  fwd: w_t = Dinv_t src_t + A_t w_{t-1};  bwd: z_t = w_t - G_t z_{t+1}.
__device__ __forceinline__ float2 scan_fwd(float2 c, M2<float> A, float2 carry, int lane) {
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
  return make_float2(c.x + A.a * carry.x + A.b * carry.y, c.y + A.c * carry.x + A.d * carry.y);
}

__device__ __forceinline__ float2 scan_bwd(float2 c, M2<float> B, float2 carry, int lane) {
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
  return make_float2(c.x + B.a * carry.x + B.b * carry.y, c.y + B.c * carry.x + B.d * carry.y);
}

// M^{-1} on one fracture line of at most kLineChunks*32 rows, all in registers.  `src[c]` holds
// the input of row k0 + 32c + lane; the result is stored to dst.  Row t's factors are
// fac[t*fs] (D'^{-1}), fac[t*fs + fa] (A) and fac[t*fs + fg] (G): shared memory when staged.
template <typename T>
__device__ __forceinline__ void line_solve_reg(int k0, int len, const float4* fac, int fs, int fa, int fg,
                                               const float2* src, typename V2<T>::t* dst) {
  const int lane = threadIdx.x & 31;
  float2 w[kLineChunks];
  float2 carry = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < kLineChunks; c++) {
    w[c] = make_float2(0.f, 0.f);
    if (c * 32 < len) {
      const int t = c * 32 + lane;
      M2<float> A = {0.f, 0.f, 0.f, 0.f};
      float2 cc = make_float2(0.f, 0.f);
      if (t < len) {
        const float4 Di = fac[(size_t)t * fs];
        cc = make_float2(Di.x * src[c].x + Di.y * src[c].y, Di.z * src[c].x + Di.w * src[c].y);
        const float4 a4 = fac[(size_t)t * fs + fa];
        A = {a4.x, a4.y, a4.z, a4.w};
      }
      w[c] = scan_fwd(cc, A, carry, lane);
      const int last = min(31, len - 1 - c * 32);
      carry.x = __shfl_sync(0xffffffffu, w[c].x, last);
      carry.y = __shfl_sync(0xffffffffu, w[c].y, last);
    }
  }
  carry = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = kLineChunks - 1; c >= 0; c--) {
    if (c * 32 < len) {
      const int t = c * 32 + lane;
      M2<float> B = {0.f, 0.f, 0.f, 0.f};
      float2 cc = make_float2(0.f, 0.f);
      if (t < len) {
        const float4 g4 = fac[(size_t)t * fs + fg];
        B = {-g4.x, -g4.y, -g4.z, -g4.w};
        cc = w[c];
      }
      const float2 z = scan_bwd(cc, B, carry, lane);
      if (t < len) dst[k0 + t] = mk<T>((T)z.x, (T)z.y);
      carry.x = __shfl_sync(0xffffffffu, z.x, 0);
      carry.y = __shfl_sync(0xffffffffu, z.y, 0);
    }
  }
}

// M^{-1} on a line longer than kLineChunks*32 rows: chunk by chunk through memory.  `make(k)`
// produces (and stores) the row's input.
template <typename T, typename MakeF>
__device__ __forceinline__ void line_solve_long(const Dev& d, int k0, int len, typename V2<T>::t* dst, MakeF make) {
  using V = typename V2<T>::t;
  const int lane = threadIdx.x & 31;
  const float* ldinv = (const float*)d.line_dinv;
  const float* la = (const float*)d.line_a;
  const float* lg = (const float*)d.line_g;
  float2 carry = make_float2(0.f, 0.f);
  for (int base = 0; base < len; base += 32) {
    const int t = base + lane;
    M2<float> A = {0.f, 0.f, 0.f, 0.f};
    float2 cc = make_float2(0.f, 0.f);
    if (t < len) {
      const size_t k = (size_t)(k0 + t);
      const V s = make((int)k);
      const float4 Di = ldf4(&ldinv[4 * k]);
      cc = make_float2(Di.x * (float)s.x + Di.y * (float)s.y, Di.z * (float)s.x + Di.w * (float)s.y);
      const float4 a4 = ldf4(&la[4 * k]);
      A = {a4.x, a4.y, a4.z, a4.w};
    }
    const float2 w = scan_fwd(cc, A, carry, lane);
    if (t < len) dst[k0 + t] = mk<T>((T)w.x, (T)w.y);
    const int last = min(31, len - 1 - base);
    carry.x = __shfl_sync(0xffffffffu, w.x, last);
    carry.y = __shfl_sync(0xffffffffu, w.y, last);
  }
  __syncwarp();
  carry = make_float2(0.f, 0.f);
  for (int ch = (len + 31) / 32 - 1; ch >= 0; ch--) {
    const int t = ch * 32 + lane;
    M2<float> B = {0.f, 0.f, 0.f, 0.f};
    float2 cc = make_float2(0.f, 0.f);
    if (t < len) {
      const V wv = ldv(&dst[k0 + t]);
      cc = make_float2((float)wv.x, (float)wv.y);
      const float4 g4 = ldf4(&lg[4 * (size_t)(k0 + t)]);
      B = {-g4.x, -g4.y, -g4.z, -g4.w};
    }
    const float2 z = scan_bwd(cc, B, carry, lane);
    if (t < len) dst[k0 + t] = mk<T>((T)z.x, (T)z.y);
    carry.x = __shfl_sync(0xffffffffu, z.x, 0);
    carry.y = __shfl_sync(0xffffffffu, z.y, 0);
  }
  __syncwarp();
}

// Shared memory of one block: the factors of up to kLineSlots of its lines (3 float4 per row),
// then the columns and blocks of its rows, packed in row order.
constexpr int kLineSlots = 4;
constexpr size_t kLineSmem = (size_t)kLineSlots * kLineChunks * 32 * 3 * sizeof(float4);
constexpr size_t kKrySmem = 200 * 1024;

template <typename T, bool LINES>
__global__ void __launch_bounds__(kKryBlk, 1) k_bicgstab(Dev d, double rtol, int maxit) {
  using V = typename V2<T>::t;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double sh[72];
  __shared__ int s_scan[kKryBlk / 32 + 1];
  const int nA = d.ctr->n_active;
  const int nb = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // rows: a contiguous chunk per block, spread over all SMs (FP64 throughput is per SM)
  const int rpb = (nA + nb - 1) / nb;
  const int r0 = min(nA, blockIdx.x * rpb), r1 = min(nA, r0 + rpb);
  const int kbeg = r0 + (int)threadIdx.x, kstep = blockDim.x;
  const int nw = min((int)(blockDim.x >> 5), (r1 - r0 + 31) / 32);
  const int nlines = LINES ? d.ctr->n_lines : 0;
  // (s, s) also collects the line rows' contributions from the line warps
  const int nw_ss = LINES ? (int)(blockDim.x >> 5) : nw;
  V* __restrict__ x = (V*)d.kx;
  V* __restrict__ r = (V*)d.kr;
  V* __restrict__ rh = (V*)d.krh;
  V* __restrict__ p = (V*)d.kp;
  V* __restrict__ v = (V*)d.kv;
  V* __restrict__ s = (V*)d.ks;
  V* __restrict__ t = (V*)d.kt;
  V* ph = LINES ? (V*)d.kph : p;
  V* shv = LINES ? (V*)d.ksh : s;
  const V* b = (const V*)d.rhs;
  const T* blocks = (const T*)d.blocks;
  const int* lflag = d.line_row_flag;
  double* part = d.partials;
  float4* s_fac = (float4*)dsm;
  const int ecap = (int)((kKrySmem - kLineSmem) / (sizeof(int) + sizeof(B4<T>)));
  B4<T>* s_blk = (B4<T>*)(dsm + kLineSmem);
  int* s_col = (int*)(dsm + kLineSmem + (size_t)ecap * sizeof(B4<T>));

  // Stage the columns and blocks of this thread's first rows in shared memory (packed in row
  // order by a block scan of the row degrees); rows that do not fit read global memory.
  const int* rcol[kRowsCached];
  const B4<T>* rblk[kRowsCached];
  int rdeg[kRowsCached], rfl[kRowsCached];
  int ebase = 0;
#pragma unroll
  for (int q = 0; q < kRowsCached; q++) {
    const int k = kbeg + q * kstep;
    int e0 = 0, deg = 0;
    rfl[q] = 1;
    if (k < r1) {
      const int i = __ldg(&d.act[k]);
      e0 = __ldg(&d.row_ptr[i]);
      deg = __ldg(&d.row_ptr[i + 1]) - e0;
      rfl[q] = LINES ? __ldg(&lflag[k]) : 0;
    }
    // exclusive block scan of deg
    int inc = deg;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_scan[wib] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        const int c = s_scan[w];
        s_scan[w] = acc;
        acc += c;
      }
      s_scan[kKryBlk / 32] = acc;
    }
    __syncthreads();
    const int off = ebase + s_scan[wib] + inc - deg;
    ebase += s_scan[kKryBlk / 32];
    __syncthreads();
    rdeg[q] = deg;
    if (off + deg <= ecap) {
      for (int j = 0; j < deg; j++) {
        s_col[off + j] = __ldg(&d.colA[e0 + j]);
        s_blk[off + j] = *(const B4<T>*)&blocks[4 * (size_t)(e0 + j)];
      }
      rcol[q] = s_col + off;
      rblk[q] = s_blk + off;
    } else {
      rcol[q] = d.colA + e0;
      rblk[q] = (const B4<T>*)&blocks[4 * (size_t)e0];
    }
  }
  // Stage the factors of this block's first kLineSlots lines (line l lives in block l % nb).
  if (LINES)
    for (int j = wib; j < kLineSlots; j += (int)(blockDim.x >> 5)) {
      const int l = (int)blockIdx.x + nb * j;
      if (l >= nlines) continue;
      const int k0 = __ldg(&d.line_start[l]), len = __ldg(&d.line_len[l]);
      if (len > kLineChunks * 32) continue;
      for (int tt = lane; tt < len; tt += 32) {
        const size_t k = (size_t)(k0 + tt);
        float4* dst = &s_fac[((size_t)j * kLineChunks * 32 + tt) * 3];
        dst[0] = ldf4(&((const float*)d.line_dinv)[4 * k]);
        dst[1] = ldf4(&((const float*)d.line_a)[4 * k]);
        dst[2] = ldf4(&((const float*)d.line_g)[4 * k]);
      }
    }
  __syncthreads();
  // visit this thread's rows: fn(k, col, blk, deg, line_flag)
  auto rows = [&](auto fn) {
#pragma unroll
    for (int q = 0; q < kRowsCached; q++) {
      const int k = kbeg + q * kstep;
      if (k < r1) fn(k, rcol[q], rblk[q], rdeg[q], rfl[q]);
    }
    for (int k = kbeg + kRowsCached * kstep; k < r1; k += kstep) {
      const int i = __ldg(&d.act[k]);
      const int e0 = __ldg(&d.row_ptr[i]);
      fn(k, d.colA + e0, (const B4<T>*)&blocks[4 * (size_t)e0], __ldg(&d.row_ptr[i + 1]) - e0,
         LINES ? __ldg(&lflag[k]) : 0);
    }
  };
  // visit this block's lines: fn(k0, len, factors, stride, offA, offG); line l lives in block l % nb
  auto lines = [&](auto fn) {
    for (int j = wib;; j += (int)(blockDim.x >> 5)) {
      const int l = (int)blockIdx.x + nb * j;
      if (l >= nlines) break;
      const int k0 = __ldg(&d.line_start[l]), len = __ldg(&d.line_len[l]);
      if (j < kLineSlots && len <= kLineChunks * 32)
        fn(k0, len, (const float4*)&s_fac[(size_t)j * kLineChunks * 32 * 3], 3, 1, 2);
      else
        fn(k0, len, (const float4*)nullptr, 0, 0, 0);
    }
  };

  // Scalars of the recurrence live in thread 0 (FP64 division and square root are long FP64
  // sequences here: computed once per block, broadcast through shared memory).
  __shared__ double s_bc[6];  // broadcast: beta, omega (phase A), alpha (C..E), omega (E), scale, 1/scale
  __shared__ int s_ctl;       // 0 continue, 1 converged, 2 breakdown
  __shared__ float4 s_df[kKryBlk / 32];
  double l_bb = 0.0;
  rows([&](int k, const int*, const B4<T>*, int, int) {
    const V bk = b[k];
    x[k] = mk<T>(0, 0);
    r[k] = bk;
    rh[k] = bk;
    p[k] = mk<T>(0, 0);
    v[k] = mk<T>(0, 0);
    l_bb += (double)bk.x * bk.x + (double)bk.y * bk.y;
  });
  block_store2(l_bb, 0.0, sh, part, 0, nb, nw);
  grid.sync();
  double bb = 0.0, dummy, rho = 0.0, rho_old = 1.0, alpha = 1.0, omega = 1.0, stop2 = 0.0, relres = 0.0;
  grid_sum2(part, 0, nb, bb, dummy);
  if (threadIdx.x == 0) {
    s_ctl = bb > 0.0 ? 0 : 1;
    rho = bb;
    stop2 = rtol * rtol * bb;
    // exact power of two near 1/bb (biased exponent 2046 - E of bb, clamped to normal range)
    long long e = bb > 0.0 ? ((__double_as_longlong(bb) >> 52) & 0x7ff) : 1023;
    e = e < 1 ? 1 : (e > 2045 ? 2045 : e);
    s_bc[4] = __longlong_as_double((2046 - e) << 52);
    s_bc[5] = __longlong_as_double(e << 52);
  }
  __syncthreads();
  const double dscale = s_bc[4], dinv = s_bc[5];
  int status = 0, it = 0;
  if (s_ctl == 0) {
    status = 1;
    for (it = 1; it <= maxit; it++) {
      if (threadIdx.x == 0) {
        s_bc[0] = it == 1 ? 0.0 : (rho / rho_old) * (alpha / omega);
        s_bc[1] = omega;
      }
      __syncthreads();
      const T beta = (T)s_bc[0];
      const T om = (T)s_bc[1];
      // Phase A: p = r + beta (p - omega v);  ph = M^{-1} p
      rows([&](int k, const int*, const B4<T>*, int, int fl) {
        if (LINES && fl) return;
        const V rk = ldv(&r[k]), pk = ldv(&p[k]), vk = ldv(&v[k]);
        const V np = mk<T>(rk.x + beta * (pk.x - om * vk.x), rk.y + beta * (pk.y - om * vk.y));
        p[k] = np;
        if (LINES) ph[k] = np;
      });
      if (LINES)
        lines([&](int k0, int len, const float4* fac, int fs, int fa, int fg) {
          if (fac) {
            // all of the line's loads first (p, then r and v), then the updates: one L2 round trip
            V pk[kLineChunks];
            float2 src[kLineChunks];
#pragma unroll
            for (int c = 0; c < kLineChunks; c++)
              if (c * 32 + lane < len) pk[c] = ldv(&p[k0 + c * 32 + lane]);
#pragma unroll
            for (int c = 0; c < kLineChunks; c++) {
              src[c] = make_float2(0.f, 0.f);
              if (c * 32 + lane < len) {
                const int k = k0 + c * 32 + lane;
                const V rk = ldv(&r[k]), vk = ldv(&v[k]);
                const V np = mk<T>(rk.x + beta * (pk[c].x - om * vk.x), rk.y + beta * (pk[c].y - om * vk.y));
                p[k] = np;
                src[c] = make_float2((float)np.x, (float)np.y);
              }
            }
            line_solve_reg<T>(k0, len, fac, fs, fa, fg, src, ph);
          } else {
            line_solve_long<T>(d, k0, len, ph, [&](int k) {
              const V rk = ldv(&r[k]), pk = ldv(&p[k]), vk = ldv(&v[k]);
              const V np = mk<T>(rk.x + beta * (pk.x - om * vk.x), rk.y + beta * (pk.y - om * vk.y));
              p[k] = np;
              return np;
            });
          }
        });
      grid.sync();
      // Phase B: v = A ph, (rh, v)
      double l_rv = 0.0;
      rows([&](int k, const int* col, const B4<T>* blk, int deg, int) {
        const V rhk = ldv(&rh[k]);
        const V vk = spmv_row<T>(col, blk, deg, k, ph);
        v[k] = vk;
        l_rv += (double)rhk.x * vk.x + (double)rhk.y * vk.y;
      });
      block_store_df(l_rv, 0.0, dscale, s_df, part, 2, nb, nw);
      grid.sync();
      {
        double rv;
        grid_sum_df(part, 2, nb, dinv, rv, dummy);
        if (threadIdx.x == 0) {
          if (rv == 0.0 || !isfinite(rv)) {
            s_ctl = 2;
          } else {
            alpha = rho / rv;
            s_bc[2] = alpha;
          }
        }
      }
      __syncthreads();
      if (s_ctl == 2) {
        status = 2;
        break;
      }
      const T al = (T)s_bc[2];
      // Phase C: s = r - alpha v; shv = M^{-1} s; (s, s)
      double l_ss = 0.0;
      rows([&](int k, const int*, const B4<T>*, int, int fl) {
        if (LINES && fl) return;
        const V rk = ldv(&r[k]), vk = ldv(&v[k]);
        const V sk = mk<T>(rk.x - al * vk.x, rk.y - al * vk.y);
        s[k] = sk;
        if (LINES) shv[k] = sk;
        l_ss += (double)sk.x * sk.x + (double)sk.y * sk.y;
      });
      if (LINES)
        lines([&](int k0, int len, const float4* fac, int fs, int fa, int fg) {
          if (fac) {
            float2 src[kLineChunks];
#pragma unroll
            for (int c = 0; c < kLineChunks; c++) {
              src[c] = make_float2(0.f, 0.f);
              if (c * 32 + lane < len) {
                const int k = k0 + c * 32 + lane;
                const V rk = ldv(&r[k]), vk = ldv(&v[k]);
                const V sk = mk<T>(rk.x - al * vk.x, rk.y - al * vk.y);
                s[k] = sk;
                l_ss += (double)sk.x * sk.x + (double)sk.y * sk.y;
                src[c] = make_float2((float)sk.x, (float)sk.y);
              }
            }
            line_solve_reg<T>(k0, len, fac, fs, fa, fg, src, shv);
          } else {
            double acc = 0.0;
            line_solve_long<T>(d, k0, len, shv, [&](int k) {
              const V rk = ldv(&r[k]), vk = ldv(&v[k]);
              const V sk = mk<T>(rk.x - al * vk.x, rk.y - al * vk.y);
              s[k] = sk;
              acc += (double)sk.x * sk.x + (double)sk.y * sk.y;
              return sk;
            });
            l_ss += acc;
          }
        });
      block_store_df(l_ss, 0.0, dscale, s_df, part, 4, nb, nw_ss);
      grid.sync();
      {
        double ss;
        grid_sum_df(part, 4, nb, dinv, ss, dummy);
        if (threadIdx.x == 0 && ss <= stop2) {
          s_ctl = 1;
          relres = sqrt(ss / bb);
        }
      }
      __syncthreads();
      if (s_ctl == 1) {
        rows([&](int k, const int*, const B4<T>*, int, int) {
          const V xk = ldv(&x[k]), pk = ldv(&ph[k]);
          x[k] = mk<T>(xk.x + al * pk.x, xk.y + al * pk.y);
        });
        status = 0;
        break;
      }
      // Phase D: t = A shv; (t, s), (t, t)
      double l_ts = 0.0, l_tt = 0.0;
      rows([&](int k, const int* col, const B4<T>* blk, int deg, int) {
        const V sk = ldv(&s[k]);
        const V tk = spmv_row<T>(col, blk, deg, k, shv);
        t[k] = tk;
        l_ts += (double)tk.x * sk.x + (double)tk.y * sk.y;
        l_tt += (double)tk.x * tk.x + (double)tk.y * tk.y;
      });
      block_store_df(l_ts, l_tt, dscale, s_df, part, 6, nb, nw);
      grid.sync();
      {
        double ts, tt;
        grid_sum_df(part, 6, nb, dinv, ts, tt);
        if (threadIdx.x == 0) {
          if (tt == 0.0 || !isfinite(tt)) {
            s_ctl = 2;
          } else {
            omega = ts / tt;
            s_bc[3] = omega;
          }
        }
      }
      __syncthreads();
      if (s_ctl == 2) {
        status = 2;
        break;
      }
      const T omg = (T)s_bc[3];
      // Phase E: x += alpha ph + omega shv; r = s - omega t; (rh, r), (r, r)
      double l_rr = 0.0, l_rhr = 0.0;
      rows([&](int k, const int*, const B4<T>*, int, int) {
        const V xk = ldv(&x[k]), pk = ldv(&ph[k]), sk2 = ldv(&shv[k]), sk = ldv(&s[k]), tk = ldv(&t[k]),
                rhk = ldv(&rh[k]);
        x[k] = mk<T>(xk.x + al * pk.x + omg * sk2.x, xk.y + al * pk.y + omg * sk2.y);
        const V rk = mk<T>(sk.x - omg * tk.x, sk.y - omg * tk.y);
        r[k] = rk;
        l_rr += (double)rk.x * rk.x + (double)rk.y * rk.y;
        l_rhr += (double)rhk.x * rk.x + (double)rhk.y * rk.y;
      });
      block_store_df(l_rhr, l_rr, dscale, s_df, part, 0, nb, nw);
      grid.sync();
      {
        double rr, rhr;
        grid_sum_df(part, 0, nb, dinv, rhr, rr);
        if (threadIdx.x == 0) {
          rho_old = rho;
          rho = rhr;
          relres = sqrt(rr / bb);
          if (rr <= stop2)
            s_ctl = 1;
          else if (rho == 0.0 || omega == 0.0 || !isfinite(rho))
            s_ctl = 2;
        }
      }
      __syncthreads();
      if (s_ctl == 1) {
        status = 0;
        break;
      }
      if (s_ctl == 2) {
        status = 2;
        break;
      }
    }
    if (it > maxit) it = maxit;
  } else {
    rows([&](int k, const int*, const B4<T>*, int, int) { x[k] = mk<T>(0, 0); });
  }
  if (tid == 0) {  // thread 0 of block 0 holds the scalars
    d.ctr->krylov_iters = it;
    d.ctr->krylov_status = status;
    d.ctr->krylov_relres = relres;
  }
}

template <typename T, bool L>
int max_blocks(int sms) {
  int nb = 0;
  cudaFuncSetAttribute(k_bicgstab<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKrySmem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab<T, L>, kKryBlk, kKrySmem);
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
  return cudaLaunchCooperativeKernel(fn, grid, kKryBlk, args, kKrySmem, c.stream);
}

}  // namespace lns
