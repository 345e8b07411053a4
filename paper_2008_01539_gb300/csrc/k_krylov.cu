// k_krylov.cu -- BiCGStab on the compacted local system J_A du_A = -F_A (Section 4.3),
// right-preconditioned by block Jacobi whose blocks are single cells (already the identity
// after the assembly's row scaling) and fracture segments (block tridiagonal, cut into blocks of
// at most 128 rows when factored).
//
// One persistent cooperative launch runs the whole Krylov loop with TWO grid-wide barriers per
// iteration.  The local systems are small (thousands of rows), so an iteration is bound by
// latency: barriers, L2 round trips and dependent FP64 chains, not bandwidth.
//
// Preconditioned vectors are carried through the recurrence by linearity of M^{-1}
// (y = M^{-1} p, z = M^{-1} s, v~ = M^{-1} v, t~ = M^{-1} t, z^ = M^{-1} s applied directly):
//   r~_{i-1} = z^_{i-1} - omega_{i-1} t~_{i-1}                 (= M^{-1} r_{i-1})
//   y_i      = r~_{i-1} + beta_i (y_{i-1} - omega_{i-1} v~_{i-1})
//   z_i      = r~_{i-1} - alpha_i v~_i
// so the preconditioner is applied only right after a product, by the owner of the rows (a
// fracture line's warp), and the products' neighbour values are formed on the fly from vectors
// written before the last barrier:
//   phase 1: x_{i-1}, r_{i-1}, r~_{i-1}, y_i, v = A y_i, v~ = M^{-1} v;  reduce (r^,v), (r,r)
//   phase 2: s = r - alpha v, z_i, t = A z_i, [z^, t~] = M^{-1} [s, t];
//            reduce (t,s), (t,t), (r^,s), (r^,t)   ->  omega, rho_{i+1} = (r^,s) - omega (r^,t), beta
// The owner and every neighbour evaluate y and z with the same fused operations on the same
// stored values, so each row of v (and t) is the product of one consistent vector with A, and the
// recurrence residual stays the true residual of x up to FP64 rounding.  r~ is rebuilt each
// iteration from the directly preconditioned s, so the FP32 rounding of M^{-1} does not accumulate.
//
// Ownership: non-line rows go to threads in contiguous chunks spread over all SMs; the rows of a
// fracture line block go to one warp (line l lives in block l mod gridDim), lane t holding rows
// t, t+32, t+64, t+96.  Matrix rows (columns and blocks) and line factors are staged in shared
// memory once per solve.  Reductions: per-row products in FP64; across lanes, warps and blocks in
// double-float (two FP32 words, Knuth's TwoSum), after scaling by an exact power of two near
// 1/||b||^2.  Every block sums the block partials in the same order, so all blocks hold identical
// scalars (computed once per block by thread 0: FP64 division is a long sequence here).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "lns_internal.cuh"

namespace cg = cooperative_groups;

namespace lns {

namespace {

constexpr int kKryBlk = 256;
constexpr int kWarps = kKryBlk / 32;
constexpr int kRowsCached = 4;   // non-line rows per thread whose matrix row is staged
constexpr int kLineChunks = kLineBlockRows / 32;  // 32-row chunks of a line block
constexpr int kLineSlots = 4;    // line blocks per block whose factors are staged in shared memory
constexpr size_t kLineSmem = (size_t)kLineSlots * kLineChunks * 32 * 3 * sizeof(float4);
constexpr size_t kKrySmem = 200 * 1024;
constexpr int kSlotS1 = 0, kSlotS2 = 2, kSlotInit = 6;  // partial-sum slots (nb entries each)

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

template <typename T>
__device__ __forceinline__ typename V2<T>::t mk(T x, T y) {
  typename V2<T>::t v;
  v.x = x;
  v.y = y;
  return v;
}

// a * b + c, one rounding (explicit, so that every evaluation of a shared formula is identical)
__device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }

// u + a w, componentwise, fused
template <typename V, typename T>
__device__ __forceinline__ V axpy(T a, V w, V u) {
  V o;
  o.x = fm(a, w.x, u.x);
  o.y = fm(a, w.y, u.y);
  return o;
}

template <typename T>
struct M2 {
  T a, b, c, d;
};
template <typename T>
__device__ __forceinline__ M2<T> mm(const M2<T>& x, const M2<T>& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}

// ---- reductions --------------------------------------------------------------------------
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

// Dot products of one thread's rows.  FP64 vectors: fused FP64 products, converted to double-float
// (after scaling) once per phase.  FP32 vectors: exact FP32 products (p + e, e = fma(a, b, -p))
// summed in double-float, so the FP32 path issues no FP64 instruction per row.
template <typename T>
struct DotAcc {
  using t = double;
};
template <>
struct DotAcc<float> {
  using t = DF;
};
__device__ __forceinline__ void dot_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void dot_zero(DF& a) { a = DF{0.f, 0.f}; }
__device__ __forceinline__ void dot_acc(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void dot_acc(DF& acc, float a, float b) {
  const float p = a * b;
  acc = df_add(acc, DF{p, fmaf(a, b, -p)});
}
__device__ __forceinline__ DF dot_df(double acc, double scale) { return df_from(acc * scale); }
__device__ __forceinline__ DF dot_df(DF acc, double) { return acc; }

// Block partials of NV values into slots [slot, slot+NV) as (hi, lo) pairs.  Warps with nothing
// to add (busy == false) contribute zeros without converting.  Contains one block barrier.
template <int NV>
__device__ __forceinline__ void block_store(const DF (&vals)[NV], bool busy, DF* sdf, double* part, int slot, int nb) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  DF a[NV];
#pragma unroll
  for (int q = 0; q < NV; q++) a[q] = busy ? vals[q] : DF{0.f, 0.f};
  if (busy) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; q++) a[q] = df_add(a[q], df_shfl_xor(a[q], o));
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; q++) sdf[q * kWarps + w] = a[q];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) a[q] = lane < kWarps ? sdf[q * kWarps + lane] : DF{0.f, 0.f};
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; q++) a[q] = df_add(a[q], df_shfl_xor(a[q], o));
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; q++)
        ((float2*)part)[(size_t)(slot + q) * nb + blockIdx.x] = make_float2(a[q].hi, a[q].lo);
  }
}

// Sum over all blocks of slots [slot, slot+NV), unscaled, in a fixed order; valid in warps 0 and
// 1 (both compute it, so that two threads can share the scalar work).  All of a lane's partial
// loads of one pass are issued before any is used.
template <int NV>
__device__ __forceinline__ void grid_sum(const double* part, int slot, int nb, double inv_scale, double (&out)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; q++) out[q] = 0.0;
  if (threadIdx.x >= 64) return;
  const int ln = threadIdx.x & 31;
  constexpr int kU = 5;
  DF a[NV];
#pragma unroll
  for (int q = 0; q < NV; q++) a[q] = {0.f, 0.f};
  for (int base = 0; base < nb; base += 32 * kU) {
    DF v[NV][kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int k = base + u * 32 + ln;
#pragma unroll
      for (int q = 0; q < NV; q++) {
        const float2 x = k < nb ? __ldcg(&((const float2*)part)[(size_t)(slot + q) * nb + k]) : make_float2(0.f, 0.f);
        v[q][u] = {x.x, x.y};
      }
    }
#pragma unroll
    for (int h = 1; h < kU; h <<= 1)
#pragma unroll
      for (int u = 0; u + h < kU; u += 2 * h)
#pragma unroll
        for (int q = 0; q < NV; q++) v[q][u] = df_add(v[q][u], v[q][u + h]);
#pragma unroll
    for (int q = 0; q < NV; q++) a[q] = df_add(a[q], v[q][0]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NV; q++) a[q] = df_add(a[q], df_shfl_xor(a[q], o));
#pragma unroll
  for (int q = 0; q < NV; q++) out[q] = ((double)a[q].hi + (double)a[q].lo) * inv_scale;
}

// ||b||^2 (once per solve, before the scale is known): FP64 block partial and grid sum.
__device__ __forceinline__ void block_store_f64(double a, double* sh, double* part, int nb) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kWarps; k++) s += sh[k];
    part[(size_t)kSlotInit * nb + blockIdx.x] = s;
  }
}

__device__ __forceinline__ double grid_sum_f64(const double* part, int nb) {
  double a = 0.0;
  if (threadIdx.x < 32) {
    for (int k = threadIdx.x; k < nb; k += 32) a += __ldcg(&part[(size_t)kSlotInit * nb + k]);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  }
  return a;
}

// ---- product of one row ------------------------------------------------------------------
// own + sum over the row's active columns j of B_kj nbv(j); `nbv` forms the neighbour's value
// from vectors written before the last barrier.  Two entries are gathered at a time and summed in
// separate accumulators (a shorter dependent FP64 chain).
template <typename T, typename NbF>
__device__ __forceinline__ typename V2<T>::t row_product(const int* col, const B4<T>* blk, int deg,
                                                         typename V2<T>::t own, NbF nbv) {
  using V = typename V2<T>::t;
  V acc0 = own, acc1 = mk<T>(0, 0);
  for (int j = 0; j < deg; j += 2) {
    const int c0 = col[j];
    const int c1 = j + 1 < deg ? col[j + 1] : -1;
    V x0 = mk<T>(0, 0), x1 = mk<T>(0, 0);
    B4<T> b0 = {0, 0, 0, 0}, b1 = {0, 0, 0, 0};
    if (c0 >= 0) {
      x0 = nbv(c0);
      b0 = blk[j];
    }
    if (c1 >= 0) {
      x1 = nbv(c1);
      b1 = blk[j + 1];
    }
    acc0.x += b0.a * x0.x + b0.b * x0.y;
    acc0.y += b0.c * x0.x + b0.d * x0.y;
    acc1.x += b1.a * x1.x + b1.b * x1.y;
    acc1.y += b1.c * x1.x + b1.d * x1.y;
  }
  return mk<T>(acc0.x + acc1.x, acc0.y + acc1.y);
}

// ---- fracture-line solve -----------------------------------------------------------------
// FP32 block-Thomas recurrences of one 32-row chunk for NR right-hand sides, as inclusive warp
// scans of 2x2 affine maps.  fwd: w_t = Dinv_t src_t + A_t w_{t-1};  bwd: z_t = w_t - G_t z_{t+1}.
template <int NR>
__device__ __forceinline__ void scan_fwd(float2 (&c)[NR], M2<float> A, const float2 (&carry)[NR], int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    M2<float> Ap;
    Ap.a = __shfl_up_sync(0xffffffffu, A.a, o);
    Ap.b = __shfl_up_sync(0xffffffffu, A.b, o);
    Ap.c = __shfl_up_sync(0xffffffffu, A.c, o);
    Ap.d = __shfl_up_sync(0xffffffffu, A.d, o);
    float2 cp[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) {
      cp[q].x = __shfl_up_sync(0xffffffffu, c[q].x, o);
      cp[q].y = __shfl_up_sync(0xffffffffu, c[q].y, o);
    }
    if (lane >= o) {
#pragma unroll
      for (int q = 0; q < NR; q++) {
        c[q].x += A.a * cp[q].x + A.b * cp[q].y;
        c[q].y += A.c * cp[q].x + A.d * cp[q].y;
      }
      A = mm(A, Ap);
    }
  }
#pragma unroll
  for (int q = 0; q < NR; q++)
    c[q] = make_float2(c[q].x + A.a * carry[q].x + A.b * carry[q].y, c[q].y + A.c * carry[q].x + A.d * carry[q].y);
}

template <int NR>
__device__ __forceinline__ void scan_bwd(float2 (&c)[NR], M2<float> B, const float2 (&carry)[NR], int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    M2<float> Bp;
    Bp.a = __shfl_down_sync(0xffffffffu, B.a, o);
    Bp.b = __shfl_down_sync(0xffffffffu, B.b, o);
    Bp.c = __shfl_down_sync(0xffffffffu, B.c, o);
    Bp.d = __shfl_down_sync(0xffffffffu, B.d, o);
    float2 cp[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) {
      cp[q].x = __shfl_down_sync(0xffffffffu, c[q].x, o);
      cp[q].y = __shfl_down_sync(0xffffffffu, c[q].y, o);
    }
    if (lane + o < 32) {
#pragma unroll
      for (int q = 0; q < NR; q++) {
        c[q].x += B.a * cp[q].x + B.b * cp[q].y;
        c[q].y += B.c * cp[q].x + B.d * cp[q].y;
      }
      B = mm(B, Bp);
    }
  }
#pragma unroll
  for (int q = 0; q < NR; q++)
    c[q] = make_float2(c[q].x + B.a * carry[q].x + B.b * carry[q].y, c[q].y + B.c * carry[q].x + B.d * carry[q].y);
}

// Factors of one line block: row t's D'^{-1}, A and G at fd[t*fs], fa[t*fs], fg[t*fs].
struct LineFac {
  const float4 *fd, *fa, *fg;
  int fs;
};

// M^{-1} on one line block (len <= 128 rows) for NR right-hand sides held in registers
// (src[c][q] = input q of row k0 + 32c + lane); results stored to dst[q][k0 + t].
template <typename T, int NR>
__device__ __forceinline__ void line_solve(int k0, int len, const LineFac& f, const float2 (&src)[kLineChunks][NR],
                                           typename V2<T>::t* const (&dst)[NR]) {
  const int lane = threadIdx.x & 31;
  float2 w[kLineChunks][NR];
  float2 carry[NR];
#pragma unroll
  for (int q = 0; q < NR; q++) carry[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < kLineChunks; c++) {
#pragma unroll
    for (int q = 0; q < NR; q++) w[c][q] = make_float2(0.f, 0.f);
    if (c * 32 < len) {
      const int t = c * 32 + lane;
      M2<float> A = {0.f, 0.f, 0.f, 0.f};
      if (t < len) {
        const float4 Di = f.fd[(size_t)t * f.fs];
#pragma unroll
        for (int q = 0; q < NR; q++)
          w[c][q] = make_float2(Di.x * src[c][q].x + Di.y * src[c][q].y, Di.z * src[c][q].x + Di.w * src[c][q].y);
        const float4 a4 = f.fa[(size_t)t * f.fs];
        A = {a4.x, a4.y, a4.z, a4.w};
      }
      scan_fwd<NR>(w[c], A, carry, lane);
      const int last = min(31, len - 1 - c * 32);
#pragma unroll
      for (int q = 0; q < NR; q++) {
        carry[q].x = __shfl_sync(0xffffffffu, w[c][q].x, last);
        carry[q].y = __shfl_sync(0xffffffffu, w[c][q].y, last);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; q++) carry[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = kLineChunks - 1; c >= 0; c--) {
    if (c * 32 < len) {
      const int t = c * 32 + lane;
      M2<float> B = {0.f, 0.f, 0.f, 0.f};
      float2 z[NR];
#pragma unroll
      for (int q = 0; q < NR; q++) z[q] = make_float2(0.f, 0.f);
      if (t < len) {
        const float4 g4 = f.fg[(size_t)t * f.fs];
        B = {-g4.x, -g4.y, -g4.z, -g4.w};
#pragma unroll
        for (int q = 0; q < NR; q++) z[q] = w[c][q];
      }
      scan_bwd<NR>(z, B, carry, lane);
#pragma unroll
      for (int q = 0; q < NR; q++) {
        if (t < len) dst[q][k0 + t] = mk<T>((T)z[q].x, (T)z[q].y);
        carry[q].x = __shfl_sync(0xffffffffu, z[q].x, 0);
        carry[q].y = __shfl_sync(0xffffffffu, z[q].y, 0);
      }
    }
  }
}

// ---- the solver --------------------------------------------------------------------------
// A matrix row: off >= 0 is its first entry in the shared-memory pool, off < 0 encodes its first
// CSR entry e0 as -(e0 + 1) (global memory); deg entries.
struct RowRef {
  int off, deg;
};

template <typename T, bool LINES>
__global__ void __launch_bounds__(kKryBlk, 1) k_bicgstab(Dev d, double rtol, int maxit) {
  using V = typename V2<T>::t;
  using B = B4<T>;
  using Ref = RowRef;
  using Acc = typename DotAcc<T>::t;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double sh[kWarps];
  __shared__ DF s_df[4 * kWarps];
  __shared__ double s_bc[8];  // beta, alpha_prev, omega_prev, alpha, scale, 1/scale, rho
  __shared__ int s_ctl;       // 0 continue, 1 stop
  __shared__ int s_epool;     // next free entry of the shared-memory pool
  const int nA = d.ctr->n_active;
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int rpb = (nA + nb - 1) / nb;
  const int r0 = min(nA, (int)blockIdx.x * rpb), r1 = min(nA, r0 + rpb);
  const int kbeg = r0 + (int)threadIdx.x, kstep = blockDim.x;
  const int nlines = LINES ? d.ctr->n_lines : 0;
  const bool has_line = LINES && (int)blockIdx.x + nb * wib < nlines;
  const bool busy = __any_sync(0xffffffffu, kbeg < r1) || has_line;  // this warp adds to the dots
  V* const x = (V*)d.kx;
  V* const r = (V*)d.kr;
  V* const rh = (V*)d.krh;
  V* const v = (V*)d.kv;
  V* const s = (V*)d.ks;
  V* const t = (V*)d.kt;
  V* const z = (V*)d.kz;
  V* const rt = LINES ? (V*)d.krt : r;  // M = I without lines: r~ = r, z^ = s, t~ = t
  V* const zf = LINES ? (V*)d.kzf : s;
  V* const tt = LINES ? (V*)d.ktt : t;
  V* const y0 = (V*)d.ky0;
  V* const y1 = (V*)d.ky1;
  V* const vt0 = (V*)d.kvt0;
  V* const vt1 = (V*)d.kvt1;
  const V* b = (const V*)d.rhs;
  const T* blocks = (const T*)d.blocks;
  const int* lflag = d.line_row_flag;
  double* part = d.partials;
  float4* s_fac = (float4*)dsm;
  const int ecap = (int)((kKrySmem - kLineSmem) / (sizeof(int) + sizeof(B)));
  B* s_blk = (B*)(dsm + kLineSmem);
  int* s_col = (int*)(dsm + kLineSmem + (size_t)ecap * sizeof(B));
  if (threadIdx.x == 0) s_epool = 0;
  __syncthreads();

  auto global_ref = [&](int k) -> Ref {
    const int i = __ldg(&d.act[k]);
    const int e0 = __ldg(&d.row_ptr[i]);
    return {-(e0 + 1), __ldg(&d.row_ptr[i + 1]) - e0};
  };
  // stage a row's columns and blocks in the shared pool (placement does not affect the result)
  auto stage = [&](int k) -> Ref {
    const Ref g = global_ref(k);
    const int off = atomicAdd(&s_epool, g.deg);
    if (off + g.deg > ecap) return g;
    const int e0 = -(g.off + 1);
    for (int j = 0; j < g.deg; j++) {
      s_col[off + j] = __ldg(&d.colA[e0 + j]);
      s_blk[off + j] = *(const B*)&blocks[4 * (size_t)(e0 + j)];
    }
    return {off, g.deg};
  };
  // product of a row with a vector whose own value is `own` and whose neighbour values come from nbv
  auto product = [&](const Ref& ref, const V& own, auto nbv) -> V {
    if (ref.off >= 0) return row_product<T>(s_col + ref.off, s_blk + ref.off, ref.deg, own, nbv);
    const size_t e0 = (size_t)(-(ref.off + 1));
    return row_product<T>(d.colA + e0, (const B*)&blocks[4 * e0], ref.deg, own, nbv);
  };
  // this thread's first non-line rows
  Ref rr_[kRowsCached];
  int rk_[kRowsCached];
#pragma unroll
  for (int q = 0; q < kRowsCached; q++) {
    const int k = kbeg + q * kstep;
    rk_[q] = -1;
    rr_[q] = {0, 0};
    if (k < r1 && !(LINES && __ldg(&lflag[k]))) {
      rk_[q] = k;
      rr_[q] = stage(k);
    }
  }
  // this warp's first line block (l = blockIdx + nb * wib): rows staged, factors staged if a slot is free
  Ref lr_[kLineChunks];
  int lk0 = 0, llen = 0;
  auto gfac = [&](int k0) -> LineFac {
    return {(const float4*)d.line_dinv + k0, (const float4*)d.line_a + k0, (const float4*)d.line_g + k0, 1};
  };
  auto sfac = [&]() -> LineFac {
    const float4* base = &s_fac[(size_t)wib * kLineChunks * 32 * 3];
    return {base, base + 1, base + 2, 3};
  };
  if (LINES) {
    if (has_line) {
      const int l = (int)blockIdx.x + nb * wib;
      lk0 = __ldg(&d.line_start[l]);
      llen = __ldg(&d.line_len[l]);
      if (wib < kLineSlots) {
        const LineFac g = gfac(lk0);
        float4* base = &s_fac[(size_t)wib * kLineChunks * 32 * 3];
        for (int q = lane; q < llen; q += 32) {
          base[3 * q] = g.fd[q];
          base[3 * q + 1] = g.fa[q];
          base[3 * q + 2] = g.fg[q];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kLineChunks; c++) {
      lr_[c] = {0, 0};
      if (c * 32 + lane < llen) lr_[c] = stage(lk0 + c * 32 + lane);
    }
  }
  __syncthreads();

  // fn(k, ref) over this thread's non-line rows
  auto rows = [&](auto fn) {
#pragma unroll
    for (int q = 0; q < kRowsCached; q++)
      if (rk_[q] >= 0) fn(rk_[q], rr_[q]);
    for (int k = kbeg + kRowsCached * kstep; k < r1; k += kstep) {
      if (LINES && __ldg(&lflag[k])) continue;
      fn(k, global_ref(k));
    }
  };
  // fn(k0, len, factors, refs) over this warp's line blocks (warp-uniform)
  auto lines = [&](auto fn) {
    if constexpr (LINES) {
      if (!has_line) return;
      fn(lk0, llen, wib < kLineSlots ? sfac() : gfac(lk0), lr_);
      for (int j = wib + kWarps;; j += kWarps) {
        const int l = (int)blockIdx.x + nb * j;
        if (l >= nlines) break;
        const int k0 = __ldg(&d.line_start[l]), len = __ldg(&d.line_len[l]);
        Ref refs[kLineChunks];
#pragma unroll
        for (int c = 0; c < kLineChunks; c++) {
          refs[c] = {0, 0};
          if (c * 32 + lane < len) refs[c] = global_ref(k0 + c * 32 + lane);
        }
        fn(k0, len, gfac(k0), refs);
      }
    }
  };

  // ---- initialisation: x = z = t = t~ = y_0 = v~_0 = 0, s = r^ = b, z^ = M^{-1} b -------------
  double l_bb = 0.0;
  auto init_row = [&](int k) -> V {
    const V bk = b[k];
    const V o = mk<T>(0, 0);
    x[k] = o;
    z[k] = o;
    t[k] = o;
    tt[k] = o;
    y0[k] = o;
    vt0[k] = o;
    s[k] = bk;
    rh[k] = bk;
    l_bb += (double)bk.x * bk.x + (double)bk.y * bk.y;
    return bk;
  };
  rows([&](int k, const Ref&) { zf[k] = init_row(k); });
  lines([&](int k0, int len, const LineFac& f, const Ref(&)[kLineChunks]) {
    float2 src[kLineChunks][1];
#pragma unroll
    for (int c = 0; c < kLineChunks; c++) {
      src[c][0] = make_float2(0.f, 0.f);
      if (c * 32 + lane < len) {
        const V bk = init_row(k0 + c * 32 + lane);
        src[c][0] = make_float2((float)bk.x, (float)bk.y);
      }
    }
    V* const dst[1] = {zf};
    line_solve<T, 1>(k0, len, f, src, dst);
  });
  block_store_f64(l_bb, sh, part, nb);
  grid.sync();
  const double bb = grid_sum_f64(part, nb);
  double rho = 0.0, alpha = 0.0, stop2 = 0.0, rr_last = 0.0;
  if (threadIdx.x == 0) {
    rho = bb;
    stop2 = rtol * rtol * bb;
    // FP64 dots are scaled by an exact power of two near 1/bb (biased exponent 2046 - E of bb,
    // clamped to the normal range) before they are carried in double-float; FP32 dots need none
    long long e = bb > 0.0 ? ((__double_as_longlong(bb) >> 52) & 0x7ff) : 1023;
    e = e < 1 ? 1 : (e > 2045 ? 2045 : e);
    const bool f64 = sizeof(T) == 8;
    s_bc[4] = f64 ? __longlong_as_double((2046 - e) << 52) : 1.0;
    s_bc[5] = f64 ? __longlong_as_double(e << 52) : 1.0;
    s_bc[0] = 0.0;  // beta_1
    s_bc[1] = 0.0;  // alpha_0
    s_bc[2] = 0.0;  // omega_0
    s_bc[6] = bb;   // rho_1
    s_ctl = 0;
  }
  __syncthreads();
  const double dscale = s_bc[4], dinv = s_bc[5];
  int status = 1, it;
  for (it = 1;; it++) {
    // ---- phase 1 -------------------------------------------------------------------------
    const T beta = (T)s_bc[0], alp = (T)s_bc[1], omp = (T)s_bc[2], nom = -omp;
    const bool odd = it & 1;
    const V* yo = odd ? y0 : y1;
    V* yn = odd ? y1 : y0;
    const V* vto = odd ? vt0 : vt1;
    V* vtn = odd ? vt1 : vt0;
    // r~_{i-1} and y_i of a row from stored vectors (the owner evaluates the same expressions)
    auto rt_of = [&](int c) { return axpy(nom, ldv(&tt[c]), ldv(&zf[c])); };
    auto y_of = [&](const V& rtc, int c) { return axpy(beta, axpy(nom, ldv(&vto[c]), ldv(&yo[c])), rtc); };
    auto ynb = [&](int c) { return y_of(rt_of(c), c); };
    Acc l_rv, l_rr;
    dot_zero(l_rv);
    dot_zero(l_rr);
    auto p1_row = [&](int k, const Ref& ref) -> V {
      const V xk = ldv(&x[k]), yk = ldv(&yo[k]), zk = ldv(&z[k]), sk = ldv(&s[k]), tk = ldv(&t[k]),
              rhk = ldv(&rh[k]);
      x[k] = mk<T>(xk.x + alp * yk.x + omp * zk.x, xk.y + alp * yk.y + omp * zk.y);
      const V rk = axpy(nom, tk, sk);
      r[k] = rk;
      dot_acc(l_rr, rk.x, rk.x);
      dot_acc(l_rr, rk.y, rk.y);
      const V rtk = rt_of(k);
      if (LINES) rt[k] = rtk;
      const V ynk = y_of(rtk, k);
      yn[k] = ynk;
      const V vv = product(ref, ynk, ynb);
      v[k] = vv;
      dot_acc(l_rv, rhk.x, vv.x);
      dot_acc(l_rv, rhk.y, vv.y);
      return vv;
    };
    rows([&](int k, const Ref& ref) { vtn[k] = p1_row(k, ref); });
    lines([&](int k0, int len, const LineFac& f, const Ref(&refs)[kLineChunks]) {
      float2 src[kLineChunks][1];
#pragma unroll
      for (int c = 0; c < kLineChunks; c++) {
        src[c][0] = make_float2(0.f, 0.f);
        if (c * 32 + lane < len) {
          const V vv = p1_row(k0 + c * 32 + lane, refs[c]);
          src[c][0] = make_float2((float)vv.x, (float)vv.y);
        }
      }
      V* const dst[1] = {vtn};
      line_solve<T, 1>(k0, len, f, src, dst);
    });
    {
      const DF vals[2] = {dot_df(l_rv, dscale), dot_df(l_rr, dscale)};
      block_store<2>(vals, busy, s_df, part, kSlotS1, nb);
    }
    grid.sync();
    {
      double o[2];
      grid_sum<2>(part, kSlotS1, nb, dinv, o);
      if (threadIdx.x == 0) {
        rr_last = o[1];
        if (o[1] <= stop2) {
          s_ctl = 1;
          status = 0;
        } else if (it > maxit) {
          s_ctl = 1;
          status = 1;
        } else if (o[0] == 0.0 || !isfinite(o[0]) || rho == 0.0 || !isfinite(rho)) {
          s_ctl = 1;
          status = 2;
        } else {
          alpha = rho / o[0];
          s_bc[3] = alpha;
        }
      }
    }
    __syncthreads();
    if (s_ctl) break;
    // ---- phase 2 -------------------------------------------------------------------------
    const T nal = -(T)s_bc[3];
    const double rho_i = s_bc[6], alpha_i = s_bc[3];  // read before thread 0 overwrites rho below
    auto znb = [&](int c) { return axpy(nal, ldv(&vtn[c]), ldv(&rt[c])); };
    Acc l_ts, l_tt, l_rs, l_rt;
    dot_zero(l_ts);
    dot_zero(l_tt);
    dot_zero(l_rs);
    dot_zero(l_rt);
    V sk_, tk_;
    auto p2_row = [&](int k, const Ref& ref) {
      const V rk = ldv(&r[k]), vk = ldv(&v[k]), rhk = ldv(&rh[k]);
      const V sk = axpy(nal, vk, rk);
      s[k] = sk;
      const V zk = znb(k);
      z[k] = zk;
      const V tk = product(ref, zk, znb);
      t[k] = tk;
      dot_acc(l_ts, tk.x, sk.x);
      dot_acc(l_ts, tk.y, sk.y);
      dot_acc(l_tt, tk.x, tk.x);
      dot_acc(l_tt, tk.y, tk.y);
      dot_acc(l_rs, rhk.x, sk.x);
      dot_acc(l_rs, rhk.y, sk.y);
      dot_acc(l_rt, rhk.x, tk.x);
      dot_acc(l_rt, rhk.y, tk.y);
      sk_ = sk;
      tk_ = tk;
    };
    rows([&](int k, const Ref& ref) {
      p2_row(k, ref);
      if (LINES) {
        zf[k] = sk_;
        tt[k] = tk_;
      }
    });
    lines([&](int k0, int len, const LineFac& f, const Ref(&refs)[kLineChunks]) {
      float2 src[kLineChunks][2];
#pragma unroll
      for (int c = 0; c < kLineChunks; c++) {
        src[c][0] = src[c][1] = make_float2(0.f, 0.f);
        if (c * 32 + lane < len) {
          p2_row(k0 + c * 32 + lane, refs[c]);
          src[c][0] = make_float2((float)sk_.x, (float)sk_.y);
          src[c][1] = make_float2((float)tk_.x, (float)tk_.y);
        }
      }
      V* const dst[2] = {zf, tt};
      line_solve<T, 2>(k0, len, f, src, dst);
    });
    {
      const DF vals[4] = {dot_df(l_ts, dscale), dot_df(l_tt, dscale), dot_df(l_rs, dscale), dot_df(l_rt, dscale)};
      block_store<4>(vals, busy, s_df, part, kSlotS2, nb);
    }
    grid.sync();
    {
      double o[4];
      grid_sum<4>(part, kSlotS2, nb, dinv, o);
      const double ts = o[0], t2 = o[1], rs = o[2], rtv = o[3];
      // the two divisions run in two warps: thread 0 omega and rho_{i+1}, thread 32 beta_{i+1}
      //   beta = (rho_{i+1} / rho_i) (alpha / omega) = alpha (rs t2 - ts rt) / (rho_i ts)
      if (threadIdx.x == 0) {
        if (!isfinite(ts) || !isfinite(t2) || !isfinite(rs) || !isfinite(rtv)) {
          s_ctl = 1;
          status = 2;
        } else {
          // t = 0 means A z = 0: omega = 0 leaves r = s and restarts the direction (beta = 0)
          const double omega = t2 > 0.0 ? ts / t2 : 0.0;
          rho = fma(-omega, rtv, rs);
          s_bc[1] = alpha;
          s_bc[2] = omega;
          s_bc[6] = rho;
        }
      } else if (threadIdx.x == 32) {
        s_bc[0] = (t2 > 0.0 && ts != 0.0) ? alpha_i * fma(rs, t2, -ts * rtv) / (rho_i * ts) : 0.0;
      }
    }
    __syncthreads();
    if (s_ctl) break;
  }
  // x holds x_{it-1} at every exit; thread 0 of block 0 reports
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr->krylov_iters = it - 1;
    d.ctr->krylov_status = status;
    d.ctr->krylov_relres = bb > 0.0 ? sqrt(rr_last / bb) : 0.0;
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
