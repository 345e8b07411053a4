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
// Ownership: each block owns a contiguous chunk of rows whose ends never split a fracture-line
// block; its threads take the chunk's rows, leave the line-solve inputs in a block buffer, and
// after a block barrier its warps apply M^{-1} to the chunk's line blocks (short blocks packed into
// warp segments, long ones a warp each).  Matrix rows (columns and blocks), row references and line
// factors are staged in shared memory once per solve.  Reductions: per-row products in FP64 (FP32
// path: exact FP32 products in double-float); across lanes, warps and blocks in
// double-float (two FP32 words, Knuth's TwoSum), after scaling by an exact power of two near
// 1/||b||^2.  Every block sums the block partials in the same order, so all blocks hold identical
// scalars (computed once per block by thread 0: FP64 division is a long sequence here).
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "lns_internal.cuh"

namespace lns {

namespace {

constexpr int kKryBlk = 256;
constexpr int kWarps = kKryBlk / 32;
constexpr int kRowsCached = 4;   // non-line rows per thread whose matrix row is staged
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

template <typename V>
struct V2pair {
  V a, b;
};

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

// Scalar arithmetic of the recurrence in double-float (FP32 instructions only; about 44
// significant bits, ample for the BiCGStab coefficients).
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return df_fast(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r = df_add(a, df_neg(df_mul(DF{q1, 0.f}, b)));
  return df_fast(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool df_finite(DF a) { return isfinite(a.hi) && isfinite(a.lo); }
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Recurrence scalars: FP64 for FP64 vectors, double-float for FP32 vectors.
__device__ __forceinline__ double sc_from(DF a, double) { return df_to_double(a); }
__device__ __forceinline__ DF sc_from(DF a, DF) { return a; }
__device__ __forceinline__ double sc_div(double a, double b) { return a / b; }
__device__ __forceinline__ DF sc_div(DF a, DF b) { return df_div(a, b); }
__device__ __forceinline__ double sc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ DF sc_mul(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ double sc_fnma(double a, double b, double c) { return fma(-a, b, c); }  // c - a b
__device__ __forceinline__ DF sc_fnma(DF a, DF b, DF c) { return df_add(c, df_neg(df_mul(a, b))); }
__device__ __forceinline__ bool sc_le(double a, double b) { return a <= b; }
__device__ __forceinline__ bool sc_le(DF a, DF b) { return df_le(a, b); }
__device__ __forceinline__ bool sc_ok(double a) { return a != 0.0 && isfinite(a); }  // usable divisor
__device__ __forceinline__ bool sc_ok(DF a) { return a.hi != 0.f && df_finite(a); }
__device__ __forceinline__ bool sc_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool sc_finite(DF a) { return df_finite(a); }
__device__ __forceinline__ bool sc_pos(double a) { return a > 0.0; }
__device__ __forceinline__ bool sc_pos(DF a) { return a.hi > 0.f; }
__device__ __forceinline__ bool sc_nonzero(double a) { return a != 0.0; }
__device__ __forceinline__ bool sc_nonzero(DF a) { return a.hi != 0.f; }
__device__ __forceinline__ void sc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void sc_zero(DF& a) { a = DF{0.f, 0.f}; }
__device__ __forceinline__ double sc_double(double a) { return a; }
__device__ __forceinline__ double sc_double(DF a) { return df_to_double(a); }
template <typename T>
__device__ __forceinline__ T sc_t(double a) { return (T)a; }
template <typename T>
__device__ __forceinline__ T sc_t(DF a) { return (T)a.hi; }

// Dot products of one thread's rows.  FP64 vectors: fused FP64 products, converted to double-float
// (after scaling) once per phase.  FP32 vectors: exact FP32 products (p + e, e = fma(a, b, -p))
// summed in double-float, so the FP32 path issues no FP64 instruction per row: the high part
// takes each p with an exact two-sum, whose rounding error and e go to the low part (left
// unnormalised until the block reduction: a thread sums a handful of rows).
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
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(acc.hi, p);
  const float bv = __fsub_rn(s, acc.hi);
  const float av = __fsub_rn(s, bv);
  const float err = __fadd_rn(__fsub_rn(acc.hi, av), __fsub_rn(p, bv));
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
  acc.hi = s;
}
__device__ __forceinline__ DF dot_df(double acc, double scale) { return df_from(acc * scale); }
__device__ __forceinline__ DF dot_df(DF acc, float scale) { return {acc.hi * scale, acc.lo * scale}; }

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

// Sum over all blocks of slots [slot, slot+NV) in a fixed order, in double-float; valid in warps 0
// and 1 (both compute it, so that two threads can share the scalar work).  All of a lane's partial
// loads of one pass are issued before any is used.
template <int NV>
__device__ __forceinline__ void grid_sum(const double* part, int slot, int nb, DF (&out)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; q++) out[q] = {0.f, 0.f};
  if (threadIdx.x >= 64) return;
  const int ln = threadIdx.x & 31;
  constexpr int kU = 5;
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
    for (int q = 0; q < NV; q++) out[q] = df_add(out[q], v[q][0]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NV; q++) out[q] = df_add(out[q], df_shfl_xor(out[q], o));
}

// ||b||^2 and ||r_0||^2 (once per solve, before the scale is known): FP64 block partial in a slot
// and its grid sum.
__device__ __forceinline__ void block_store_f64(double a, double* sh, double* part, int nb, int slot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kWarps; k++) s += sh[k];
    part[(size_t)slot * nb + blockIdx.x] = s;
  }
}

__device__ __forceinline__ double grid_sum_f64(const double* part, int nb, int slot) {
  double a = 0.0;
  if (threadIdx.x < 32) {
    for (int k = threadIdx.x; k < nb; k += 32) a += __ldcg(&part[(size_t)slot * nb + k]);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  }
  return a;
}

// ---- product of one row ------------------------------------------------------------------
// own + sum over the row's active columns j of B_kj x_j, where x_j = comb(load(j)) is formed from
// vectors written before the last barrier.  The loads of up to kBatch neighbours are issued before
// any is used, so a row of degree <= kBatch costs one L2 round trip: BATCH neighbours at a time in
// FP32 (4, or 6 in the grid solver on models of more than 5 neighbours a cell, which fits its 255
// registers), 2 in FP64, whose gathered values take twice the registers.
template <typename T, int BATCH = 4, typename LoadF, typename CombF>
__device__ __forceinline__ typename V2<T>::t row_product(const int* col, const B4<T>* blk, int deg,
                                                         typename V2<T>::t own, LoadF load, CombF comb) {
  using V = typename V2<T>::t;
  using Raw = decltype(load(0));
  constexpr int kBatch = sizeof(T) == 8 ? 2 : BATCH;
  V acc0 = own, acc1 = mk<T>(0, 0);
  for (int j = 0; j < deg; j += kBatch) {
    int c[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; q++) c[q] = j + q < deg ? col[j + q] : -1;
    Raw raw[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; q++)
      if (c[q] >= 0) raw[q] = load(c[q]);
#pragma unroll
    for (int q = 0; q < kBatch; q++)
      if (c[q] >= 0) {
        const V xv = comb(raw[q]);
        const B4<T> bq = blk[j + q];
        V& acc = (q & 1) ? acc1 : acc0;
        acc.x += bq.a * xv.x + bq.b * xv.y;
        acc.y += bq.c * xv.x + bq.d * xv.y;
      }
  }
  return mk<T>(acc0.x + acc1.x, acc0.y + acc1.y);
}

// ---- fracture-line solve -----------------------------------------------------------------
// FP32 block-Thomas recurrences of a fracture-line block for NR right-hand sides,
//   fwd: w_t = Dinv_t src_t + A_t w_{t-1};   bwd: z_t = w_t - G_t z_{t+1},
// as inclusive warp scans of 2x2 affine maps (one map per lane: a row, or the composite of the
// lane's rows), local to a segment of seg lanes (zero carry-in).  On return lane t holds c_t and
// the composite map P_t such that the value at lane t is c_t + P_t * (the value entering the
// segment).
// A lane with no partner at a level takes the identity map and a zero value from it, so every
// lane runs the same instructions (no divergent branch per level).
template <int NR>
__device__ __forceinline__ void scan_fwd(float2 (&c)[NR], M2<float>& A, int lane, int seg = 32) {
  const int t = lane & (seg - 1);  // position in the segment of seg lanes (a power of two)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= seg) break;  // uniform
    const bool in = t >= o;
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
      cp[q] = in ? cp[q] : make_float2(0.f, 0.f);
    }
    Ap = in ? Ap : M2<float>{1.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int q = 0; q < NR; q++) {
      c[q].x += A.a * cp[q].x + A.b * cp[q].y;
      c[q].y += A.c * cp[q].x + A.d * cp[q].y;
    }
    A = mm(A, Ap);
  }
}

template <int NR>
__device__ __forceinline__ void scan_bwd(float2 (&c)[NR], M2<float>& B, int lane, int seg = 32) {
  const int t = lane & (seg - 1);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= seg) break;  // uniform
    const bool in = t + o < seg;
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
      cp[q] = in ? cp[q] : make_float2(0.f, 0.f);
    }
    Bp = in ? Bp : M2<float>{1.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int q = 0; q < NR; q++) {
      c[q].x += B.a * cp[q].x + B.b * cp[q].y;
      c[q].y += B.c * cp[q].x + B.d * cp[q].y;
    }
    B = mm(B, Bp);
  }
}

// Factors of one line block: row t's D'^{-1}, A and G at fd[at(t)], fa[at(t)], fg[at(t)], with
// at(t) = (o + t) fs + ((o + t) / 4) pad: the global arrays (fs 1, pad 0), or the rows staged in
// shared memory at fac_slot (fs 3, pad 1).
struct LineFac {
  const float4 *fd, *fa, *fg;
  int o, fs, pad;
  __device__ __forceinline__ int at(int t) const {
    const int i = o + t;
    return i * fs + (i >> 2) * pad;
  }
};
// Staged line factors: row i of a chunk at float4 slots fac_slot(i) + 0, 1, 2.  A pad slot after
// every four rows puts the four consecutive rows each lane of a whole-warp line solve reads at a
// stride of 13 slots, so the lanes of a quarter warp hit distinct banks.
__device__ __forceinline__ int fac_slot(int i) { return 3 * i + (i >> 2); }
constexpr size_t fac_slots(size_t rows) { return 3 * rows + rows / 4 + 1; }

constexpr int kLineRpl = kLineBlockRows / 32;  // rows per lane of a whole-warp line solve

// affine maps on a row value v -> M v + c: the map of row t after the map of the rows before it
__device__ __forceinline__ float2 mv2(const M2<float>& M, float2 v) {
  return make_float2(M.a * v.x + M.b * v.y, M.c * v.x + M.d * v.y);
}

// M^{-1} on line blocks for NR right-hand sides, in segments of seg lanes (4, 8, 16 or 32; one
// block of len <= seg * RPL rows per segment, 32 / seg blocks per warp; a lane whose segment holds
// no block has len = 0 and carries zeros).  Input q of row k0 + t is buf[q * bstride + t]; results
// are stored to dst[q][k0 + t].  Lane t of a segment holds the RPL consecutive rows starting at
// RPL * t.  Each sweep composes its rows' affine maps inside the lane, scans the lane maps across
// the segment (log2(seg) shuffle levels for the whole block), and recomputes its rows from the
// value entering the lane.  Rows at or beyond len are zero maps and zero values, so they pass
// nothing to the rows of the block.
template <typename T, int NR, int RPL>
__device__ __forceinline__ void line_solve_rpl(int seg, int k0, int len, const LineFac& f, const float2* buf,
                                               int bstride, typename V2<T>::t* const (&dst)[NR]) {
  const int lane = threadIdx.x & 31, t = lane & (seg - 1);
  float2 c[RPL][NR];
  M2<float> A[RPL], B[RPL];
  // every load of the lane's rows (both sweeps) is issued first
#pragma unroll
  for (int j = 0; j < RPL; j++) {
    const int r = RPL * t + j;
    A[j] = {0.f, 0.f, 0.f, 0.f};
    B[j] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NR; q++) c[j][q] = make_float2(0.f, 0.f);
    if (r < len) {
      const int fr = f.at(r);
      const float4 Di = f.fd[fr];
      const float4 a4 = f.fa[fr];
      const float4 g4 = f.fg[fr];
#pragma unroll
      for (int q = 0; q < NR; q++) c[j][q] = mv2({Di.x, Di.y, Di.z, Di.w}, buf[q * bstride + r]);
      A[j] = {a4.x, a4.y, a4.z, a4.w};
      B[j] = {-g4.x, -g4.y, -g4.z, -g4.w};
    }
  }
  // forward sweep w_t = Dinv_t src_t + A_t w_{t-1}: the lane's composite map, the segment scan,
  // then the rows from the last row of the lane before
  {
    M2<float> M = A[0];
    float2 cl[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) cl[q] = c[0][q];
#pragma unroll
    for (int j = 1; j < RPL; j++) {
#pragma unroll
      for (int q = 0; q < NR; q++) {
        const float2 u = mv2(A[j], cl[q]);
        cl[q] = make_float2(u.x + c[j][q].x, u.y + c[j][q].y);
      }
      M = mm(A[j], M);
    }
    scan_fwd<NR>(cl, M, lane, seg);
#pragma unroll
    for (int q = 0; q < NR; q++) {
      float2 w;
      w.x = __shfl_up_sync(0xffffffffu, cl[q].x, 1);
      w.y = __shfl_up_sync(0xffffffffu, cl[q].y, 1);
      if (t == 0) w = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < RPL; j++) {
        const float2 u = mv2(A[j], w);
        w = make_float2(u.x + c[j][q].x, u.y + c[j][q].y);
        c[j][q] = w;
      }
    }
  }
  // backward sweep z_t = w_t - G_t z_{t+1}, mirrored
  {
    M2<float> M = B[RPL - 1];
    float2 cl[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) cl[q] = c[RPL - 1][q];
#pragma unroll
    for (int j = RPL - 2; j >= 0; j--) {
#pragma unroll
      for (int q = 0; q < NR; q++) {
        const float2 u = mv2(B[j], cl[q]);
        cl[q] = make_float2(u.x + c[j][q].x, u.y + c[j][q].y);
      }
      M = mm(B[j], M);
    }
    scan_bwd<NR>(cl, M, lane, seg);
#pragma unroll
    for (int q = 0; q < NR; q++) {
      float2 z;
      z.x = __shfl_down_sync(0xffffffffu, cl[q].x, 1);
      z.y = __shfl_down_sync(0xffffffffu, cl[q].y, 1);
      if (t == seg - 1) z = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = RPL - 1; j >= 0; j--) {
        const float2 u = mv2(B[j], z);
        z = make_float2(u.x + c[j][q].x, u.y + c[j][q].y);
        const int r = RPL * t + j;
        if (r < len) dst[q][k0 + r] = mk<T>((T)z.x, (T)z.y);
      }
    }
  }
}

// a whole warp on one block of up to kLineBlockRows rows (kLineRpl rows per lane)
template <typename T, int NR>
__device__ __forceinline__ void line_solve(int k0, int len, const LineFac& f, const float2* buf, int bstride,
                                           typename V2<T>::t* const (&dst)[NR]) {
  line_solve_rpl<T, NR, kLineRpl>(32, k0, len, f, buf, bstride, dst);
}

// short blocks, two rows per lane, 32 / seg of them per warp
template <typename T, int NR>
__device__ __forceinline__ void line_solve_seg(int seg, int k0, int len, const LineFac& f, const float2* buf,
                                               int bstride, typename V2<T>::t* const (&dst)[NR]) {
  line_solve_rpl<T, NR, 2>(seg, k0, len, f, buf, bstride, dst);
}

// FP32 solves stop when ||r|| has not halved for this many iterations (see the phase-1 test)
#ifndef LNS_STAG_ITERS
#define LNS_STAG_ITERS 40
#endif
constexpr int kStagIters = LNS_STAG_ITERS;

// length class of a line block: 0..3 for len <= 8, 16, 32, 64 (segments of 4 << c lanes, two rows
// per lane), 4 above (a whole warp)
__device__ __forceinline__ int line_class(int len) {
  return len <= 8 ? 0 : (len <= 16 ? 1 : (len <= 32 ? 2 : (len <= 64 ? 3 : 4)));
}

// Systems of more rows than this (vectors and matrix of ~500 B a row in FP32: about the 126 MB L2)
// prefetch each thread's next rows into L2 (see the grid solver's row loop).
constexpr int kPrefetchRows = 200000;
// L2 prefetch of the line holding a global address (no register result, no wait)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// row_product over a staged row whose neighbours are given by the shared::cluster address of their
// entry in the owner CTA's first vector array (0xffffffff: an inactive column), so that no owner
// search or address map is repeated in the iterations.
template <typename T, typename LoadF, typename CombF>
__device__ __forceinline__ typename V2<T>::t row_product_cla(const unsigned* adr, const B4<T>* blk, int deg,
                                                             typename V2<T>::t own, LoadF load, CombF comb) {
  using V = typename V2<T>::t;
  using Raw = decltype(load(0u));
  constexpr int kBatch = sizeof(T) == 8 ? 2 : 4;
  V acc0 = own, acc1 = mk<T>(0, 0);
  for (int j = 0; j < deg; j += kBatch) {
    unsigned c[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; q++) c[q] = j + q < deg ? adr[j + q] : 0xffffffffu;
    Raw raw[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; q++)
      if (c[q] != 0xffffffffu) raw[q] = load(c[q]);
#pragma unroll
    for (int q = 0; q < kBatch; q++)
      if (c[q] != 0xffffffffu) {
        const V xv = comb(raw[q]);
        const B4<T> bq = blk[j + q];
        V& acc = (q & 1) ? acc1 : acc0;
        acc.x += bq.a * xv.x + bq.b * xv.y;
        acc.y += bq.c * xv.x + bq.d * xv.y;
      }
  }
  return mk<T>(acc0.x + acc1.x, acc0.y + acc1.y);
}

// ---- grid barrier --------------------------------------------------------------------------
// All blocks of the (cooperative, hence co-resident) launch add to one counter (zeroed before the
// launch): block 0 adds 2^31 - (nb - 1), the others 1, so each barrier adds exactly 2^31 and the
// counter's top bit flips when the last block arrives; after barrier g it equals g & 1.  The adds
// are fire-and-forget reductions with release semantics and the waits are acquire loads, so a
// block pays no round trip for its own arrival.  Every wait is bounded: after kBarrierTimeoutNs
// the block records a timeout and stops waiting, and the kernel ends its loop at the next check
// (the host reports an error).  Block barriers on both sides.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// gen: 1 for the first barrier of the launch, 2 for the second, ...
// skip: this block does not arrive (injected fault: every wait of this barrier then runs out)
__device__ __forceinline__ void grid_barrier(IterCounters* ctr, unsigned nb, unsigned gen, bool skip = false) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!skip) red_release_add(&ctr->bar_count, blockIdx.x == 0 ? 0x80000000u - (nb - 1u) : 1u);
    const unsigned want = (gen & 1u) << 31;
    const unsigned long long t0 = global_ns();
    unsigned k = 0;
    while ((ld_acquire(&ctr->bar_count) & 0x80000000u) != want) {
      if ((++k & 63u) == 0u && global_ns() - t0 > kBarrierTimeoutNs) {
        atomicExch(&ctr->bar_timeout, 1);
        break;
      }
    }
  }
  __syncthreads();
}

// ---- the solver --------------------------------------------------------------------------
// A matrix row: off >= 0 is its first entry in the shared-memory pool, off < 0 encodes its first
// CSR entry e0 as -(e0 + 1) (global memory); deg entries; line: a fracture-line row.
struct RowRef {
  int off, deg, line;
};

// Rows are split into one contiguous chunk per block, by cost (weighted_edge: a line row counts
// more), whose ends are moved forward so that no fracture-line block straddles two chunks: a block solves its own line blocks after a block
// barrier, from inputs its threads left in a block buffer.  Dynamic shared memory of a block:
// the references of its first kRowsCached rows per thread, the line input buffer (two float2
// per row), the line factors of its first kFacRows rows, the line-block table, and the pool of
// staged matrix rows (columns and blocks).
constexpr int kBufRows = 2048;   // chunk rows whose line inputs fit the shared buffer
constexpr int kFacRows = 512;    // chunk rows whose line factors are staged
constexpr int kLineList = 1024;  // line blocks of a chunk listed in shared memory (else in d.lsort)
constexpr size_t kSmRref = (size_t)kRowsCached * kKryBlk * sizeof(RowRef);
constexpr size_t kSmBuf = (size_t)2 * kBufRows * sizeof(float2);
constexpr size_t kSmFac = fac_slots(kFacRows) * sizeof(float4);
constexpr size_t kSmLines = (size_t)kLineList * sizeof(int2);
constexpr size_t kSmPool = kKrySmem - kSmRref - kSmBuf - kSmFac - kSmLines;

// First row >= k that does not continue a line block (the end of a chunk starting or ending at
// k), found 32 rows at a time by one warp; valid in all lanes.
__device__ __forceinline__ int chunk_edge(const Dev& d, int k, int nA) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int q = k + lane;
    bool inside = false;
    if (q < nA) inside = __ldg(&d.line_row_flag[q]) == 2 && !((__ldg(&d.lblk[q >> 5]) >> (q & 31)) & 1u);
    const unsigned m = __ballot_sync(0xffffffffu, !inside);
    if (m) return min(nA, k + __ffs(m) - 1);
    k += 32;
  }
}

// First index q in [0, n) with pred(q) true, pred false then true along q (n if none), by one warp
// in steps that narrow the range 32-fold; valid in all lanes.
template <typename Pred>
__device__ __forceinline__ int warp_first(int n, Pred pred) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) / 32;
    const int q = lo + lane * step;
    // samples at or beyond hi count as true (the answer is at most hi)
    const unsigned m = __ballot_sync(0xffffffffu, q >= hi || pred(q));
    const int f = m ? __ffs(m) - 1 : 32;  // first true sample
    const int nhi = f < 32 ? min(hi, lo + f * step) : hi;
    if (f > 0) lo += (f - 1) * step;      // sample f-1 is false
    hi = nhi;
  }
  const int q = lo + lane;
  const unsigned m = __ballot_sync(0xffffffffu, q < hi && pred(q));
  return m ? lo + __ffs(m) - 1 : hi;
}

// First index l with line_start[l] >= k (line_start ascending, n entries); valid in all lanes.
__device__ __forceinline__ int line_lower_bound(const int* ls, int n, int k) {
  return warp_first(n, [&](int q) { return __ldg(&ls[q]) >= k; });
}

// Where the grid solver's row chunk b of nb starts.  A fracture-line row costs a different amount
// than another row (its line solve follows its product, its product is cheaper), so the rows are
// split by cost: 2 units per row plus w per line row (Dev::line_w, -2 < w; w < 0 where line rows
// are the cheaper ones).  The cost of rows [0, k) is 2 k + w LR(k), LR(k) the line rows among
// them (line_cum at the line-block starts); chunk b starts where that cost reaches b / nb of the
// total, and a start inside a line block moves to the nearer end of the block.  Nondecreasing in
// b, 0 at b = 0 and n_A at b = nb.  One warp; valid in all lanes.
__device__ __forceinline__ int weighted_edge(const Dev& d, int w, int b, int nb, int nA, int nl) {
  const long long tot = 2LL * nA + (long long)w * __ldg(&d.line_cum[nl]);
  const long long T = tot * b / nb;
  // cost of the rows before line block l: 2 s_l + w line_cum[l], ascending in l
  auto key = [&](int l) { return 2LL * __ldg(&d.line_start[l]) + (long long)w * __ldg(&d.line_cum[l]); };
  const int f = warp_first(nl, [&](int l) { return key(l) > T; });
  if (f == 0) return (int)min(T / 2, (long long)nA);  // before the first line block
  const int s = __ldg(&d.line_start[f - 1]), len = __ldg(&d.line_len[s]);
  const long long ks = key(f - 1), ke = ks + (2 + w) * (long long)len;
  if (T < ke) return T - ks < ke - T ? s : s + len;
  return (int)min(s + len + (T - ke) / 2, (long long)nA);
}

template <typename T, bool LINES, int BATCH>
__global__ void __launch_bounds__(kKryBlk, 1) k_bicgstab(Dev d, double rtol, int maxit, int cl_cap) {
  using V = typename V2<T>::t;
  using B = B4<T>;
  using Ref = RowRef;
  using Acc = typename DotAcc<T>::t;
  constexpr bool kF64 = sizeof(T) == 8;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double sh[kWarps];
  __shared__ DF s_df[4 * kWarps];
  using S = std::conditional_t<kF64, double, DF>;  // recurrence scalars
  __shared__ S s_sc[4];       // beta, alpha_prev, omega_prev, alpha
  __shared__ int s_ctl;       // 0 continue, 1 stop
  __shared__ int s_epool;     // next free entry of the shared-memory pool
  __shared__ int s_rng[4];    // chunk start, chunk end, first line block, line-block count
  // line blocks by length class c: len <= 8 << c in segments (c < 4), longer ones one per warp (c = 4)
  __shared__ int s_ccount[5], s_coff[5], s_cfill[5], s_citem[6];
  const int nA = d.ctr->n_active;
  if (nA <= cl_cap && *d.fault != 1) return;  // the cluster solver takes this system (uniform exit)
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nlines = LINES ? d.ctr->n_lines : 0;
  unsigned bar_gen = 0;  // grid barriers passed so far
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
  double* part = d.partials;
  Ref* s_rref = (Ref*)dsm;
  float2* s_buf = (float2*)(dsm + kSmRref);
  float4* s_fac = (float4*)(dsm + kSmRref + kSmBuf);
  int2* s_lines = (int2*)(dsm + kSmRref + kSmBuf + kSmFac);
  const int ecap = (int)(kSmPool / (sizeof(int) + sizeof(B)));
  B* s_blk = (B*)(dsm + kKrySmem - kSmPool);
  int* s_col = (int*)(dsm + kKrySmem - kSmPool + (size_t)ecap * sizeof(B));

  // ---- this block's rows and line blocks ------------------------------------------------
  // warp 0 finds where the chunk starts, warp 1 where it ends (the next chunk's start), at once
  if (wib < 2) {
    const int e = (int)blockIdx.x + wib;
    const int rpb = (nA + nb - 1) / nb;
    int c = (int)min((long long)nA, (long long)e * rpb);
    if (LINES && nlines > 0) c = weighted_edge(d, d.line_w[sizeof(T) == 4 ? 1 : 0], e, nb, nA, nlines);
    if (LINES) c = chunk_edge(d, c, nA);
    int l = 0;
    if (LINES && nlines > 0) l = line_lower_bound(d.line_start, nlines, c);
    if (lane == 0) {
      s_rng[wib] = c;
      s_rng[2 + wib] = l;
      if (wib == 0) {
        s_epool = 0;
        for (int q = 0; q < 5; q++) s_ccount[q] = 0;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // start, end, first line block, line-block count
    s_rng[1] = max(s_rng[0], s_rng[1]);
    s_rng[3] = max(0, s_rng[3] - s_rng[2]);
  }
  __syncthreads();
  const int r0 = s_rng[0], r1 = s_rng[1], l0 = s_rng[2], nlb = s_rng[3];
  const int kbeg = r0 + (int)threadIdx.x, kstep = blockDim.x;
  const bool busy = __any_sync(0xffffffffu, kbeg < r1) || (LINES && wib < nlb);  // adds to the dots
  // line inputs: the shared buffer, or (a chunk too long for it) global scratch, two float2 per row
  const bool buf_sm = r1 - r0 <= kBufRows;
  float2* const lbuf = buf_sm ? s_buf : (float2*)d.kls + 2 * (size_t)r0;
  const int bstride = buf_sm ? kBufRows : r1 - r0;

  auto global_ref = [&](int k) -> Ref {
    const int2 a = __ldg(&d.arow[k]);
    return {-(a.x + 1), a.y & 0xffffff, LINES ? (a.y >> 24) : 0};
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
    return {off, g.deg, g.line};
  };
  // product of a row with a vector whose own value is `own` and whose neighbour values are
  // comb(load(j))
  auto product = [&](const Ref& ref, const V& own, auto load, auto comb) -> V {
    if (ref.off >= 0) return row_product<T, BATCH>(s_col + ref.off, s_blk + ref.off, ref.deg, own, load, comb);
    const size_t e0 = (size_t)(-(ref.off + 1));
    return row_product<T, BATCH>(d.colA + e0, (const B*)&blocks[4 * e0], ref.deg, own, load, comb);
  };
  for (int q = 0; q < kRowsCached; q++) {
    const int k = kbeg + q * kstep;
    if (k < r1) s_rref[q * kKryBlk + threadIdx.x] = stage(k);
  }
  if (LINES) {
    for (int k = kbeg; k < min(r1, r0 + kFacRows); k += kstep)
      if (__ldg(&d.line_row_flag[k])) {
        float4* f = &s_fac[fac_slot(k - r0)];
        f[0] = __ldg((const float4*)d.line_dinv + k);
        f[1] = __ldg((const float4*)d.line_a + k);
        f[2] = __ldg((const float4*)d.line_g + k);
      }
    // list the chunk's line blocks by length class (the order inside a class does not matter: each
    // block is solved alone, the same way wherever it sits), in shared memory or, for a chunk with
    // more line blocks than that holds, in the chunk's own range of d.lsort
    {
      int2* const ltab = nlb <= kLineList ? s_lines : d.lsort + l0;
      for (int j = threadIdx.x; j < nlb; j += kstep)
        atomicAdd(&s_ccount[line_class(__ldg(&d.line_len[__ldg(&d.line_start[l0 + j])]))], 1);
      __syncthreads();
      if (threadIdx.x == 0) {
        int off = 0;
        s_citem[0] = 0;
        for (int c = 0; c < 5; c++) {
          s_coff[c] = off;
          s_cfill[c] = off;
          off += s_ccount[c];
          const int per = c < 4 ? 8 >> c : 1;  // line blocks per warp item
          s_citem[c + 1] = s_citem[c] + (s_ccount[c] + per - 1) / per;
        }
      }
      __syncthreads();
      for (int j = threadIdx.x; j < nlb; j += kstep) {
        const int k0 = __ldg(&d.line_start[l0 + j]);
        const int len = __ldg(&d.line_len[k0]);
        ltab[atomicAdd(&s_cfill[line_class(len)], 1)] = make_int2(k0, len);
      }
    }
  }
  __syncthreads();
  const int2* const ltab = nlb <= kLineList ? s_lines : d.lsort + l0;

  // fn(k, ref) over this thread's rows of the chunk (one call site: one copy of the row code).  A
  // software pipeline over the thread's rows: the reference of the row after next is loaded before
  // the current row is processed, and on systems larger than L2 (kPrefetchRows) the next row's
  // matrix entries (from its reference, loaded an iteration earlier) and own vector entries (pf) are
  // prefetched into L2, so that a row waits for L2 rather than DRAM.
  auto ref_of = [&](int k, int q) -> Ref { return q < kRowsCached ? s_rref[q * kKryBlk + threadIdx.x] : global_ref(k); };
  auto prefetch_row = [&](const Ref& ref) {
    if (ref.off < 0 && ref.deg > 0) {  // entries e0 .. e0 + deg - 1, all in bounds
      const size_t e0 = (size_t)(-(ref.off + 1));
      prefetch_l2(d.colA + e0);
      const T* bl = &blocks[4 * e0];
      prefetch_l2(bl);
      prefetch_l2(bl + 4 * (size_t)(ref.deg - 1));
    }
  };
  const bool big = nA > kPrefetchRows;
  auto rows = [&](auto fn, auto pf) {
    if (kbeg >= r1) return;
    Ref ref = ref_of(kbeg, 0);
    Ref nref = kbeg + kstep < r1 ? ref_of(kbeg + kstep, 1) : ref;
#pragma unroll 1
    for (int k = kbeg, q = 0;; q++) {
      const int kn = k + kstep, knn = kn + kstep;
      Ref nnref = nref;
      if (knn < r1) nnref = ref_of(knn, q + 2);
      if (big && kn < r1) {
        prefetch_row(nref);
        pf(kn);
      }
      fn(k, ref);
      if (kn >= r1) break;
      k = kn;
      ref = nref;
      nref = nnref;
    }
  };
  // after a block barrier: M^{-1} on this block's line blocks.  The warps share out items: 32 / seg
  // short blocks of one length class in segments of seg lanes, or one block longer than 32 rows.
  // solvefn(k0, len, factors, inputs, seg), seg = 0 for a whole-warp multi-chunk solve.
  auto lines = [&](auto solvefn) {
    if constexpr (LINES) {
      __syncthreads();
      auto fac = [&](const int2& kl) -> LineFac {
        const int o = kl.x - r0;
        return o + kl.y <= kFacRows ? LineFac{s_fac, s_fac + 1, s_fac + 2, o, 3, 1}
                                    : LineFac{(const float4*)d.line_dinv + kl.x, (const float4*)d.line_a + kl.x,
                                              (const float4*)d.line_g + kl.x, 0, 1, 0};
      };
      const int nit = s_citem[5];
#pragma unroll 1
      for (int it = wib; it < nit; it += kWarps) {
        int c = 0;
        while (c < 4 && it >= s_citem[c + 1]) c++;
        const int idx = it - s_citem[c];
        if (c < 4) {
          const int seg = 4 << c, li = idx * (8 >> c) + (lane >> (c + 2));
          const int2 kl = li < s_ccount[c] ? ltab[s_coff[c] + li] : make_int2(r0, 0);
          solvefn(kl.x, kl.y, fac(kl), lbuf + (kl.x - r0), seg);
        } else {
          const int2 kl = ltab[s_coff[4] + idx];
          solvefn(kl.x, kl.y, fac(kl), lbuf + (kl.x - r0), 0);
        }
      }
    }
  };

  // ---- initialisation: x = x_0 (0, or with krylov_warm the FP32 iterate in kx0), z = t = t~ =
  // y_0 = v~_0 = 0, s = r^ = r_0 = b - A x_0, z^ = M^{-1} r_0 ----------------------------------
  const bool warm = d.krylov_warm != 0;
  auto x0_of = [&](int j) -> V {
    const float2 f = ((const float2*)d.kx0)[j];
    return mk<T>((T)f.x, (T)f.y);
  };
  double l_bb = 0.0, l_rr0 = 0.0;
  rows([&](int k, const Ref& ref) {
    const V bk = b[k];
    const V o = mk<T>(0, 0);
    V rk = bk;
    if (warm) {
      const V xk = x0_of(k);
      const V ax = product(ref, xk, x0_of, [](const V& u) { return u; });
      rk = mk<T>(bk.x - ax.x, bk.y - ax.y);
      x[k] = xk;
    } else {
      x[k] = o;
    }
    z[k] = o;
    t[k] = o;
    tt[k] = o;
    y0[k] = o;
    vt0[k] = o;
    s[k] = rk;
    rh[k] = rk;
    l_bb += (double)bk.x * bk.x + (double)bk.y * bk.y;
    l_rr0 += (double)rk.x * rk.x + (double)rk.y * rk.y;
    if (LINES && ref.line)
      lbuf[k - r0] = make_float2((float)rk.x, (float)rk.y);
    else
      zf[k] = rk;
  }, [&](int) {});
  lines([&](int k0, int len, const LineFac& f, float2* buf, int seg) {
    V* const dst[1] = {zf};
    if (seg)
      line_solve_seg<T, 1>(seg, k0, len, f, buf, bstride, dst);
    else
      line_solve<T, 1>(k0, len, f, buf, bstride, dst);
  });
  // injected faults (failure tests): 1 = block 0 never arrives at this barrier, 2 = rho_1 = 0,
  // 3 = rho_1 = 0 in FP32 solves only
  const int fault = *d.fault;
  block_store_f64(l_bb, sh, part, nb, kSlotInit);
  if (warm) {
    __syncthreads();
    block_store_f64(l_rr0, sh, part, nb, kSlotInit + 1);
  }
  grid_barrier(d.ctr, nb, ++bar_gen, fault == 1 && blockIdx.x == 0);
  const bool timed_out = *(volatile int*)&d.ctr->bar_timeout;
  // ||b||^2 (and ||r_0||^2) are summed by warp 0; every thread scales its dot products by the same
  // power of two
  __shared__ double s_bbv, s_rrv;
  {
    const double bb0 = grid_sum_f64(part, nb, kSlotInit);
    const double rr0 = warm ? grid_sum_f64(part, nb, kSlotInit + 1) : bb0;
    if (threadIdx.x == 0) {
      s_bbv = bb0;
      s_rrv = rr0;
    }
  }
  __syncthreads();
  const double bb = s_bbv, rr0 = s_rrv;
  // Dots are scaled by an exact power of two near 1/bb before they are carried in double-float,
  // so that the reductions and the scalar arithmetic stay far from the FP32 range limits (the
  // scalars are ratios of dots and do not depend on the scale).  2^(1023 - E) with E the unbiased
  // exponent of bb, clamped to what FP32 represents exactly.
  long long eb = bb > 0.0 ? ((__double_as_longlong(bb) >> 52) & 0x7ff) - 1023 : 0;
  eb = eb < -126 ? -126 : (eb > 126 ? 126 : eb);
  const double dscale = __longlong_as_double((1023 - eb) << 52);
  const float fscale = (float)dscale;
  auto to_df = [&](const Acc& a) -> DF {
    if constexpr (kF64)
      return dot_df(a, dscale);
    else
      return dot_df(a, fscale);
  };
  S rho, alpha, stop2, rr_last, rr_ref;
  sc_zero(rho);
  sc_zero(alpha);
  sc_zero(stop2);
  sc_zero(rr_last);
  sc_zero(rr_ref);
  int it_ref = 0;  // FP32 stagnation test: iteration at which ||r||^2 last fell below rr_ref / 4
  if (threadIdx.x == 0) {  // thread 0 tracks the scalars
    rho = sc_from(df_from(fault == 2 || (fault == 3 && sizeof(T) == 4) ? 0.0 : rr0 * dscale), S{});
    stop2 = sc_from(df_from(rtol * rtol * bb * dscale), S{});
    rr_ref = sc_from(df_from(rr0 * dscale), S{});
    sc_zero(s_sc[0]);  // beta_1
    sc_zero(s_sc[1]);  // alpha_0
    sc_zero(s_sc[2]);  // omega_0
    s_ctl = timed_out ? 1 : 0;
  }
  __syncthreads();
  int status = timed_out ? 3 : 1, it = 1;
  for (it = 1; !s_ctl; it++) {
    // ---- phase 1 -------------------------------------------------------------------------
    const T beta = sc_t<T>(s_sc[0]), alp = sc_t<T>(s_sc[1]), omp = sc_t<T>(s_sc[2]);
    const T nom = -omp;
    const bool odd = it & 1;
    const V* yo = odd ? y0 : y1;
    V* yn = odd ? y1 : y0;
    const V* vto = odd ? vt0 : vt1;
    V* vtn = odd ? vt1 : vt0;
    // y_i of a row from stored vectors: r~_{i-1} = z^ - omega t~, y_i = r~ + beta (y_{i-1} - omega v~);
    // the owner evaluates the same expressions on the same values
    struct Raw1 {
      V tt, zf, vt, y;
    };
    auto ld1 = [&](int c) { return Raw1{ldv(&tt[c]), ldv(&zf[c]), ldv(&vto[c]), ldv(&yo[c])}; };
    auto rt_of = [&](const Raw1& a) { return axpy(nom, a.tt, a.zf); };
    auto y_of = [&](const Raw1& a, const V& rtc) { return axpy(beta, axpy(nom, a.vt, a.y), rtc); };
    auto cb1 = [&](const Raw1& a) { return y_of(a, rt_of(a)); };
    Acc l_rv, l_rr;
    dot_zero(l_rv);
    dot_zero(l_rr);
    // all loads of a row (own and neighbours) are issued before its stores
    rows([&](int k, const Ref& ref) {
      const V xk = ldv(&x[k]), zk = ldv(&z[k]), sk = ldv(&s[k]), tk = ldv(&t[k]), rhk = ldv(&rh[k]);
      const Raw1 own = ld1(k);
      const V rtk = rt_of(own);
      const V ynk = y_of(own, rtk);
      const V vv = product(ref, ynk, ld1, cb1);
      const V rk = axpy(nom, tk, sk);
      x[k] = mk<T>(xk.x + alp * own.y.x + omp * zk.x, xk.y + alp * own.y.y + omp * zk.y);
      r[k] = rk;
      if (LINES) rt[k] = rtk;
      yn[k] = ynk;
      v[k] = vv;
      if (LINES && ref.line)
        lbuf[k - r0] = make_float2((float)vv.x, (float)vv.y);
      else
        vtn[k] = vv;
      dot_acc(l_rr, rk.x, rk.x);
      dot_acc(l_rr, rk.y, rk.y);
      dot_acc(l_rv, rhk.x, vv.x);
      dot_acc(l_rv, rhk.y, vv.y);
    }, [&](int kp) {
      prefetch_l2(&x[kp]);
      prefetch_l2(&z[kp]);
      prefetch_l2(&s[kp]);
      prefetch_l2(&t[kp]);
      prefetch_l2(&rh[kp]);
      prefetch_l2(&tt[kp]);
      prefetch_l2(&zf[kp]);
      prefetch_l2(&vto[kp]);
      prefetch_l2(&yo[kp]);
    });
    lines([&](int k0, int len, const LineFac& f, float2* buf, int seg) {
      V* const dst[1] = {vtn};
      if (seg)
        line_solve_seg<T, 1>(seg, k0, len, f, buf, bstride, dst);
      else
        line_solve<T, 1>(k0, len, f, buf, bstride, dst);
    });
    {
      const DF vals[2] = {to_df(l_rv), to_df(l_rr)};
      block_store<2>(vals, busy, s_df, part, kSlotS1, nb);
    }
    grid_barrier(d.ctr, nb, ++bar_gen);
    {
      DF o[2];
      grid_sum<2>(part, kSlotS1, nb, o);
      if (threadIdx.x == 0) {
        const S rv = sc_from(o[0], S{});
        rr_last = sc_from(o[1], S{});
        if (sc_le(sc_mul(rr_last, sc_from(df_from(4.0), S{})), rr_ref)) {
          rr_ref = rr_last;
          it_ref = it;
        }
        if (*(volatile int*)&d.ctr->bar_timeout) {
          s_ctl = 1;
          status = 3;
        } else if (sc_le(rr_last, stop2)) {
          s_ctl = 1;
          status = 0;
        } else if (it > maxit || (!kF64 && fault == 4 && it > 1)) {  // (4: an injected stall)
          s_ctl = 1;
          status = 1;
        } else if (!kF64 && it - it_ref > kStagIters) {
          // FP32 stagnation: ||r|| has not halved in kStagIters iterations, the FP32 rounding
          // floor of this system is near; stop as at maxit (accepted as an inexact Newton step
          // when ||r|| / ||b|| <= krylov_fail_rtol, else redone in FP64 by the host)
          s_ctl = 1;
          status = 1;
        } else if (!sc_ok(rv) || !sc_ok(rho)) {
          s_ctl = 1;
          status = 2;
        } else {
          alpha = sc_div(rho, rv);
          s_sc[3] = alpha;
        }
      }
    }
    __syncthreads();
    if (s_ctl) break;
    // ---- phase 2 -------------------------------------------------------------------------
    const T nal = -sc_t<T>(s_sc[3]);
    // z_i of a row: r~_{i-1} - alpha v~_i (the owner evaluates the same expression)
    auto ld2 = [&](int c) { return V2pair<V>{ldv(&vtn[c]), ldv(&rt[c])}; };
    auto cb2 = [&](const V2pair<V>& a) { return axpy(nal, a.a, a.b); };
    Acc l_ts, l_tt, l_rs, l_rt;
    dot_zero(l_ts);
    dot_zero(l_tt);
    dot_zero(l_rs);
    dot_zero(l_rt);
    rows([&](int k, const Ref& ref) {
      const V rk = ldv(&r[k]), vk = ldv(&v[k]), rhk = ldv(&rh[k]);
      const V zk = cb2(ld2(k));
      const V tk = product(ref, zk, ld2, cb2);
      const V sk = axpy(nal, vk, rk);
      s[k] = sk;
      z[k] = zk;
      t[k] = tk;
      if (LINES && ref.line) {
        lbuf[k - r0] = make_float2((float)sk.x, (float)sk.y);
        lbuf[bstride + k - r0] = make_float2((float)tk.x, (float)tk.y);
      } else if (LINES) {
        zf[k] = sk;
        tt[k] = tk;
      }
      dot_acc(l_ts, tk.x, sk.x);
      dot_acc(l_ts, tk.y, sk.y);
      dot_acc(l_tt, tk.x, tk.x);
      dot_acc(l_tt, tk.y, tk.y);
      dot_acc(l_rs, rhk.x, sk.x);
      dot_acc(l_rs, rhk.y, sk.y);
      dot_acc(l_rt, rhk.x, tk.x);
      dot_acc(l_rt, rhk.y, tk.y);
    }, [&](int kp) {
      prefetch_l2(&r[kp]);
      prefetch_l2(&v[kp]);
      prefetch_l2(&rh[kp]);
      prefetch_l2(&vtn[kp]);
      prefetch_l2(&rt[kp]);
    });
    lines([&](int k0, int len, const LineFac& f, float2* buf, int seg) {
      V* const dst[2] = {zf, tt};
      if (seg)
        line_solve_seg<T, 2>(seg, k0, len, f, buf, bstride, dst);
      else
        line_solve<T, 2>(k0, len, f, buf, bstride, dst);
    });
    {
      const DF vals[4] = {to_df(l_ts), to_df(l_tt), to_df(l_rs), to_df(l_rt)};
      block_store<4>(vals, busy, s_df, part, kSlotS2, nb);
    }
    grid_barrier(d.ctr, nb, ++bar_gen);
    {
      DF o[4];
      grid_sum<4>(part, kSlotS2, nb, o);
      if (threadIdx.x == 0) {
        const S ts = sc_from(o[0], S{}), t2 = sc_from(o[1], S{}), rs = sc_from(o[2], S{}), rtv = sc_from(o[3], S{});
        if (*(volatile int*)&d.ctr->bar_timeout) {
          s_ctl = 1;
          status = 3;
        } else if (!sc_finite(ts) || !sc_finite(t2) || !sc_finite(rs) || !sc_finite(rtv)) {
          s_ctl = 1;
          status = 2;
        } else {
          // t = 0 means A z = 0: omega = 0 leaves r = s and restarts the direction (beta = 0).
          // Only ratios of dots are formed, so nothing underflows at tight tolerances.
          S omega, beta;
          sc_zero(omega);
          sc_zero(beta);
          if (sc_pos(t2)) omega = sc_div(ts, t2);
          const S rho_new = sc_fnma(omega, rtv, rs);
          if (sc_nonzero(omega)) beta = sc_mul(sc_div(rho_new, rho), sc_div(alpha, omega));
          s_sc[0] = beta;
          s_sc[1] = alpha;
          s_sc[2] = omega;
          rho = rho_new;
        }
      }
    }
    __syncthreads();
    if (s_ctl) break;
  }
  // x holds x_{it-1} at every exit; thread 0 of block 0 reports
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr->krylov_iters = it - 1;
    d.ctr->krylov_status = status;
    d.ctr->krylov_solver = 2;
    d.ctr->krylov_relres = bb > 0.0 ? sqrt(sc_double(rr_last) / (bb * dscale)) : 0.0;
  }
}

// =========================================================================================
// Cluster BiCGStab for small local systems.
//
// The same recurrence as k_bicgstab, run by ONE thread-block cluster of C CTAs (C <= 16) instead
// of a cooperative grid over every SM.  The local systems of the localized method are small
// (thousands of rows), so an iteration of the grid solver is bound by latency: two ~1 us grid
// barriers, L2 round trips for every neighbour gather and for the 152 block partials.  Here:
//   - each CTA owns a contiguous chunk of rows (ends never split a fracture-line block, as in the
//     grid solver); a row's own vectors (x, r, r^, v, s, t, z) stay in the owning thread's
//     registers for the whole solve, the vectors its neighbours read (y, v~ of both parities, r~,
//     t~, z^) sit in the CTA's shared memory, indexed by local row;
//   - a neighbour in another CTA of the cluster is read through distributed shared memory
//     (mapa + ld.shared::cluster), so no vector goes through L2 during the iterations;
//   - a reduction is a block reduction into the CTA's shared memory, one barrier.cluster
//     (arrive.release / wait.acquire), and a read of the C partials by DSMEM in a fixed order, so
//     every CTA holds identical scalars; the cluster barrier is a hardware barrier of CTAs the
//     launch guarantees co-scheduled (no spin-wait);
//   - matrix rows (columns and blocks), row references and line factors are staged in shared
//     memory once per solve (rows beyond the pool are read from L2).
// The kernel and the grid solver are both launched for every solve; a size test on the device
// (n_A <= cap, computed by the host from C and the chunk capacity) makes exactly one of them run
// it, so the choice needs no host round trip and fits a captured CUDA graph.
// =========================================================================================
constexpr int kClThreads = 256;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClMaxCtas = 16;
template <typename T>
struct ClShape {
  static constexpr int kRpt = sizeof(T) == 4 ? 4 : 2;  // rows per thread (own vectors in registers)
  static constexpr int kRows = kClThreads * kRpt;       // rows per CTA
};
constexpr int kClLineList = 1024;
constexpr size_t kClSmem = 220 * 1024;

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// all threads of all CTAs of the cluster; shared-memory writes before it are visible to
// ld.shared::cluster of any CTA after it
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// (mapa is a pure address map, so the compiler may schedule it freely)
__device__ __forceinline__ unsigned cl_addr(const void* local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// A vector entry at a shared::cluster address (this CTA's or another's).
__device__ __forceinline__ void ld_cla(unsigned a, float2& v) {
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
}
__device__ __forceinline__ void ld_cla(unsigned a, double2& v) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
}
// A neighbour's vector entry in another CTA's shared memory.  Within a phase no thread writes what
// these loads read (that happened before the last cluster barrier, whose asm orders them), so they
// carry no memory clobber: the compiler may issue a row's loads ahead of the previous row's
// arithmetic and stores.
__device__ __forceinline__ float2 ld_cl(const float2* local, unsigned rank) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(cl_addr(local, rank)));
  return v;
}
__device__ __forceinline__ double2 ld_cl(const double2* local, unsigned rank) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(cl_addr(local, rank)));
  return v;
}
__device__ __forceinline__ double ld_cl(const double* local, unsigned rank) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(cl_addr(local, rank)) : "memory");
  return v;
}

// Sum of NV double-float values over the cluster: block reduction into this CTA's s_part, one
// cluster barrier, then warp 0 reads the C partials (lane c from CTA c) and reduces them in a fixed
// tree; thread 0 holds the result (identical in every CTA).
template <int NV>
__device__ __forceinline__ void cl_sum(const DF (&vals)[NV], bool busy, DF* sdf, float2* s_part, unsigned C,
                                       DF (&out)[NV]) {
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
    for (int q = 0; q < NV; q++) sdf[q * kClWarps + w] = a[q];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) a[q] = lane < kClWarps ? sdf[q * kClWarps + lane] : DF{0.f, 0.f};
#pragma unroll
    for (int o = kClWarps / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; q++) a[q] = df_add(a[q], df_shfl_xor(a[q], o));
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; q++) s_part[q] = make_float2(a[q].hi, a[q].lo);
  }
  cl_sync();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      const float2 x = lane < (int)C ? ld_cl(&s_part[q], (unsigned)lane) : make_float2(0.f, 0.f);
      a[q] = {x.x, x.y};
    }
#pragma unroll
    for (int o = kClMaxCtas / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; q++) a[q] = df_add(a[q], df_shfl_xor(a[q], o));
  }
#pragma unroll
  for (int q = 0; q < NV; q++) out[q] = a[q];
}

template <typename T, bool LINES>
__global__ void __launch_bounds__(kClThreads, 1) k_bicgstab_cl(Dev d, double rtol, int maxit, int cap) {
  using V = typename V2<T>::t;
  using B = B4<T>;
  using Ref = RowRef;
  using Acc = typename DotAcc<T>::t;
  constexpr bool kF64 = sizeof(T) == 8;
  constexpr int RPT = ClShape<T>::kRpt;
  constexpr int R = ClShape<T>::kRows;
  const int nA = d.ctr->n_active;
  if (nA > cap || *d.fault == 1) return;  // the grid solver takes this system (uniform exit)
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double sh[kClWarps], sh2[kClWarps];
  __shared__ double s_bb, s_rr0;
  __shared__ DF s_df[4 * kClWarps];
  __shared__ float2 s_part[2][4];  // this CTA's partial sums: [0] phase 1 / init, [1] phase 2
  using S = std::conditional_t<kF64, double, DF>;
  __shared__ S s_sc[4];
  __shared__ int s_ctl, s_epool, s_nlb, s_l0;
  __shared__ int s_cb[kClMaxCtas + 1];
  __shared__ int s_ccount[5], s_coff[5], s_cfill[5], s_citem[6];
  const unsigned C = cl_size(), me = cl_rank();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nlines = LINES ? d.ctr->n_lines : 0;
  // shared-memory layout: neighbour-read vectors [7][R] (y0, y1, vt0, vt1, r~, t~, z^), line inputs
  // [2][R], line factors [3][R], row references [R], line-block list, then the matrix pool
  V* const s_vec = (V*)dsm;
  V* const sy[2] = {s_vec, s_vec + R};
  V* const svt[2] = {s_vec + 2 * R, s_vec + 3 * R};
  V* const srt = s_vec + 4 * R;
  V* const stt = s_vec + 5 * R;
  V* const szf = s_vec + 6 * R;
  float2* const lbuf = (float2*)(dsm + 7 * (size_t)R * sizeof(V));
  float4* const s_fac = (float4*)((unsigned char*)lbuf + 2 * (size_t)R * sizeof(float2));
  Ref* const s_ref = (Ref*)((unsigned char*)s_fac + fac_slots(R) * sizeof(float4));
  int2* const s_lines = (int2*)((unsigned char*)s_ref + (size_t)R * sizeof(Ref));
  unsigned char* const pool = (unsigned char*)s_lines + (size_t)kClLineList * sizeof(int2);
  const size_t pool_bytes = kClSmem - (size_t)(pool - dsm);
  const int ecap = (int)(pool_bytes / (sizeof(int) + sizeof(B)));
  B* const s_blk = (B*)pool;
  int* const s_col = (int*)(pool + (size_t)ecap * sizeof(B));
  const T* blocks = (const T*)d.blocks;
  const V* b = (const V*)d.rhs;

  // ---- chunk boundaries of every CTA (identical in all CTAs) -----------------------------
  {
    const int R0 = (nA + (int)C - 1) / (int)C;
    for (int w = wib; w < (int)C; w += kClWarps) {  // warp-uniform
      if (w == 0) continue;
      int e = min(nA, w * R0);
      if (LINES) e = chunk_edge(d, e, nA);
      if (lane == 0) s_cb[w] = e;
    }
    if (threadIdx.x == 0) {
      s_cb[0] = 0;
      s_cb[C] = nA;
      s_epool = 0;
      for (int c = 0; c < 5; c++) s_ccount[c] = 0;
    }
  }
  __syncthreads();
  const int c0 = s_cb[me], c1 = max(c0, s_cb[me + 1]);
  const int nr = c1 - c0;
  if (LINES && wib == 0) {
    int l0 = 0, l1 = 0;
    if (nlines > 0) {
      l0 = line_lower_bound(d.line_start, nlines, c0);
      l1 = line_lower_bound(d.line_start, nlines, c1);
    }
    if (lane == 0) {
      s_l0 = l0;
      s_nlb = max(0, l1 - l0);
    }
  }
  // owner CTA of compact row j: the last c with s_cb[c] <= j
  // (binary search over the C <= 16 ascending boundaries: four dependent shared loads instead of
  // fifteen compares, on the row phases' instruction-bound path)
  auto owner = [&](int j) -> unsigned {
    unsigned o = 0;
#pragma unroll
    for (unsigned step = kClMaxCtas / 2; step > 0; step >>= 1)
      if (o + step < C && s_cb[o + step] <= j) o += step;
    return o;
  };
  auto global_ref = [&](int k) -> Ref {
    const int2 a = __ldg(&d.arow[k]);
    return {-(a.x + 1), a.y & 0xffffff, LINES ? (a.y >> 24) : 0};
  };
  auto stage = [&](int k) -> Ref {
    const Ref g = global_ref(k);
    const int off = atomicAdd(&s_epool, g.deg);
    if (off + g.deg > ecap) return g;
    const int e0 = -(g.off + 1);
    for (int j = 0; j < g.deg; j++) {
      const int col = __ldg(&d.colA[e0 + j]);
      unsigned a = 0xffffffffu;
      if (col >= 0) {
        const unsigned o = owner(col);
        a = cl_addr(&s_vec[col - s_cb[o]], o);
      }
      s_col[off + j] = (int)a;
      s_blk[off + j] = *(const B*)&blocks[4 * (size_t)(e0 + j)];
    }
    return {off, g.deg, g.line};
  };
  // staged rows read their neighbours by address (loada), the others by compact row (load)
  auto product = [&](const Ref& ref, const V& own, auto loada, auto load, auto comb) -> V {
    if (ref.off >= 0)
      return row_product_cla<T>((const unsigned*)s_col + ref.off, s_blk + ref.off, ref.deg, own, loada, comb);
    const size_t e0 = (size_t)(-(ref.off + 1));
    return row_product<T>(d.colA + e0, (const B*)&blocks[4 * e0], ref.deg, own, load, comb);
  };
  // byte offset of a vector array from the first one (the staged addresses point into that one)
  auto voff = [&](const V* arr) -> unsigned { return (unsigned)((const char*)arr - (const char*)s_vec); };
  __syncthreads();
  const int nlb = LINES ? s_nlb : 0, l0 = LINES ? s_l0 : 0;
  for (int i = threadIdx.x; i < nr; i += kClThreads) {
    s_ref[i] = stage(c0 + i);
    if (LINES && __ldg(&d.line_row_flag[c0 + i])) {
      float4* f = &s_fac[fac_slot(i)];
      f[0] = __ldg((const float4*)d.line_dinv + c0 + i);
      f[1] = __ldg((const float4*)d.line_a + c0 + i);
      f[2] = __ldg((const float4*)d.line_g + c0 + i);
    }
  }
  if (LINES && nlb <= kClLineList) {
    for (int j = threadIdx.x; j < nlb; j += kClThreads)
      atomicAdd(&s_ccount[line_class(__ldg(&d.line_len[__ldg(&d.line_start[l0 + j])]))], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      int off = 0;
      s_citem[0] = 0;
      for (int c = 0; c < 5; c++) {
        s_coff[c] = off;
        s_cfill[c] = off;
        off += s_ccount[c];
        const int per = c < 4 ? 8 >> c : 1;
        s_citem[c + 1] = s_citem[c] + (s_ccount[c] + per - 1) / per;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nlb; j += kClThreads) {
      const int k0 = __ldg(&d.line_start[l0 + j]);
      const int len = __ldg(&d.line_len[k0]);
      s_lines[atomicAdd(&s_cfill[line_class(len)], 1)] = make_int2(k0 - c0, len);  // local start
    }
  }
  __syncthreads();

  // after a block barrier: M^{-1} on this CTA's line blocks (inputs lbuf by local row, outputs by
  // local row); solvefn(k0 local, len, factors, inputs, seg)
  auto lines = [&](auto solvefn) {
    if constexpr (LINES) {
      __syncthreads();
      auto fac = [&](int k0) -> LineFac {
        return LineFac{s_fac, s_fac + 1, s_fac + 2, k0, 3, 1};
      };
      if (nlb <= kClLineList) {
        const int nit = s_citem[5];
#pragma unroll 1
        for (int it = wib; it < nit; it += kClWarps) {
          int c = 0;
          while (c < 4 && it >= s_citem[c + 1]) c++;
          const int idx = it - s_citem[c];
          if (c < 4) {
            const int seg = 4 << c, li = idx * (8 >> c) + (lane >> (c + 2));
            const int2 kl = li < s_ccount[c] ? s_lines[s_coff[c] + li] : make_int2(0, 0);
            solvefn(kl.x, kl.y, fac(kl.x), lbuf + kl.x, seg);
          } else {
            const int2 kl = s_lines[s_coff[4] + idx];
            solvefn(kl.x, kl.y, fac(kl.x), lbuf + kl.x, 0);
          }
        }
      } else {
#pragma unroll 1
        for (int j = wib; j < nlb; j += kClWarps) {
          const int k0 = __ldg(&d.line_start[l0 + j]);
          const int2 kl = make_int2(k0 - c0, __ldg(&d.line_len[k0]));
          solvefn(kl.x, kl.y, fac(kl.x), lbuf + kl.x, 0);
        }
      }
    }
  };

  // ---- own rows: registers --------------------------------------------------------------
  V ox[RPT], o_r[RPT], orh[RPT], ov[RPT], os[RPT], ot[RPT], oz[RPT];
  Ref oref[RPT];
  const V zero = mk<T>(0, 0);
  // x_0 = 0, or with krylov_warm the FP32 iterate in kx0 (r_0 = b - A x_0 over the global rows)
  const bool warm = d.krylov_warm != 0;
  auto x0_of = [&](int j) -> V {
    const float2 f = ((const float2*)d.kx0)[j];
    return mk<T>((T)f.x, (T)f.y);
  };
  double l_bb = 0.0, l_rr0 = 0.0;
#pragma unroll
  for (int q = 0; q < RPT; q++) {
    const int i = threadIdx.x + q * kClThreads;
    ox[q] = zero;
    oz[q] = zero;
    ot[q] = zero;
    ov[q] = zero;
    o_r[q] = zero;
    os[q] = zero;
    orh[q] = zero;
    oref[q] = Ref{0, 0, 0};
    if (i < nr) {
      const V bk = b[c0 + i];
      V rk = bk;
      if (warm) {
        const Ref g = global_ref(c0 + i);
        const size_t e0 = (size_t)(-(g.off + 1));
        ox[q] = x0_of(c0 + i);
        const V ax = row_product<T>(d.colA + e0, (const B*)&blocks[4 * e0], g.deg, ox[q], x0_of,
                                    [](const V& u) { return u; });
        rk = mk<T>(bk.x - ax.x, bk.y - ax.y);
      }
      oref[q] = s_ref[i];
      os[q] = rk;
      orh[q] = rk;
      l_bb += (double)bk.x * bk.x + (double)bk.y * bk.y;
      l_rr0 += (double)rk.x * rk.x + (double)rk.y * rk.y;
      stt[i] = zero;
      sy[0][i] = zero;
      svt[0][i] = zero;
      if (LINES && oref[q].line)
        lbuf[i] = make_float2((float)rk.x, (float)rk.y);
      else
        szf[i] = rk;
    }
  }
  lines([&](int k0, int len, const LineFac& f, const float2* buf, int seg) {
    V* const dst[1] = {szf};
    if (seg)
      line_solve_seg<T, 1>(seg, k0, len, f, buf, R, dst);
    else
      line_solve<T, 1>(k0, len, f, buf, R, dst);
  });
  // ||b||^2 (and ||r_0||^2) over the cluster in FP64
  {
    double a = l_bb, a2 = l_rr0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      sh[wib] = a;
      sh2[wib] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0, t2 = 0.0;
      for (int k = 0; k < kClWarps; k++) {
        t += sh[k];
        t2 += sh2[k];
      }
      s_bb = t;
      s_rr0 = t2;
    }
  }
  cl_sync();
  __shared__ double s_bbv, s_rrv;  // the cluster sums, read by every thread (all scale their dots alike)
  if (threadIdx.x < 32) {
    double a = threadIdx.x < C ? ld_cl(&s_bb, threadIdx.x) : 0.0;
    double a2 = warm && threadIdx.x < C ? ld_cl(&s_rr0, threadIdx.x) : 0.0;
    for (int o = kClMaxCtas / 2; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (threadIdx.x == 0) {
      s_bbv = a;
      s_rrv = warm ? a2 : a;
    }
  }
  __syncthreads();
  const double bb = s_bbv, rr0 = s_rrv;
  long long eb = bb > 0.0 ? ((__double_as_longlong(bb) >> 52) & 0x7ff) - 1023 : 0;
  eb = eb < -126 ? -126 : (eb > 126 ? 126 : eb);
  const double dscale = __longlong_as_double((1023 - eb) << 52);
  const float fscale = (float)dscale;
  auto to_df = [&](const Acc& a) -> DF {
    if constexpr (kF64)
      return dot_df(a, dscale);
    else
      return dot_df(a, fscale);
  };
  const int fault = *d.fault;
  S rho, alpha, stop2, rr_last, rr_ref;
  sc_zero(rho);
  sc_zero(alpha);
  sc_zero(stop2);
  sc_zero(rr_last);
  sc_zero(rr_ref);
  int it_ref = 0;
  if (threadIdx.x == 0) {
    rho = sc_from(df_from(fault == 2 || (fault == 3 && sizeof(T) == 4) ? 0.0 : rr0 * dscale), S{});
    stop2 = sc_from(df_from(rtol * rtol * bb * dscale), S{});
    rr_ref = sc_from(df_from(rr0 * dscale), S{});
    sc_zero(s_sc[0]);
    sc_zero(s_sc[1]);
    sc_zero(s_sc[2]);
    s_ctl = 0;
  }
  __syncthreads();
  const bool busy = __any_sync(0xffffffffu, (int)threadIdx.x < nr) || (LINES && wib < nlb);
  int status = 1, it = 1;
  for (it = 1; !s_ctl; it++) {
    // ---- phase 1 ---------------------------------------------------------------------------
    const T beta = sc_t<T>(s_sc[0]), alp = sc_t<T>(s_sc[1]), omp = sc_t<T>(s_sc[2]);
    const T nom = -omp;
    const int po = (it & 1) ? 0 : 1, pn = 1 - po;
    const V* const yo = sy[po];
    V* const yn = sy[pn];
    const V* const vto = svt[po];
    V* const vtn = svt[pn];
    struct Raw1 {
      V tt, zf, vt, y;
    };
    // a neighbour in this CTA is read from its own shared memory (a distributed-shared-memory
    // request costs far more than a local load, and most neighbours are local)
    auto ld1 = [&](int j) {
      const unsigned o = owner(j);
      const int i = j - s_cb[o];
      if (o == me) return Raw1{stt[i], szf[i], vto[i], yo[i]};
      return Raw1{ld_cl(&stt[i], o), ld_cl(&szf[i], o), ld_cl(&vto[i], o), ld_cl(&yo[i], o)};
    };
    const unsigned f_tt = voff(stt), f_zf = voff(szf), f_vt = voff(vto), f_y = voff(yo);
    auto ld1a = [&](unsigned a) {
      Raw1 r;
      ld_cla(a + f_tt, r.tt);
      ld_cla(a + f_zf, r.zf);
      ld_cla(a + f_vt, r.vt);
      ld_cla(a + f_y, r.y);
      return r;
    };
    auto rt_of = [&](const Raw1& a) { return axpy(nom, a.tt, a.zf); };
    auto y_of = [&](const Raw1& a, const V& rtc) { return axpy(beta, axpy(nom, a.vt, a.y), rtc); };
    auto cb1 = [&](const Raw1& a) { return y_of(a, rt_of(a)); };
    Acc l_rv, l_rr;
    dot_zero(l_rv);
    dot_zero(l_rr);
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int i = threadIdx.x + q * kClThreads;
      if (i < nr) {
        const Raw1 own{stt[i], szf[i], vto[i], yo[i]};
        const V rtk = rt_of(own);
        const V ynk = y_of(own, rtk);
        const V vv = product(oref[q], ynk, ld1a, ld1, cb1);
        const V rk = axpy(nom, ot[q], os[q]);
        ox[q] = mk<T>(ox[q].x + alp * own.y.x + omp * oz[q].x, ox[q].y + alp * own.y.y + omp * oz[q].y);
        o_r[q] = rk;
        srt[i] = rtk;
        yn[i] = ynk;
        ov[q] = vv;
        if (LINES && oref[q].line)
          lbuf[i] = make_float2((float)vv.x, (float)vv.y);
        else
          vtn[i] = vv;
        dot_acc(l_rr, rk.x, rk.x);
        dot_acc(l_rr, rk.y, rk.y);
        dot_acc(l_rv, orh[q].x, vv.x);
        dot_acc(l_rv, orh[q].y, vv.y);
      }
    }
    lines([&](int k0, int len, const LineFac& f, const float2* buf, int seg) {
      V* const dst[1] = {vtn};
      if (seg)
        line_solve_seg<T, 1>(seg, k0, len, f, buf, R, dst);
      else
        line_solve<T, 1>(k0, len, f, buf, R, dst);
    });
    {
      const DF vals[2] = {to_df(l_rv), to_df(l_rr)};
      DF o[2];
      cl_sum<2>(vals, busy, s_df, s_part[0], C, o);
      if (threadIdx.x == 0) {
        const S rv = sc_from(o[0], S{});
        rr_last = sc_from(o[1], S{});
        if (sc_le(sc_mul(rr_last, sc_from(df_from(4.0), S{})), rr_ref)) {
          rr_ref = rr_last;
          it_ref = it;
        }
        if (sc_le(rr_last, stop2)) {
          s_ctl = 1;
          status = 0;
        } else if (it > maxit || (!kF64 && fault == 4 && it > 1)) {
          s_ctl = 1;
          status = 1;
        } else if (!kF64 && it - it_ref > kStagIters) {
          s_ctl = 1;
          status = 1;
        } else if (!sc_ok(rv) || !sc_ok(rho)) {
          s_ctl = 1;
          status = 2;
        } else {
          alpha = sc_div(rho, rv);
          s_sc[3] = alpha;
        }
      }
    }
    __syncthreads();
    if (s_ctl) break;
    // ---- phase 2 ---------------------------------------------------------------------------
    const T nal = -sc_t<T>(s_sc[3]);
    auto ld2 = [&](int j) {
      const unsigned o = owner(j);
      const int i = j - s_cb[o];
      if (o == me) return V2pair<V>{vtn[i], srt[i]};
      return V2pair<V>{ld_cl(&vtn[i], o), ld_cl(&srt[i], o)};
    };
    const unsigned f_vn = voff(vtn), f_rt = voff(srt);
    auto ld2a = [&](unsigned a) {
      V2pair<V> r;
      ld_cla(a + f_vn, r.a);
      ld_cla(a + f_rt, r.b);
      return r;
    };
    auto cb2 = [&](const V2pair<V>& a) { return axpy(nal, a.a, a.b); };
    Acc l_ts, l_tt, l_rs, l_rt;
    dot_zero(l_ts);
    dot_zero(l_tt);
    dot_zero(l_rs);
    dot_zero(l_rt);
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int i = threadIdx.x + q * kClThreads;
      if (i < nr) {
        const V zk = cb2(V2pair<V>{vtn[i], srt[i]});
        const V tk = product(oref[q], zk, ld2a, ld2, cb2);
        const V sk = axpy(nal, ov[q], o_r[q]);
        os[q] = sk;
        oz[q] = zk;
        ot[q] = tk;
        if (LINES && oref[q].line) {
          lbuf[i] = make_float2((float)sk.x, (float)sk.y);
          lbuf[R + i] = make_float2((float)tk.x, (float)tk.y);
        } else {
          szf[i] = sk;
          stt[i] = tk;
        }
        dot_acc(l_ts, tk.x, sk.x);
        dot_acc(l_ts, tk.y, sk.y);
        dot_acc(l_tt, tk.x, tk.x);
        dot_acc(l_tt, tk.y, tk.y);
        dot_acc(l_rs, orh[q].x, sk.x);
        dot_acc(l_rs, orh[q].y, sk.y);
        dot_acc(l_rt, orh[q].x, tk.x);
        dot_acc(l_rt, orh[q].y, tk.y);
      }
    }
    lines([&](int k0, int len, const LineFac& f, const float2* buf, int seg) {
      V* const dst[2] = {szf, stt};
      if (seg)
        line_solve_seg<T, 2>(seg, k0, len, f, buf, R, dst);
      else
        line_solve<T, 2>(k0, len, f, buf, R, dst);
    });
    {
      const DF vals[4] = {to_df(l_ts), to_df(l_tt), to_df(l_rs), to_df(l_rt)};
      DF o[4];
      cl_sum<4>(vals, busy, s_df, s_part[1], C, o);
      if (threadIdx.x == 0) {
        const S ts = sc_from(o[0], S{}), t2 = sc_from(o[1], S{}), rs = sc_from(o[2], S{}), rtv = sc_from(o[3], S{});
        if (!sc_finite(ts) || !sc_finite(t2) || !sc_finite(rs) || !sc_finite(rtv)) {
          s_ctl = 1;
          status = 2;
        } else {
          S omega, beta;
          sc_zero(omega);
          sc_zero(beta);
          if (sc_pos(t2)) omega = sc_div(ts, t2);
          const S rho_new = sc_fnma(omega, rtv, rs);
          if (sc_nonzero(omega)) beta = sc_mul(sc_div(rho_new, rho), sc_div(alpha, omega));
          s_sc[0] = beta;
          s_sc[1] = alpha;
          s_sc[2] = omega;
          rho = rho_new;
        }
      }
    }
    __syncthreads();
    if (s_ctl) break;
  }
  // x_{it-1} to the solution vector; every CTA waits until no CTA reads its shared memory
  V* const xg = (V*)d.kx;
#pragma unroll
  for (int q = 0; q < RPT; q++) {
    const int i = threadIdx.x + q * kClThreads;
    if (i < nr) xg[c0 + i] = ox[q];
  }
  if (me == 0 && threadIdx.x == 0) {
    d.ctr->krylov_iters = it - 1;
    d.ctr->krylov_status = status;
    d.ctr->krylov_solver = 1;
    d.ctr->krylov_relres = bb > 0.0 ? sqrt(sc_double(rr_last) / (bb * dscale)) : 0.0;
  }
  cl_sync();
}

template <typename T, bool L, int BATCH = 4>
int max_blocks(int sms) {
  int nb = 0;
  cudaFuncSetAttribute(k_bicgstab<T, L, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKrySmem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab<T, L, BATCH>, kKryBlk, kKrySmem);
  if (nb > 2) nb = 2;
  if (nb < 1) nb = 1;
  return nb * sms;
}

}  // namespace

int krylov_grid(int fp32, int sms) {
  int a = fp32 ? max_blocks<float, true>(sms) : max_blocks<double, true>(sms);
  int b = fp32 ? max_blocks<float, false>(sms) : max_blocks<double, false>(sms);
  if (fp32) {  // the wide-batch variants (Dev::wide_rows)
    const int a6 = max_blocks<float, true, 6>(sms), b6 = max_blocks<float, false, 6>(sms);
    a = a6 < a ? a6 : a;
    b = b6 < b ? b6 : b;
  }
  return a < b ? a : b;
}

namespace {
template <typename T, bool L>
int cluster_fits(int ctas) {
  auto fn = k_bicgstab_cl<T, L>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem) != cudaSuccess) return 0;
  if (ctas > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = kClSmem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T, bool L>
ClusterShape cluster_shape_t(int max_ctas) {
  for (int c = kClMaxCtas; c >= 2; c >>= 1) {
    if (c > max_ctas) continue;
    if (cluster_fits<T, L>(c) >= 1) {
      const int per = ClShape<T>::kRows - (L ? kLineBlockRows : 0);
      return ClusterShape{c, c * per};
    }
  }
  cudaGetLastError();
  return ClusterShape{0, -1};
}
}  // namespace

ClusterShape krylov_cluster_shape(int fp32, int lines, int max_ctas) {
  if (max_ctas <= 0) return ClusterShape{0, -1};
  if (fp32) return lines ? cluster_shape_t<float, true>(max_ctas) : cluster_shape_t<float, false>(max_ctas);
  return lines ? cluster_shape_t<double, true>(max_ctas) : cluster_shape_t<double, false>(max_ctas);
}

// The grid solver's blocks fill every SM, so two of its solves must never be resident at once:
// launches from different streams (models served concurrently) are chained through one event per
// device, each waiting for the previous one to finish.  Cluster solves occupy C SMs and run
// concurrently with anything.
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_coop_mu;
cudaEvent_t g_coop_ev[kMaxDevices] = {};
}  // namespace

// One solver only (the host has read n_A): which = 1 the cluster solver (n_A <= cl.cap), 2 the grid
// solver.  Same kernels and arguments as launch_bicgstab's, so the results are the same bits.
cudaError_t launch_bicgstab_which(const Dev& d, int fp32, int lines, double rtol, int maxit, int grid, ClusterShape cl,
                                  int which, LaunchCfg c) {
  if (which == 1 && cl.ctas > 0) {
    ClusterShape only = cl;
    cudaError_t e = cudaMemsetAsync(&d.ctr->bar_count, 0, 3 * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    Dev dd = d;
    int cap = cl.cap;
    void* cfn = fp32 ? (lines ? (void*)k_bicgstab_cl<float, true> : (void*)k_bicgstab_cl<float, false>)
                     : (lines ? (void*)k_bicgstab_cl<double, true> : (void*)k_bicgstab_cl<double, false>);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = only.ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(only.ctas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = kClSmem;
    cfg.stream = c.stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* cargs[] = {&dd, &rtol, &maxit, &cap};
    count_launches(1);
    return cudaLaunchKernelExC(&cfg, cfn, cargs);
  }
  return launch_bicgstab(d, fp32, lines, rtol, maxit, grid, ClusterShape{0, -1}, c);
}

cudaError_t launch_bicgstab(const Dev& d, int fp32, int lines, double rtol, int maxit, int grid, ClusterShape cl,
                            LaunchCfg c) {
  // barrier counter and timeout flag start from zero in every launch
  cudaError_t e = cudaMemsetAsync(&d.ctr->bar_count, 0, 3 * sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  Dev dd = d;
  int cap = cl.ctas > 0 ? cl.cap : -1;
  if (cl.ctas > 0) {
    void* cfn = fp32 ? (lines ? (void*)k_bicgstab_cl<float, true> : (void*)k_bicgstab_cl<float, false>)
                     : (lines ? (void*)k_bicgstab_cl<double, true> : (void*)k_bicgstab_cl<double, false>);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl.ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl.ctas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = kClSmem;
    cfg.stream = c.stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* cargs[] = {&dd, &rtol, &maxit, &cap};
    count_launches(1);
    e = cudaLaunchKernelExC(&cfg, cfn, cargs);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {&dd, &rtol, &maxit, &cap};
  count_launches(1);
  void* fn = fp32 ? (d.wide_rows ? (lines ? (void*)k_bicgstab<float, true, 6> : (void*)k_bicgstab<float, false, 6>)
                                  : (lines ? (void*)k_bicgstab<float, true, 4> : (void*)k_bicgstab<float, false, 4>))
                  : (lines ? (void*)k_bicgstab<double, true, 4> : (void*)k_bicgstab<double, false, 4>);
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(c.stream, &cap_st);
  if (e != cudaSuccess) return e;
  if (cap_st != cudaStreamCaptureStatusNone)  // captured into a model's graph: ordered by its own stream
    return cudaLaunchCooperativeKernel(fn, grid, kKryBlk, args, kKrySmem, c.stream);
  std::lock_guard<std::mutex> lk(g_coop_mu);
  if (!g_coop_ev[dev]) {
    e = cudaEventCreateWithFlags(&g_coop_ev[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      g_coop_ev[dev] = nullptr;
      return e;
    }
  } else {
    e = cudaStreamWaitEvent(c.stream, g_coop_ev[dev], 0);
    if (e != cudaSuccess) return e;
  }
  e = cudaLaunchCooperativeKernel(fn, grid, kKryBlk, args, kKrySmem, c.stream);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(g_coop_ev[dev], c.stream);
}

}  // namespace lns
