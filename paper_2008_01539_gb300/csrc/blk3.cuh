// 3x3 block arithmetic of the black-oil solver (three unknowns per cell): the block inverse, and
// the fracture-line block of the preconditioner, factored and solved by the block Thomas
// algorithm.  Written once for the device kernels and for their check on the host.
//
// A fracture-line block of the row-scaled system (each row block multiplied by the inverse of its
// diagonal block, so the diagonal blocks are I) is block tridiagonal with L_t (row t -> t-1) and
// U_t (row t -> t+1).  Its factorization:
//   D'_0 = I,  D'_t = I - L_t G_{t-1},  G_t = D'_t^{-1} U_t,  A_t = -D'_t^{-1} L_t
// so that M^{-1} r is  w_t = D'_t^{-1} r_t + A_t w_{t-1},  z_t = w_t - G_t z_{t+1}.
// Blocks are row-major, 9 values.
#pragma once

#ifdef __CUDACC__
#define B3_HD __host__ __device__ __forceinline__
#else
#define B3_HD inline
#endif

namespace lns {
namespace b3 {

// c = a b
template <typename F>
B3_HD void mul(const F* a, const F* b, F* c) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

// y = a x
template <typename F>
B3_HD void mulv(const F* a, const F* x, F* y) {
  for (int i = 0; i < 3; i++) y[i] = a[3 * i] * x[0] + a[3 * i + 1] * x[1] + a[3 * i + 2] * x[2];
}

// r = a^{-1} by cofactors (the adjugate over the determinant); false when the determinant is 0
// or not finite
template <typename F>
B3_HD bool inv(const F* a, F* r) {
  const F c00 = a[4] * a[8] - a[5] * a[7];
  const F c01 = a[5] * a[6] - a[3] * a[8];
  const F c02 = a[3] * a[7] - a[4] * a[6];
  const F det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(det != F(0)) || !(det - det == F(0))) return false;
  const F id = F(1) / det;
  r[0] = c00 * id;
  r[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  r[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  r[3] = c01 * id;
  r[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  r[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  r[6] = c02 * id;
  r[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  r[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}

// Factors of a line block of len rows (L_0 and U_{len-1} are not read).  Returns false on a
// singular D'_t.
template <typename F>
B3_HD bool line_factor(int len, const F* L, const F* U, F* Dinv, F* A, F* G) {
  F Gp[9];
  for (int t = 0; t < len; t++) {
    F Dp[9];
    if (t == 0) {
      for (int k = 0; k < 9; k++) Dp[k] = (k % 4 == 0) ? F(1) : F(0);
    } else {
      F LG[9];
      mul(L + 9 * t, Gp, LG);
      for (int k = 0; k < 9; k++) Dp[k] = ((k % 4 == 0) ? F(1) : F(0)) - LG[k];
    }
    F* Di = Dinv + 9 * t;
    if (!inv(Dp, Di)) return false;
    F* At = A + 9 * t;
    if (t == 0) {
      for (int k = 0; k < 9; k++) At[k] = F(0);
    } else {
      mul(Di, L + 9 * t, At);
      for (int k = 0; k < 9; k++) At[k] = -At[k];
    }
    F* Gt = G + 9 * t;
    if (t + 1 < len) {
      mul(Di, U + 9 * t, Gt);
    } else {
      for (int k = 0; k < 9; k++) Gt[k] = F(0);
    }
    for (int k = 0; k < 9; k++) Gp[k] = Gt[k];
  }
  return true;
}

// z = M^{-1} r on one line block (sequential recurrences; the kernels run them as warp scans of
// the same affine maps)
template <typename F>
B3_HD void line_solve(int len, const F* Dinv, const F* A, const F* G, const F* r, F* z) {
  F w[3] = {F(0), F(0), F(0)};
  for (int t = 0; t < len; t++) {
    F a[3], b[3];
    mulv(Dinv + 9 * t, r + 3 * t, a);
    mulv(A + 9 * t, w, b);
    for (int i = 0; i < 3; i++) w[i] = a[i] + b[i];
    for (int i = 0; i < 3; i++) z[3 * t + i] = w[i];
  }
  for (int t = len - 2; t >= 0; t--) {
    F g[3];
    mulv(G + 9 * t, z + 3 * (t + 1), g);
    for (int i = 0; i < 3; i++) z[3 * t + i] -= g[i];
  }
}

}  // namespace b3
}  // namespace lns
