// Host build of the black-oil physics header (the code the black-oil kernels run), so that the
// CPU tests can compare it with the black-oil oracle.  Test infrastructure: the library never
// links it.
#include <cstring>

#include "../../paper_2008_01539_gb300/csrc/blk3.cuh"
#include "../../paper_2008_01539_gb300/csrc/bo_physics.cuh"

using namespace lns::bo;

extern "C" {

// Residual F (n, 3), diagonal blocks Jd (n, 3, 3), off-diagonal blocks Jo (n_adj, 3, 3) and CNV (n)
// of every cell, cell by cell and face by face as an assembly thread does.
void bo_host_assemble(const Fluid* f, int n, const int* row_ptr, const int* nbr, const double* trans,
                      const double* pv_ref, const double* depth, int n_wells, const int* well_cell,
                      const double* well_wi, const double* well_bhp, const double* p, const double* sw,
                      const double* x, const unsigned char* sat, const double* p_old, const double* sw_old,
                      const double* x_old, const unsigned char* sat_old, double dt, double* F, double* Jd,
                      double* Jo, double* cnv_out) {
  for (int i = 0; i < n; i++) {
    const Props qi = cell_props(*f, pv_ref[i], p[i], sw[i], x[i], sat[i]);
    const Props qo = cell_props(*f, pv_ref[i], p_old[i], sw_old[i], x_old[i], sat_old[i]);
    double R[3] = {0.0, 0.0, 0.0}, D[9];
    std::memset(D, 0, sizeof(D));
    const double m_old[3] = {qo.mass[0].v, qo.mass[1].v, qo.mass[2].v};
    accumulation(qi, m_old, dt, R, D);
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      const int j = nbr[e];
      const Props qj = cell_props(*f, pv_ref[j], p[j], sw[j], x[j], sat[j]);
      double* O = Jo + 9 * (long)e;
      std::memset(O, 0, 9 * sizeof(double));
      face_flux(*f, qi, qj, p[i], p[j], trans[e], depth[i] - depth[j], i < j, R, D, O);
    }
    for (int w = 0; w < n_wells; w++)
      if (well_cell[w] == i) producer(qi, p[i], well_wi[w], well_bhp[w], R, D);
    for (int c = 0; c < 3; c++) F[3 * (long)i + c] = R[c];
    std::memcpy(Jd + 9 * (long)i, D, sizeof(D));
    cnv_out[i] = cnv(qi, R, dt);
  }
}

// The update with the saturation chop and the switch, cell by cell; returns the number of switches.
int bo_host_update(const Fluid* f, double chop, int n, const double* du, double* p, double* sw, double* sg,
                   double* rs, unsigned char* sat, unsigned char* switched) {
  int k = 0;
  for (int i = 0; i < n; i++) {
    switched[i] = (unsigned char)update_cell(*f, chop, du[3 * (long)i], du[3 * (long)i + 1], du[3 * (long)i + 2],
                                             &p[i], &sw[i], &sg[i], &rs[i], &sat[i]);
    k += switched[i];
  }
  return k;
}

// 3x3 block inverse; returns 0 on a singular block
int b3_host_inv(const double* a, double* r) { return lns::b3::inv(a, r) ? 1 : 0; }

// factor a line block (L, U: len x 9) and solve M z = r, in FP64 (fp32 = 0) or FP32 (inputs
// rounded to float, as the FP32 preconditioner stores them); returns 0 on a singular pivot
int b3_host_line(int len, const double* L, const double* U, const double* r, double* z, int fp32) {
  if (len <= 0 || len > 256) return 0;
  if (!fp32) {
    static double Di[9 * 256], A[9 * 256], G[9 * 256];
    if (!lns::b3::line_factor(len, L, U, Di, A, G)) return 0;
    lns::b3::line_solve(len, Di, A, G, r, z);
    return 1;
  }
  static float Lf[9 * 256], Uf[9 * 256], rf[3 * 256], zf[3 * 256], Di[9 * 256], A[9 * 256], G[9 * 256];
  for (int k = 0; k < 9 * len; k++) {
    Lf[k] = (float)L[k];
    Uf[k] = (float)U[k];
  }
  for (int k = 0; k < 3 * len; k++) rf[k] = (float)r[k];
  if (!lns::b3::line_factor(len, Lf, Uf, Di, A, G)) return 0;
  lns::b3::line_solve(len, Di, A, G, rf, zf);
  for (int k = 0; k < 3 * len; k++) z[k] = zf[k];
  return 1;
}
}
