// k_blackoil.cu -- the three-phase black-oil model's residual and Jacobian assembly and its update
// with the primary-variable switch, on caller-owned device arrays (lns_bo_assemble, lns_bo_update).
//
// The arithmetic is bo_physics.cuh's (Appendix A with gas dissolving in oil; Section 3.1's
// variable substitution in black-oil form).  The assembly runs one thread per cell: the cell's
// properties with their derivatives, its accumulation, one face flux per CSR entry (the
// neighbour's properties evaluated by the thread) and the producers in the cell, writing the
// cell's residual row, its diagonal 3x3 block and the off-diagonal block of every CSR entry of the
// row.  FP64 throughout, bound by the FP64 pipe as the oil-water assembly is.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "bo_physics.cuh"
#include "lns_internal.cuh"

namespace {

constexpr int kBoBlk = 128;

static_assert(sizeof(lns_bo_fluid) == sizeof(lns::bo::Fluid), "lns_bo_fluid and bo::Fluid must share a layout");

lns::bo::Fluid to_fluid(const lns_bo_fluid& f) {
  lns::bo::Fluid g;
  g.p_ref = f.p_ref;
  g.c_r = f.c_r;
  g.b_w_ref = f.b_w_ref;
  g.c_w = f.c_w;
  g.rho_w_sc = f.rho_w_sc;
  g.mu_w = f.mu_w;
  g.b_o_ref = f.b_o_ref;
  g.c_o = f.c_o;
  g.kappa = f.kappa;
  g.rho_o_sc = f.rho_o_sc;
  g.mu_o = f.mu_o;
  g.b_g_per_pa = f.b_g_per_pa;
  g.rho_g_sc = f.rho_g_sc;
  g.mu_g = f.mu_g;
  g.rs_max = f.rs_max;
  g.p_bubble = f.p_bubble;
  g.swc = f.swc;
  g.sor = f.sor;
  g.gravity = f.gravity;
  g.n_w = f.n_w;
  g.n_o = f.n_o;
  g.n_g = f.n_g;
  return g;
}

lns_status bo_fail(lns_status s, const std::string& m) {
  lns::set_last_error(m.c_str());
  return s;
}

struct BoState {
  const double *p, *sw, *sg, *rs;
  const uint8_t* sat;
};

struct BoGraph {
  int n, n_wells;
  const int *row_ptr, *nbr, *well_cell;
  const double *trans, *pv_ref, *depth, *well_wi, *well_bhp;
};

__device__ __forceinline__ lns::bo::Props props_of(const lns::bo::Fluid& f, const BoGraph& g, const BoState& s,
                                                   int i) {
  const int sat = s.sat[i];
  return lns::bo::cell_props(f, g.pv_ref[i], s.p[i], s.sw[i], sat ? s.sg[i] : s.rs[i], sat);
}

__global__ void __launch_bounds__(kBoBlk) k_bo_assemble(lns::bo::Fluid f, BoGraph g, BoState s, BoState o, double dt,
                                                       double* F, double* Jd, double* Jo, double* cnv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const lns::bo::Props qi = props_of(f, g, s, i);
  const lns::bo::Props qo = props_of(f, g, o, i);
  double R[3] = {0.0, 0.0, 0.0}, D[9];
  for (int k = 0; k < 9; k++) D[k] = 0.0;
  const double m_old[3] = {qo.mass[0].v, qo.mass[1].v, qo.mass[2].v};
  lns::bo::accumulation(qi, m_old, dt, R, D);
  const double pi = s.p[i], zi = g.depth[i];
  for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; e++) {
    const int j = g.nbr[e];
    const lns::bo::Props qj = props_of(f, g, s, j);
    double O[9];
    for (int k = 0; k < 9; k++) O[k] = 0.0;
    lns::bo::face_flux(f, qi, qj, pi, s.p[j], g.trans[e], zi - g.depth[j], i < j, R, D, O);
    if (Jo)
      for (int k = 0; k < 9; k++) Jo[9 * (size_t)e + k] = O[k];
  }
  for (int w = 0; w < g.n_wells; w++)
    if (g.well_cell[w] == i) lns::bo::producer(qi, pi, g.well_wi[w], g.well_bhp[w], R, D);
  if (F)
    for (int c = 0; c < 3; c++) F[3 * (size_t)i + c] = R[c];
  if (Jd)
    for (int k = 0; k < 9; k++) Jd[9 * (size_t)i + k] = D[k];
  if (cnv) cnv[i] = lns::bo::cnv(qi, R, dt);
}

__global__ void __launch_bounds__(kBoBlk) k_bo_update(lns::bo::Fluid f, int n, double chop, const double* du,
                                                     const uint32_t* va_bits, double* p, double* sw, double* sg,
                                                     double* rs, uint8_t* sat, uint8_t* switched) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (va_bits && !((va_bits[i >> 5] >> (i & 31)) & 1u)) {
    if (switched) switched[i] = 0;
    return;
  }
  double pi = p[i], swi = sw[i], sgi = sg[i], rsi = rs[i];
  unsigned char si = sat[i];
  const int k = lns::bo::update_cell(f, chop, du[3 * (size_t)i], du[3 * (size_t)i + 1], du[3 * (size_t)i + 2], &pi,
                                     &swi, &sgi, &rsi, &si);
  p[i] = pi;
  sw[i] = swi;
  sg[i] = sgi;
  rs[i] = rsi;
  sat[i] = si;
  if (switched) switched[i] = (uint8_t)k;
}

lns_status finish(cudaStream_t stream, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return bo_fail(LNS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return LNS_OK;
}

}  // namespace

extern "C" lns_status lns_bo_assemble(const lns_bo_fluid* fluid, int32_t n_cells, const int32_t* row_ptr,
                                      const int32_t* nbr, const double* trans, const double* pv_ref,
                                      const double* depth, int32_t n_wells, const int32_t* well_cell,
                                      const double* well_wi, const double* well_bhp, const double* p,
                                      const double* sw, const double* sg, const double* rs, const uint8_t* sat,
                                      const double* p_old, const double* sw_old, const double* sg_old,
                                      const double* rs_old, const uint8_t* sat_old, double dt, double* F,
                                      double* Jd, double* Jo, double* cnv, void* cuda_stream) {
  if (!fluid) return bo_fail(LNS_EINVAL, "fluid must be non-NULL");
  if (n_cells < 0 || n_wells < 0) return bo_fail(LNS_EINVAL, "n_cells and n_wells must be >= 0");
  if (!(dt > 0.0)) return bo_fail(LNS_EINVAL, "dt must be > 0");
  if (n_cells == 0) return LNS_OK;
  if (!row_ptr || !nbr || !trans || !pv_ref || !depth || !p || !sw || !sg || !rs || !sat || !p_old || !sw_old ||
      !sg_old || !rs_old || !sat_old)
    return bo_fail(LNS_EINVAL, "the graph and both states must be device pointers (non-NULL)");
  if (n_wells > 0 && (!well_cell || !well_wi || !well_bhp))
    return bo_fail(LNS_EINVAL, "well_cell, well_wi and well_bhp must be non-NULL when n_wells > 0");
  const lns::bo::Fluid f = to_fluid(*fluid);
  if (!(f.p_bubble > 0.0) || !(1.0 - f.swc - f.sor > 0.0) || f.n_w < 1 || f.n_o < 1 || f.n_g < 1)
    return bo_fail(LNS_EINVAL, "fluid: p_bubble > 0, swc + sor < 1 and Corey exponents >= 1 are required");
  BoGraph g{n_cells, n_wells, row_ptr, nbr, well_cell, trans, pv_ref, depth, well_wi, well_bhp};
  BoState s{p, sw, sg, rs, sat}, o{p_old, sw_old, sg_old, rs_old, sat_old};
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  k_bo_assemble<<<(n_cells + kBoBlk - 1) / kBoBlk, kBoBlk, 0, stream>>>(f, g, s, o, dt, F, Jd, Jo, cnv);
  lns::count_launches(1);
  return finish(stream, "lns_bo_assemble");
}

extern "C" lns_status lns_bo_update(const lns_bo_fluid* fluid, int32_t n_cells, double sat_chop, const double* du,
                                    const uint32_t* va_bits, double* p, double* sw, double* sg, double* rs,
                                    uint8_t* sat, uint8_t* switched, void* cuda_stream) {
  if (!fluid) return bo_fail(LNS_EINVAL, "fluid must be non-NULL");
  if (n_cells < 0) return bo_fail(LNS_EINVAL, "n_cells must be >= 0");
  if (n_cells == 0) return LNS_OK;
  if (!du || !p || !sw || !sg || !rs || !sat)
    return bo_fail(LNS_EINVAL, "du, p, sw, sg, rs and sat must be device pointers (non-NULL)");
  const lns::bo::Fluid f = to_fluid(*fluid);
  if (!(f.p_bubble > 0.0)) return bo_fail(LNS_EINVAL, "fluid: p_bubble must be > 0");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  k_bo_update<<<(n_cells + kBoBlk - 1) / kBoBlk, kBoBlk, 0, stream>>>(f, n_cells, sat_chop, du, va_bits, p, sw, sg,
                                                                     rs, sat, switched);
  lns::count_launches(1);
  return finish(stream, "lns_bo_update");
}
