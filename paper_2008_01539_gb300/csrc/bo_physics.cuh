// Three-phase black-oil cell properties, face fluxes, producer terms and the primary-variable
// switch, written once for the black-oil assembly and update kernels (device) and for their check
// on the host.
//
// Model (Appendix A's backward-Euler TPFA with phase-potential upwinding, three phases, gas
// dissolving in oil; surface volumes):
//   R_c,i = [M_c(u_i) - M_c(u_i^n)] / dt + sum_j F_c,ij + q_c,i          c = oil, water, gas
//   M_o = PV b_o So,  M_w = PV b_w Sw,  M_g = PV (b_g Sg + Rs b_o So),  So = 1 - Sw - Sg
//   F_l,ij = T_ij (lambda_l b_l)_up dPhi_l,ij (l = o, w, g); F_g,ij += T_ij (Rs lambda_o b_o)_up(o) dPhi_o,ij
//   dPhi_l,ij = (p_i - p_j) - g (rho_l,i + rho_l,j) / 2 (z_i - z_j); up = i if dPhi > 0, j if < 0,
//   the lower cell index on a tie; producer q_c = WI (lambda_c b_c) max(p - BHP, 0), q_g += Rs q_o.
//   PV = PV_ref (1 + c_r (p - p_ref)), b_w = b_w_ref (1 + c_w (p - p_ref)),
//   b_o = b_o_ref (1 + c_o (p - p_ref)) / (1 + kappa Rs), b_g = b_g_per_pa p,
//   rho_w = rho_w_sc b_w, rho_o = b_o (rho_o_sc + Rs rho_g_sc), rho_g = rho_g_sc b_g,
//   Rs_sat(p) = rs_max p / p_bubble; Corey kr_w = Sw*^n_w, kr_o = So*^n_o, kr_g = Sg*^n_g with
//   Sw* = (Sw - swc) / span, So* = (So - sor) / span, Sg* = Sg / span clamped to [0, 1],
//   span = 1 - swc - sor (zero slope outside).
// Unknowns per cell (p, Sw, X): X = Sg where free gas is present (sat = 1, Rs = Rs_sat(p)), X = Rs
// where it is not (sat = 0, Sg = 0).  Section 3.1's variable substitution, black-oil form: after an
// update, a cell whose Sg < 0 loses its gas phase (Sg = 0, Rs = Rs_sat(p)); a cell without free gas
// whose Rs > Rs_sat(p) splits (Sg = 0, Rs = Rs_sat(p)).
// Derivatives are written out by hand (chain rule), tracking which unknowns each quantity
// depends on; equations are ordered (oil, water, gas), unknowns (p, Sw, X).
#pragma once

#ifdef __CUDACC__
#define BO_HD __host__ __device__ __forceinline__
#else
#define BO_HD inline
#endif

namespace lns {
namespace bo {

struct Fluid {
  double p_ref, c_r;
  double b_w_ref, c_w, rho_w_sc, mu_w;
  double b_o_ref, c_o, kappa, rho_o_sc, mu_o;
  double b_g_per_pa, rho_g_sc, mu_g;
  double rs_max, p_bubble;
  double swc, sor, gravity;
  int n_w, n_o, n_g;
};

// a value and its derivatives in (p, Sw, X)
struct D3 {
  double v, dp, ds, dx;
};

enum { kOil = 0, kWat = 1, kGas = 2 };

struct Props {
  D3 pv, b[3], rho[3], mob[3], rsmob, mass[3], rs;
};

BO_HD double rs_sat(const Fluid& f, double p) { return f.rs_max * p / f.p_bubble; }

// x^n for a small integer n >= 1, and n x^(n-1)
BO_HD void ipow_d(double x, int n, double* v, double* d) {
  double r = 1.0;
  for (int k = 1; k < n; k++) r *= x;
  *d = (double)n * r;
  *v = r * x;
}

// Corey relative permeability of a normalised saturation s* = (s - s0) / span, clamped to [0, 1]
// (slope 0 outside); returns kr and dkr/ds
BO_HD void corey(double s, double s0, double span, int n, double* kr, double* dkr) {
  double e = (s - s0) / span;
  if (e <= 0.0) {
    *kr = 0.0;
    *dkr = 0.0;
  } else if (e >= 1.0) {
    *kr = 1.0;
    *dkr = 0.0;
  } else {
    double d;
    ipow_d(e, n, kr, &d);
    *dkr = d / span;
  }
}

BO_HD Props cell_props(const Fluid& f, double pv_ref, double p, double sw, double x, int sat) {
  Props q;
  const double dpr = p - f.p_ref;
  const double sg = sat ? x : 0.0;
  const double rs = sat ? rs_sat(f, p) : x;
  // dRs/dp and dRs/dX, dSg/dX
  const double rs_p = sat ? f.rs_max / f.p_bubble : 0.0, rs_x = sat ? 0.0 : 1.0, sg_x = sat ? 1.0 : 0.0;
  const double so = 1.0 - sw - sg;
  q.rs = {rs, rs_p, 0.0, rs_x};
  q.pv = {pv_ref * (1.0 + f.c_r * dpr), pv_ref * f.c_r, 0.0, 0.0};
  // water, gas: functions of p
  q.b[kWat] = {f.b_w_ref * (1.0 + f.c_w * dpr), f.b_w_ref * f.c_w, 0.0, 0.0};
  q.b[kGas] = {f.b_g_per_pa * p, f.b_g_per_pa, 0.0, 0.0};
  // oil: b_o = a(p) / (1 + kappa Rs)
  const double a = f.b_o_ref * (1.0 + f.c_o * dpr), a_p = f.b_o_ref * f.c_o;
  const double den = 1.0 + f.kappa * rs;
  const double bo = a / den;
  const double bo_rs = -bo * f.kappa / den;  // d b_o / d Rs at fixed p
  q.b[kOil] = {bo, a_p / den + bo_rs * rs_p, 0.0, bo_rs * rs_x};
  q.rho[kWat] = {f.rho_w_sc * q.b[kWat].v, f.rho_w_sc * q.b[kWat].dp, 0.0, 0.0};
  q.rho[kGas] = {f.rho_g_sc * q.b[kGas].v, f.rho_g_sc * q.b[kGas].dp, 0.0, 0.0};
  {
    const double m = f.rho_o_sc + f.rho_g_sc * rs;
    q.rho[kOil] = {bo * m, q.b[kOil].dp * m + bo * f.rho_g_sc * rs_p, 0.0, q.b[kOil].dx * m + bo * f.rho_g_sc * rs_x};
  }
  // relative permeabilities
  const double span = 1.0 - f.swc - f.sor;
  double krw, krw_s, kro, kro_so, krg, krg_sg;
  corey(sw, f.swc, span, f.n_w, &krw, &krw_s);
  corey(so, f.sor, span, f.n_o, &kro, &kro_so);
  corey(sg, 0.0, span, f.n_g, &krg, &krg_sg);
  // So = 1 - Sw - Sg: dSo/dSw = -1, dSo/dX = -dSg/dX
  const double kro_s = -kro_so, kro_x = -kro_so * sg_x, krg_x = krg_sg * sg_x;
  q.mob[kWat] = {krw / f.mu_w * q.b[kWat].v, krw / f.mu_w * q.b[kWat].dp, krw_s / f.mu_w * q.b[kWat].v, 0.0};
  q.mob[kGas] = {krg / f.mu_g * q.b[kGas].v, krg / f.mu_g * q.b[kGas].dp, 0.0, krg_x / f.mu_g * q.b[kGas].v};
  q.mob[kOil] = {kro / f.mu_o * bo, kro / f.mu_o * q.b[kOil].dp, kro_s / f.mu_o * bo,
                 (kro_x * bo + kro * q.b[kOil].dx) / f.mu_o};
  const D3& mo = q.mob[kOil];
  q.rsmob = {rs * mo.v, rs_p * mo.v + rs * mo.dp, rs * mo.ds, rs_x * mo.v + rs * mo.dx};
  // masses
  const D3 &pv = q.pv, &bw = q.b[kWat], &bg = q.b[kGas], &bob = q.b[kOil];
  q.mass[kWat] = {pv.v * bw.v * sw, (pv.dp * bw.v + pv.v * bw.dp) * sw, pv.v * bw.v, 0.0};
  const double pbo = pv.v * bob.v;  // PV b_o
  const double pbo_p = pv.dp * bob.v + pv.v * bob.dp, pbo_x = pv.v * bob.dx;
  q.mass[kOil] = {pbo * so, pbo_p * so, -pbo, pbo_x * so - pbo * sg_x};
  // M_g = PV b_g Sg + Rs M_o
  const D3& mo_ = q.mass[kOil];
  const double fg = pv.v * bg.v;
  q.mass[kGas] = {fg * sg + rs * mo_.v, (pv.dp * bg.v + pv.v * bg.dp) * sg + rs_p * mo_.v + rs * mo_.dp,
                  rs * mo_.ds, fg * sg_x + rs_x * mo_.v + rs * mo_.dx};
  return q;
}

BO_HD void d3_row(double* J, const D3& a, double s) {  // J[0..2] += s * (d/dp, d/dSw, d/dX) of a
  J[0] += s * a.dp;
  J[1] += s * a.ds;
  J[2] += s * a.dx;
}

// Accumulation of cell i: R += (M(u) - M_old) / dt, Jd += dM/du / dt.  M_old: the old masses.
BO_HD void accumulation(const Props& q, const double* M_old, double dt, double* R, double* Jd /* 3x3 */) {
  for (int c = 0; c < 3; c++) {
    R[c] += (q.mass[c].v - M_old[c]) / dt;
    Jd[3 * c + 0] += q.mass[c].dp / dt;
    Jd[3 * c + 1] += q.mass[c].ds / dt;
    Jd[3 * c + 2] += q.mass[c].dx / dt;
  }
}

// Outflow from i to its neighbour j over a face of transmissibility T, z_i - z_j = dz; i_first:
// i < j (the tie rule).  Adds to R (3, row i), Ji (3x3, d/du_i) and Jj (3x3, d/du_j).
BO_HD void face_flux(const Fluid& f, const Props& qi, const Props& qj, double p_i, double p_j, double T, double dz,
                     bool i_first, double* R, double* Ji, double* Jj) {
  const double gdz = f.gravity * dz;
  bool up_oil = true;
  double dphi_oil = 0.0;
  for (int l = 0; l < 3; l++) {
    const D3 &ri = qi.rho[l], &rj = qj.rho[l];
    const double dphi = (p_i - p_j) - gdz * (0.5 * (ri.v + rj.v));
    const bool up = dphi > 0.0 || (dphi == 0.0 && i_first);
    const D3& mu = up ? qi.mob[l] : qj.mob[l];
    const double tm = T * mu.v;
    // d dPhi / du_i = (1, 0, 0) - gdz / 2 drho_i; d dPhi / du_j = (-1, 0, 0) - gdz / 2 drho_j
    double* Jr_i = Ji + 3 * l;
    double* Jr_j = Jj + 3 * l;
    R[l] += tm * dphi;
    Jr_i[0] += tm;
    Jr_j[0] -= tm;
    d3_row(Jr_i, ri, -0.5 * gdz * tm);
    d3_row(Jr_j, rj, -0.5 * gdz * tm);
    d3_row(up ? Jr_i : Jr_j, mu, T * dphi);
    if (l == kOil) {
      up_oil = up;
      dphi_oil = dphi;
    }
  }
  // dissolved gas with the oil: T (Rs mob_o)_up(o) dPhi_o
  const D3& rm = up_oil ? qi.rsmob : qj.rsmob;
  const double tm = T * rm.v;
  double* Jg_i = Ji + 3 * kGas;
  double* Jg_j = Jj + 3 * kGas;
  R[kGas] += tm * dphi_oil;
  Jg_i[0] += tm;
  Jg_j[0] -= tm;
  d3_row(Jg_i, qi.rho[kOil], -0.5 * gdz * tm);
  d3_row(Jg_j, qj.rho[kOil], -0.5 * gdz * tm);
  d3_row(up_oil ? Jg_i : Jg_j, rm, T * dphi_oil);
}

// Producer at fixed BHP in cell i: q_c = WI (lambda_c b_c) max(p - BHP, 0), q_g += Rs q_o.
BO_HD void producer(const Props& q, double p, double wi, double bhp, double* R, double* Jd) {
  const double dpw = p - bhp;
  if (dpw <= 0.0) return;
  for (int l = 0; l < 3; l++) {
    R[l] += wi * q.mob[l].v * dpw;
    Jd[3 * l + 0] += wi * (q.mob[l].dp * dpw + q.mob[l].v);
    Jd[3 * l + 1] += wi * q.mob[l].ds * dpw;
    Jd[3 * l + 2] += wi * q.mob[l].dx * dpw;
  }
  R[kGas] += wi * q.rsmob.v * dpw;
  Jd[3 * kGas + 0] += wi * (q.rsmob.dp * dpw + q.rsmob.v);
  Jd[3 * kGas + 1] += wi * q.rsmob.ds * dpw;
  Jd[3 * kGas + 2] += wi * q.rsmob.dx * dpw;
}

// CNV_i = max over components of |R_c| dt / (PV b_c) (b of the phase carrying c)
BO_HD double cnv(const Props& q, const double* R, double dt) {
  double m = 0.0;
  for (int c = 0; c < 3; c++) {
    double v = (R[c] < 0.0 ? -R[c] : R[c]) * dt / (q.pv.v * q.b[c].v);
    m = v > m ? v : m;
  }
  return m;
}

// u <- u + du with the saturation chop (|dSw|, and |dSg| in cells with free gas, at most chop when
// chop > 0), then the switch.  Returns 1 when the cell's variable set changed.
BO_HD int update_cell(const Fluid& f, double chop, double dp, double dsw, double dx, double* p, double* sw, double* sg,
                      double* rs, unsigned char* sat) {
  if (chop > 0.0) {
    dsw = dsw > chop ? chop : (dsw < -chop ? -chop : dsw);
    if (*sat) dx = dx > chop ? chop : (dx < -chop ? -chop : dx);
  }
  *p += dp;
  *sw += dsw;
  if (*sat) {
    *sg += dx;
    *rs = rs_sat(f, *p);
    if (*sg < 0.0) {  // the gas phase disappears
      *sat = 0;
      *sg = 0.0;
      *rs = rs_sat(f, *p);
      return 1;
    }
    return 0;
  }
  *rs += dx;
  if (*rs > rs_sat(f, *p)) {  // free gas appears
    *sat = 1;
    *sg = 0.0;
    *rs = rs_sat(f, *p);
    return 1;
  }
  return 0;
}

}  // namespace bo
}  // namespace lns
