/*
 * lns_oracle.c -- CPU FP64 oracle for the localized fully implicit Newton solver.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, never by the library.  Plain serial C, double precision, no
 * blocking or fusion beyond what each definition states.  See lns_oracle.h for the
 * list of paper passages followed and the pins that check this file.
 */
#include "lns_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Fluid and rock properties (Section 2 / Appendix A reduced to oil-water):
 *   phi(p) PV_ref-scaled pore volume  PV = PV_ref (1 + c_r (p - p_ref))
 *   b_l(p) = b_l,ref (1 + c_l (p - p_ref))         (inverse formation volume factor)
 *   rho_l = rho_l,ref b_l                          (phase density)
 *   Se = (Sw - Swc) / (1 - Swc - Sor) clamped to [0, 1]
 *   k_rw = Se^n_w, k_ro = (1 - Se)^n_o             (Corey)
 *   lambda_l b_l = k_rl / mu_l * b_l               (the upwinded flux coefficient)
 *   M_o = PV b_o (1 - Sw), M_w = PV b_w Sw         (mass per cell, surface volume)
 * Phase index 0 = oil, 1 = water; unknowns (p, Sw).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  double pv, dpv;
  double b[2], db[2];
  double rho[2], drho[2];
  double mob[2], dmob_dp[2], dmob_ds[2];
  double mass[2], dmass_dp[2], dmass_ds[2];
} props;

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; i++) r *= x;
  return r;
}

static void cell_props(const orc_fluid* f, double pv_ref, double p, double sw, props* q) {
  double dpr = p - f->p_ref;
  q->pv = pv_ref * (1.0 + f->c_r * dpr);
  q->dpv = pv_ref * f->c_r;
  q->b[0] = f->b_o_ref * (1.0 + f->c_o * dpr);
  q->db[0] = f->b_o_ref * f->c_o;
  q->b[1] = f->b_w_ref * (1.0 + f->c_w * dpr);
  q->db[1] = f->b_w_ref * f->c_w;
  q->rho[0] = f->rho_o_ref * q->b[0];
  q->drho[0] = f->rho_o_ref * q->db[0];
  q->rho[1] = f->rho_w_ref * q->b[1];
  q->drho[1] = f->rho_w_ref * q->db[1];
  double span = 1.0 - f->swc - f->sor;
  double se = (sw - f->swc) / span, dse = 1.0 / span;
  if (se <= 0.0) {
    se = 0.0;
    dse = 0.0;
  } else if (se >= 1.0) {
    se = 1.0;
    dse = 0.0;
  }
  double kr[2], dkr[2];
  kr[0] = ipow(1.0 - se, f->n_o);
  dkr[0] = -(double)f->n_o * ipow(1.0 - se, f->n_o - 1) * dse;
  kr[1] = ipow(se, f->n_w);
  dkr[1] = (double)f->n_w * ipow(se, f->n_w - 1) * dse;
  double mu[2] = {f->mu_o, f->mu_w};
  for (int l = 0; l < 2; l++) {
    q->mob[l] = kr[l] / mu[l] * q->b[l];
    q->dmob_dp[l] = kr[l] / mu[l] * q->db[l];
    q->dmob_ds[l] = dkr[l] / mu[l] * q->b[l];
  }
  double so = 1.0 - sw;
  q->mass[0] = q->pv * q->b[0] * so;
  q->dmass_dp[0] = (q->dpv * q->b[0] + q->pv * q->db[0]) * so;
  q->dmass_ds[0] = -q->pv * q->b[0];
  q->mass[1] = q->pv * q->b[1] * sw;
  q->dmass_dp[1] = (q->dpv * q->b[1] + q->pv * q->db[1]) * sw;
  q->dmass_ds[1] = q->pv * q->b[1];
}

/* ------------------------------------------------------------------------------------
 * Residual and Jacobian (Appendix A, oil-water reading).  For cell i and phase l:
 *   R_l,i = [M_l(u_i) - M_l(u_i^n)] / dt + sum_j F_l,ij + q_l,i
 *   F_l,ij = T_ij (lambda_l b_l)_up dPhi_l,ij        (outflow from i to j)
 *   dPhi_l,ij = (p_i - p_j) - g rho_l,ij (z_i - z_j),  rho_l,ij = (rho_l,i + rho_l,j)/2
 *   up = i if dPhi > 0, j if dPhi < 0, min(i, j) on a tie  (phase-potential upwinding)
 *   q_l,i = WI (lambda_l b_l)_i max(p_i - BHP, 0)  (producer at fixed BHP)
 * ---------------------------------------------------------------------------------- */
void orc_assemble(const orc_model* m, const double* p, const double* sw, const double* pn,
                  const double* swn, double dt, double* F, double* Jd, double* Jo) {
  const orc_fluid* f = &m->fl;
  const double g = f->gravity;
  for (int32_t i = 0; i < m->n; i++) {
    props qi, qn;
    cell_props(f, m->pv_ref[i], p[i], sw[i], &qi);
    cell_props(f, m->pv_ref[i], pn[i], swn[i], &qn);
    double R[2], D[2][2];
    for (int l = 0; l < 2; l++) {
      R[l] = (qi.mass[l] - qn.mass[l]) / dt;
      D[l][0] = qi.dmass_dp[l] / dt;
      D[l][1] = qi.dmass_ds[l] / dt;
    }
    for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++) {
      int32_t j = m->nbr[e];
      props qj;
      cell_props(f, m->pv_ref[j], p[j], sw[j], &qj);
      double dz = m->depth[i] - m->depth[j];
      double dpp = p[i] - p[j];
      double O[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      for (int l = 0; l < 2; l++) {
        double rho_avg = 0.5 * (qi.rho[l] + qj.rho[l]);
        double dphi = dpp - (g * rho_avg) * dz;
        int up_is_i = dphi > 0.0 ? 1 : (dphi < 0.0 ? 0 : (i < j));
        const props* qu = up_is_i ? &qi : &qj;
        double tm = m->trans[e] * qu->mob[l];
        R[l] += tm * dphi;
        D[l][0] += tm * (1.0 - g * dz * 0.5 * qi.drho[l]);
        O[l][0] += tm * (-1.0 - g * dz * 0.5 * qj.drho[l]);
        if (up_is_i) {
          D[l][0] += m->trans[e] * qi.dmob_dp[l] * dphi;
          D[l][1] += m->trans[e] * qi.dmob_ds[l] * dphi;
        } else {
          O[l][0] += m->trans[e] * qj.dmob_dp[l] * dphi;
          O[l][1] += m->trans[e] * qj.dmob_ds[l] * dphi;
        }
      }
      if (Jo) {
        Jo[4 * (int64_t)e + 0] = O[0][0];
        Jo[4 * (int64_t)e + 1] = O[0][1];
        Jo[4 * (int64_t)e + 2] = O[1][0];
        Jo[4 * (int64_t)e + 3] = O[1][1];
      }
    }
    if (F) {
      F[2 * (int64_t)i] = R[0];
      F[2 * (int64_t)i + 1] = R[1];
    }
    if (Jd) {
      Jd[4 * (int64_t)i + 0] = D[0][0];
      Jd[4 * (int64_t)i + 1] = D[0][1];
      Jd[4 * (int64_t)i + 2] = D[1][0];
      Jd[4 * (int64_t)i + 3] = D[1][1];
    }
  }
  /* producers */
  for (int32_t w = 0; w < m->n_wells; w++) {
    int32_t i = m->well_cell[w];
    props qi;
    cell_props(f, m->pv_ref[i], p[i], sw[i], &qi);
    double dpw = p[i] - m->well_bhp[w];
    if (dpw <= 0.0) continue;
    for (int l = 0; l < 2; l++) {
      double wi = m->well_wi[w];
      if (F) F[2 * (int64_t)i + l] += wi * qi.mob[l] * dpw;
      if (Jd) {
        Jd[4 * (int64_t)i + 2 * l + 0] += wi * (qi.dmob_dp[l] * dpw + qi.mob[l]);
        Jd[4 * (int64_t)i + 2 * l + 1] += wi * qi.dmob_ds[l] * dpw;
      }
    }
  }
}

void orc_cnv(const orc_model* m, const double* p, const double* F, double dt, double* cnv) {
  for (int32_t i = 0; i < m->n; i++) {
    props q;
    cell_props(&m->fl, m->pv_ref[i], p[i], 0.5, &q);
    double c0 = fabs(F[2 * (int64_t)i]) * dt / (q.pv * q.b[0]);
    double c1 = fabs(F[2 * (int64_t)i + 1]) * dt / (q.pv * q.b[1]);
    cnv[i] = c0 > c1 ? c0 : c1;
  }
}

/* ------------------------------------------------------------------------------------
 * Hand-written block sparse LU.
 *   1. Nested-dissection ordering: split each connected piece at the middle level of a
 *      breadth-first level structure rooted at a pseudo-peripheral node; order the two
 *      halves recursively, the separator last.
 *   2. Symbolic factorization: elimination tree (Liu), row patterns of L by walking
 *      the tree from each entry of A's lower row; U's pattern is L's transposed
 *      (the pattern of A is structurally symmetric).
 *   3. Numeric: row-by-row Doolittle elimination with 2x2 block pivots.
 *   4. Forward and backward substitution.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  const int32_t *xadj, *adj;
  int32_t *mark, *vis, *lev, *queue;
  int32_t mark_id, vis_id;
  int32_t* perm;
  int32_t npos;
} nd_ctx;

static int32_t nd_bfs(nd_ctx* c, int32_t root, int32_t* order, int32_t* nlev) {
  /* BFS from root within nodes whose mark == mark_id; returns the number reached,
     fills order and lev; *nlev = number of levels. */
  c->vis_id++;
  int32_t head = 0, tail = 0;
  order[tail++] = root;
  c->vis[root] = c->vis_id;
  c->lev[root] = 0;
  int32_t maxl = 0;
  while (head < tail) {
    int32_t v = order[head++];
    for (int32_t e = c->xadj[v]; e < c->xadj[v + 1]; e++) {
      int32_t w = c->adj[e];
      if (c->mark[w] != c->mark_id || c->vis[w] == c->vis_id) continue;
      c->vis[w] = c->vis_id;
      c->lev[w] = c->lev[v] + 1;
      if (c->lev[w] > maxl) maxl = c->lev[w];
      order[tail++] = w;
    }
  }
  *nlev = maxl + 1;
  return tail;
}

static void nd_rec(nd_ctx* c, int32_t* S, int32_t ns);

static void nd_component(nd_ctx* c, int32_t* C, int32_t nc) {
  if (nc <= 64) {
    for (int32_t k = 0; k < nc; k++) c->perm[c->npos++] = C[k];
    return;
  }
  c->mark_id++;
  for (int32_t k = 0; k < nc; k++) c->mark[C[k]] = c->mark_id;
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * nc);
  int32_t nlev;
  nd_bfs(c, C[0], order, &nlev);
  int32_t a = order[nc - 1];
  nd_bfs(c, a, order, &nlev);
  int32_t b = order[nc - 1];
  int32_t nlev2;
  nd_bfs(c, b, order, &nlev2);
  if (nlev2 < nlev) nd_bfs(c, a, order, &nlev2);
  nlev = nlev2;
  if (nlev < 3) {
    for (int32_t k = 0; k < nc; k++) c->perm[c->npos++] = C[k];
    free(order);
    return;
  }
  /* count per level; choose the separator level where the cumulative count crosses nc/2 */
  int32_t* cnt = (int32_t*)calloc(nlev, sizeof(int32_t));
  for (int32_t k = 0; k < nc; k++) cnt[c->lev[order[k]]]++;
  int32_t cum = 0, sep = 1;
  for (int32_t l = 0; l < nlev; l++) {
    cum += cnt[l];
    if (cum >= nc / 2) {
      sep = l;
      break;
    }
  }
  if (sep < 1) sep = 1;
  if (sep > nlev - 2) sep = nlev - 2;
  int32_t *A = (int32_t*)malloc(sizeof(int32_t) * nc), *B = (int32_t*)malloc(sizeof(int32_t) * nc),
          *Z = (int32_t*)malloc(sizeof(int32_t) * nc);
  int32_t na = 0, nb = 0, nz = 0;
  for (int32_t k = 0; k < nc; k++) {
    int32_t v = order[k];
    int32_t l = c->lev[v];
    if (l < sep)
      A[na++] = v;
    else if (l > sep)
      B[nb++] = v;
    else
      Z[nz++] = v;
  }
  free(cnt);
  free(order);
  nd_rec(c, A, na);
  nd_rec(c, B, nb);
  for (int32_t k = 0; k < nz; k++) c->perm[c->npos++] = Z[k];
  free(A);
  free(B);
  free(Z);
}

static void nd_rec(nd_ctx* c, int32_t* S, int32_t ns) {
  if (ns == 0) return;
  /* split S into connected components (written back to back into comp, sizes in csz)
     and order each */
  c->mark_id++;
  int32_t my_mark = c->mark_id;
  for (int32_t k = 0; k < ns; k++) c->mark[S[k]] = my_mark;
  int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * ns);
  int32_t* csz = (int32_t*)malloc(sizeof(int32_t) * ns);
  int32_t ncomp = 0, tail = 0;
  c->vis_id++;
  int32_t comp_vis = c->vis_id;
  for (int32_t k = 0; k < ns; k++) {
    int32_t s = S[k];
    if (c->vis[s] == comp_vis) continue;
    int32_t head = tail, start = tail;
    comp[tail++] = s;
    c->vis[s] = comp_vis;
    while (head < tail) {
      int32_t v = comp[head++];
      for (int32_t e = c->xadj[v]; e < c->xadj[v + 1]; e++) {
        int32_t w = c->adj[e];
        if (c->mark[w] != my_mark || c->vis[w] == comp_vis) continue;
        c->vis[w] = comp_vis;
        comp[tail++] = w;
      }
    }
    csz[ncomp++] = tail - start;
  }
  int32_t start = 0;
  for (int32_t q = 0; q < ncomp; q++) {
    nd_component(c, comp + start, csz[q]);
    start += csz[q];
  }
  free(comp);
  free(csz);
}

static void nd_order(int32_t n, const int32_t* xadj, const int32_t* adj, int32_t* perm) {
  nd_ctx c;
  c.n = n;
  c.xadj = xadj;
  c.adj = adj;
  c.mark = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  c.vis = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  c.lev = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  c.queue = NULL;
  for (int32_t i = 0; i < n; i++) {
    c.mark[i] = 0;
    c.vis[i] = 0;
  }
  c.mark_id = 0;
  c.vis_id = 0;
  c.perm = perm;
  c.npos = 0;
  int32_t* all = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  for (int32_t i = 0; i < n; i++) all[i] = i;
  nd_rec(&c, all, n);
  free(all);
  free(c.mark);
  free(c.vis);
  free(c.lev);
}

static void blk_mul(const double* a, const double* b, double* c) { /* c = a b */
  c[0] = a[0] * b[0] + a[1] * b[2];
  c[1] = a[0] * b[1] + a[1] * b[3];
  c[2] = a[2] * b[0] + a[3] * b[2];
  c[3] = a[2] * b[1] + a[3] * b[3];
}

static int blk_inv(const double* a, double* r) {
  double det = a[0] * a[3] - a[1] * a[2];
  if (det == 0.0 || !isfinite(det)) return -1;
  r[0] = a[3] / det;
  r[1] = -a[1] / det;
  r[2] = -a[2] / det;
  r[3] = a[0] / det;
  return 0;
}

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

int orc_lu_solve(int32_t nb, const int32_t* row_ptr, const int32_t* col, const double* diag,
                 const double* off, const double* rhs, double* x, int64_t* fill) {
  if (nb <= 0) {
    if (fill) *fill = 0;
    return 0;
  }
  int32_t N = nb;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * N);
  int32_t* iperm = (int32_t*)malloc(sizeof(int32_t) * N);
  nd_order(N, row_ptr, col, perm);
  for (int32_t r = 0; r < N; r++) iperm[perm[r]] = r;
  /* permuted pattern */
  int32_t* pxadj = (int32_t*)malloc(sizeof(int32_t) * (N + 1));
  int32_t* padj = (int32_t*)malloc(sizeof(int32_t) * (row_ptr[N] > 0 ? row_ptr[N] : 1));
  int32_t* psrc = (int32_t*)malloc(sizeof(int32_t) * (row_ptr[N] > 0 ? row_ptr[N] : 1));
  pxadj[0] = 0;
  for (int32_t r = 0; r < N; r++) {
    int32_t o = perm[r];
    int32_t k = pxadj[r];
    for (int32_t e = row_ptr[o]; e < row_ptr[o + 1]; e++) {
      padj[k] = iperm[col[e]];
      psrc[k] = e;
      k++;
    }
    pxadj[r + 1] = k;
  }
  /* elimination tree */
  int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * N);
  int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * N);
  for (int32_t i = 0; i < N; i++) {
    parent[i] = -1;
    anc[i] = -1;
    for (int32_t e = pxadj[i]; e < pxadj[i + 1]; e++) {
      int32_t r = padj[e];
      if (r >= i) continue;
      while (anc[r] != -1 && anc[r] != i) {
        int32_t t = anc[r];
        anc[r] = i;
        r = t;
      }
      if (anc[r] == -1) {
        anc[r] = i;
        parent[r] = i;
      }
    }
  }
  /* row patterns of L: two passes (count, fill) */
  int32_t* mark = anc; /* reuse */
  for (int32_t i = 0; i < N; i++) mark[i] = -1;
  int64_t* lp = (int64_t*)malloc(sizeof(int64_t) * (N + 1));
  lp[0] = 0;
  for (int32_t i = 0; i < N; i++) {
    int64_t cnt = 0;
    mark[i] = i;
    for (int32_t e = pxadj[i]; e < pxadj[i + 1]; e++) {
      int32_t j = padj[e];
      if (j >= i) continue;
      while (mark[j] != i) {
        mark[j] = i;
        cnt++;
        j = parent[j];
      }
    }
    lp[i + 1] = lp[i] + cnt;
  }
  int64_t nl = lp[N];
  int32_t* li = (int32_t*)malloc(sizeof(int32_t) * (nl > 0 ? nl : 1));
  for (int32_t i = 0; i < N; i++) mark[i] = -1;
  for (int32_t i = 0; i < N; i++) {
    int64_t k = lp[i];
    mark[i] = i;
    for (int32_t e = pxadj[i]; e < pxadj[i + 1]; e++) {
      int32_t j = padj[e];
      if (j >= i) continue;
      while (mark[j] != i) {
        mark[j] = i;
        li[k++] = j;
        j = parent[j];
      }
    }
    qsort(li + lp[i], (size_t)(lp[i + 1] - lp[i]), sizeof(int32_t), cmp_i32);
  }
  /* U pattern = transpose of L pattern (rows ascending) */
  int64_t* up = (int64_t*)calloc((size_t)N + 1u, sizeof(int64_t));
  for (int64_t k = 0; k < nl; k++) up[li[k] + 1]++;
  for (int32_t i = 0; i < N; i++) up[i + 1] += up[i];
  int32_t* ui = (int32_t*)malloc(sizeof(int32_t) * (nl > 0 ? nl : 1));
  int64_t* upos = (int64_t*)malloc(sizeof(int64_t) * N);
  for (int32_t i = 0; i < N; i++) upos[i] = up[i];
  for (int32_t i = 0; i < N; i++)
    for (int64_t k = lp[i]; k < lp[i + 1]; k++) ui[upos[li[k]]++] = i;
  /* numeric */
  double* lv = (double*)malloc(sizeof(double) * 4 * (nl > 0 ? nl : 1));
  double* uv = (double*)malloc(sizeof(double) * 4 * (nl > 0 ? nl : 1));
  double* dinv = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  double* W = (double*)calloc((size_t)N * 4, sizeof(double));
  int status = 0;
  for (int32_t i = 0; i < N && status == 0; i++) {
    for (int64_t k = lp[i]; k < lp[i + 1]; k++) memset(W + 4 * (int64_t)li[k], 0, 4 * sizeof(double));
    for (int64_t k = up[i]; k < up[i + 1]; k++) memset(W + 4 * (int64_t)ui[k], 0, 4 * sizeof(double));
    int32_t o = perm[i];
    memcpy(W + 4 * (int64_t)i, diag + 4 * (int64_t)o, 4 * sizeof(double));
    for (int32_t e = pxadj[i]; e < pxadj[i + 1]; e++)
      memcpy(W + 4 * (int64_t)padj[e], off + 4 * (int64_t)psrc[e], 4 * sizeof(double));
    for (int64_t k = lp[i]; k < lp[i + 1]; k++) {
      int32_t kk = li[k];
      double lik[4];
      blk_mul(W + 4 * (int64_t)kk, dinv + 4 * (int64_t)kk, lik);
      memcpy(lv + 4 * k, lik, 4 * sizeof(double));
      for (int64_t q = up[kk]; q < up[kk + 1]; q++) {
        double t[4];
        blk_mul(lik, uv + 4 * q, t);
        double* w = W + 4 * (int64_t)ui[q];
        w[0] -= t[0];
        w[1] -= t[1];
        w[2] -= t[2];
        w[3] -= t[3];
      }
    }
    if (blk_inv(W + 4 * (int64_t)i, dinv + 4 * (int64_t)i) != 0) status = -1;
    for (int64_t k = up[i]; k < up[i + 1]; k++) memcpy(uv + 4 * k, W + 4 * (int64_t)ui[k], 4 * sizeof(double));
  }
  if (status == 0) {
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    for (int32_t r = 0; r < N; r++) {
      y[2 * r] = rhs[2 * (int64_t)perm[r]];
      y[2 * r + 1] = rhs[2 * (int64_t)perm[r] + 1];
    }
    for (int32_t i = 0; i < N; i++)
      for (int64_t k = lp[i]; k < lp[i + 1]; k++) {
        const double* L = lv + 4 * k;
        int32_t j = li[k];
        double y0 = y[2 * j], y1 = y[2 * j + 1];
        y[2 * i] -= L[0] * y0 + L[1] * y1;
        y[2 * i + 1] -= L[2] * y0 + L[3] * y1;
      }
    for (int32_t i = N - 1; i >= 0; i--) {
      for (int64_t k = up[i]; k < up[i + 1]; k++) {
        const double* U = uv + 4 * k;
        int32_t j = ui[k];
        double y0 = y[2 * j], y1 = y[2 * j + 1];
        y[2 * i] -= U[0] * y0 + U[1] * y1;
        y[2 * i + 1] -= U[2] * y0 + U[3] * y1;
      }
      const double* D = dinv + 4 * (int64_t)i;
      double a = y[2 * i], b = y[2 * i + 1];
      y[2 * i] = D[0] * a + D[1] * b;
      y[2 * i + 1] = D[2] * a + D[3] * b;
    }
    for (int32_t r = 0; r < N; r++) {
      x[2 * (int64_t)perm[r]] = y[2 * r];
      x[2 * (int64_t)perm[r] + 1] = y[2 * r + 1];
    }
    free(y);
  }
  if (fill) *fill = 2 * nl;
  free(perm);
  free(iperm);
  free(pxadj);
  free(padj);
  free(psrc);
  free(parent);
  free(anc);
  free(lp);
  free(li);
  free(up);
  free(ui);
  free(upos);
  free(lv);
  free(uv);
  free(dinv);
  free(W);
  return status;
}

/* ------------------------------------------------------------------------------------
 * Set logic (Section 4.3).
 *   V_nbr^{i,m}: all cells within m connection hops of cell i, i included.
 *   V_B: cells of V_A with at least one neighbour outside V_A (outermost layer).
 *   V_dB: cells outside V_A with at least one neighbour in V_A (outer halo, Section 4.4).
 * ---------------------------------------------------------------------------------- */
void orc_dilate(const orc_model* m, const uint8_t* seed, int32_t layers, uint8_t* out) {
  int32_t n = m->n;
  uint8_t* cur = (uint8_t*)malloc(n > 0 ? n : 1);
  memcpy(cur, seed, n);
  for (int32_t h = 0; h < layers; h++) {
    memcpy(out, cur, n);
    for (int32_t i = 0; i < n; i++) {
      if (!cur[i]) continue;
      for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++) out[m->nbr[e]] = 1;
    }
    memcpy(cur, out, n);
  }
  memcpy(out, cur, n);
  free(cur);
}

void orc_boundary(const orc_model* m, const uint8_t* va, uint8_t* vb) {
  for (int32_t i = 0; i < m->n; i++) {
    vb[i] = 0;
    if (!va[i]) continue;
    for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++)
      if (!va[m->nbr[e]]) {
        vb[i] = 1;
        break;
      }
  }
}

void orc_outer_halo(const orc_model* m, const uint8_t* va, uint8_t* vdb) {
  for (int32_t i = 0; i < m->n; i++) {
    vdb[i] = 0;
    if (va[i]) continue;
    for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++)
      if (va[m->nbr[e]]) {
        vdb[i] = 1;
        break;
      }
  }
}

/* |du_i| >= eps on pressure, or on saturation when that cutoff is enabled */
static int is_big(const orc_opts* o, double dp, double dsw) {
  if (fabs(dp) >= o->eps_p) return 1;
  if (o->eps_sw > 0.0 && fabs(dsw) >= o->eps_sw) return 1;
  return 0;
}

void orc_active_set_update(const orc_model* m, const orc_opts* o, uint8_t* va, const double* dp,
                           const double* dsw, int32_t converged, uint8_t* vb, int32_t* is_expand) {
  int32_t n = m->n;
  uint8_t* vb_old = (uint8_t*)malloc(n > 0 ? n : 1);
  uint8_t* E = (uint8_t*)calloc(n > 0 ? n : 1, 1);
  uint8_t* S = (uint8_t*)calloc(n > 0 ? n : 1, 1);
  orc_boundary(m, va, vb_old);
  int any_e = 0, any_s = 0;
  for (int32_t i = 0; i < n; i++) {
    if (!va[i]) continue;
    if (is_big(o, dp[i], dsw[i])) {
      S[i] = 1;
      any_s = 1;
      if (vb_old[i]) {
        E[i] = 1;
        any_e = 1;
      }
    }
  }
  if (any_e) {
    /* expand mode: V_A <- V_A united with V_nbr^{i,m} of every boundary cell with a
       non-negligible update (Algorithm 1, the loop over V_B) */
    uint8_t* R = (uint8_t*)malloc(n > 0 ? n : 1);
    orc_dilate(m, E, o->m_layers, R);
    for (int32_t i = 0; i < n; i++) va[i] = (uint8_t)(va[i] | R[i] | m->always[i]);
    free(R);
    *is_expand = 1;
  } else {
    /* shrink mode: V_A <- supp du_A (fractures and wells stay active); an empty support
       before convergence keeps the previous set */
    if (any_s || converged)
      for (int32_t i = 0; i < n; i++) va[i] = (uint8_t)(S[i] | m->always[i]);
    *is_expand = 0;
  }
  orc_boundary(m, va, vb);
  free(vb_old);
  free(E);
  free(S);
}

void orc_dd_expand(const orc_model* m, const orc_opts* o, const uint8_t* vb_k, const double* dp,
                   const double* dsw, uint8_t* vt, uint8_t* va_next, uint8_t* vb_next,
                   uint8_t* vdb_next, int32_t* is_expand) {
  int32_t n = m->n;
  uint8_t* E = (uint8_t*)calloc(n > 0 ? n : 1, 1);
  int any_e = 0;
  for (int32_t i = 0; i < n; i++)
    if (vb_k[i] && is_big(o, dp[i], dsw[i])) {
      E[i] = 1;
      any_e = 1;
    }
  uint8_t* R = (uint8_t*)malloc(n > 0 ? n : 1);
  orc_dilate(m, E, o->m_layers, R);
  int any_new = 0;
  for (int32_t i = 0; i < n; i++) {
    /* the next subdomain holds the newly reached cells only (partitions are disjoint) */
    va_next[i] = (uint8_t)(any_e && R[i] && !vt[i]);
    if (va_next[i]) any_new = 1;
  }
  for (int32_t i = 0; i < n; i++)
    if (any_e) vt[i] = (uint8_t)(vt[i] | R[i]);
  *is_expand = (any_e && any_new) ? 1 : 0;
  if (*is_expand) {
    uint8_t* vbt = (uint8_t*)malloc(n > 0 ? n : 1);
    orc_boundary(m, vt, vbt);
    for (int32_t i = 0; i < n; i++) vb_next[i] = (uint8_t)(vbt[i] & va_next[i]);
    orc_outer_halo(m, va_next, vdb_next);
    free(vbt);
  } else {
    memset(vb_next, 0, n);
    memset(vdb_next, 0, n);
  }
  free(E);
  free(R);
}

/* ------------------------------------------------------------------------------------
 * Localized Newton step: J_A du_A = -F_A with J_A = R_A J R_A^T (Section 4.3).  The
 * full residual and Jacobian are assembled and the active rows and columns taken out,
 * which is the definition; inactive cells act as Dirichlet values.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Block ILU(0) and BiCGStab (the oracle's iterative linear step, for models too large for
 * the sparse LU).  2x2 blocks; the factors overwrite copies of the matrix: row i's blocks left
 * of the diagonal hold L_ik (unit block diagonal), the diagonal and the blocks right of it hold
 * U.  Elimination in row order, no fill: A_ij -= L_ik U_kj only where (i, j) is in the pattern.
 * ---------------------------------------------------------------------------------- */
static int inv2(const double* a, double* out) {
  double det = a[0] * a[3] - a[1] * a[2];
  if (det == 0.0 || !isfinite(det)) return 1;
  out[0] = a[3] / det;
  out[1] = -a[1] / det;
  out[2] = -a[2] / det;
  out[3] = a[0] / det;
  return 0;
}

static void mm2(const double* a, const double* b, double* c) { /* c = a b */
  c[0] = a[0] * b[0] + a[1] * b[2];
  c[1] = a[0] * b[1] + a[1] * b[3];
  c[2] = a[2] * b[0] + a[3] * b[2];
  c[3] = a[2] * b[1] + a[3] * b[3];
}

static void mv2(const double* a, const double* x, double* y) { /* y = a x */
  y[0] = a[0] * x[0] + a[1] * x[1];
  y[1] = a[2] * x[0] + a[3] * x[1];
}

typedef struct {
  int32_t nb;
  const int32_t *rp, *cl;
  double *ld, *lo; /* factored diagonal (U_ii) and off-diagonal blocks */
  double* dinv;    /* U_ii^{-1} */
} ilu0;

static int ilu0_factor(ilu0* f, const double* diag, const double* off) {
  int32_t nb = f->nb;
  memcpy(f->ld, diag, sizeof(double) * 4 * (size_t)nb);
  memcpy(f->lo, off, sizeof(double) * 4 * (size_t)f->rp[nb]);
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (nb > 0 ? nb : 1));
  for (int32_t j = 0; j < nb; j++) pos[j] = -1;
  int bad = 0;
  for (int32_t i = 0; i < nb && !bad; i++) {
    for (int32_t q = f->rp[i]; q < f->rp[i + 1]; q++) pos[f->cl[q]] = q;
    for (int32_t q = f->rp[i]; q < f->rp[i + 1]; q++) {
      int32_t k = f->cl[q];
      if (k >= i) continue;                    /* row i's lower blocks, in column order */
      double l[4];
      mm2(f->lo + 4 * (int64_t)q, f->dinv + 4 * (int64_t)k, l); /* L_ik = A_ik U_kk^{-1} */
      memcpy(f->lo + 4 * (int64_t)q, l, sizeof(l));
      for (int32_t q2 = f->rp[k]; q2 < f->rp[k + 1]; q2++) {
        int32_t j = f->cl[q2];
        if (j <= k) continue;                  /* U_kj, j > k */
        double t[4];
        mm2(l, f->lo + 4 * (int64_t)q2, t);
        double* dst = (j == i) ? f->ld + 4 * (int64_t)i : (pos[j] >= 0 ? f->lo + 4 * (int64_t)pos[j] : NULL);
        if (!dst) continue;                    /* outside the pattern: dropped (no fill) */
        for (int c = 0; c < 4; c++) dst[c] -= t[c];
      }
    }
    if (inv2(f->ld + 4 * (int64_t)i, f->dinv + 4 * (int64_t)i)) bad = 1;
    for (int32_t q = f->rp[i]; q < f->rp[i + 1]; q++) pos[f->cl[q]] = -1;
  }
  free(pos);
  return bad;
}

/* z = (LU)^{-1} r */
static void ilu0_apply(const ilu0* f, const double* r, double* z) {
  int32_t nb = f->nb;
  for (int32_t i = 0; i < nb; i++) { /* L y = r, unit block diagonal */
    double y[2] = {r[2 * i], r[2 * i + 1]};
    for (int32_t q = f->rp[i]; q < f->rp[i + 1]; q++) {
      int32_t k = f->cl[q];
      if (k >= i) continue;
      double t[2];
      mv2(f->lo + 4 * (int64_t)q, z + 2 * (int64_t)k, t);
      y[0] -= t[0];
      y[1] -= t[1];
    }
    z[2 * i] = y[0];
    z[2 * i + 1] = y[1];
  }
  for (int32_t i = nb - 1; i >= 0; i--) { /* U x = y */
    double y[2] = {z[2 * i], z[2 * i + 1]};
    for (int32_t q = f->rp[i]; q < f->rp[i + 1]; q++) {
      int32_t j = f->cl[q];
      if (j <= i) continue;
      double t[2];
      mv2(f->lo + 4 * (int64_t)q, z + 2 * (int64_t)j, t);
      y[0] -= t[0];
      y[1] -= t[1];
    }
    mv2(f->dinv + 4 * (int64_t)i, y, z + 2 * (int64_t)i);
  }
}

static void bmatvec(int32_t nb, const int32_t* rp, const int32_t* cl, const double* diag, const double* off,
                    const double* x, double* y) {
  for (int32_t i = 0; i < nb; i++) {
    double a[2];
    mv2(diag + 4 * (int64_t)i, x + 2 * (int64_t)i, a);
    for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
      double t[2];
      mv2(off + 4 * (int64_t)q, x + 2 * (int64_t)cl[q], t);
      a[0] += t[0];
      a[1] += t[1];
    }
    y[2 * i] = a[0];
    y[2 * i + 1] = a[1];
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

int orc_ilu0_bicgstab(int32_t nb, const int32_t* row_ptr, const int32_t* col, const double* diag,
                      const double* off, const double* rhs, double* x, double rtol, int32_t maxit, int32_t* iters) {
  int64_t n2 = 2 * (int64_t)nb;
  size_t v = sizeof(double) * (size_t)(n2 > 0 ? n2 : 1);
  const size_t nd = sizeof(double) * 4 * (size_t)(nb > 0 ? nb : 1);
  const size_t no = sizeof(double) * 4 * (size_t)(row_ptr[nb] > 0 ? row_ptr[nb] : 1);
  ilu0 f = {nb, row_ptr, col, (double*)malloc(nd), (double*)malloc(no), (double*)malloc(nd)};
  double *r = (double*)malloc(v), *rh = (double*)malloc(v), *pv = (double*)malloc(v), *vv = (double*)malloc(v);
  double *ph = (double*)malloc(v), *sv = (double*)malloc(v), *sh = (double*)malloc(v), *tv = (double*)malloc(v);
  int status = 1, it = 0;
  for (int64_t i = 0; i < n2; i++) {
    x[i] = 0.0;
    r[i] = rhs[i];
    rh[i] = rhs[i];
    pv[i] = 0.0;
    vv[i] = 0.0;
  }
  double bn = sqrt(dot(n2, rhs, rhs));
  if (nb == 0 || bn == 0.0) {
    status = 0;
  } else if (ilu0_factor(&f, diag, off)) {
    status = 2;
  } else {
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    for (it = 1; it <= maxit; it++) {
      double rho1 = dot(n2, rh, r);
      if (rho1 == 0.0 || !isfinite(rho1)) {
        status = 2;
        break;
      }
      double beta = (rho1 / rho) * (alpha / omega);
      for (int64_t i = 0; i < n2; i++) pv[i] = r[i] + beta * (pv[i] - omega * vv[i]);
      ilu0_apply(&f, pv, ph);
      bmatvec(nb, row_ptr, col, diag, off, ph, vv);
      double rv = dot(n2, rh, vv);
      if (rv == 0.0 || !isfinite(rv)) {
        status = 2;
        break;
      }
      alpha = rho1 / rv;
      for (int64_t i = 0; i < n2; i++) sv[i] = r[i] - alpha * vv[i];
      if (sqrt(dot(n2, sv, sv)) <= rtol * bn) {
        for (int64_t i = 0; i < n2; i++) x[i] += alpha * ph[i];
        status = 0;
        break;
      }
      ilu0_apply(&f, sv, sh);
      bmatvec(nb, row_ptr, col, diag, off, sh, tv);
      double tt = dot(n2, tv, tv);
      omega = tt > 0.0 ? dot(n2, tv, sv) / tt : 0.0;
      for (int64_t i = 0; i < n2; i++) {
        x[i] += alpha * ph[i] + omega * sh[i];
        r[i] = sv[i] - omega * tv[i];
      }
      if (sqrt(dot(n2, r, r)) <= rtol * bn) {
        status = 0;
        break;
      }
      if (omega == 0.0) {
        status = 2;
        break;
      }
      rho = rho1;
    }
    if (it > maxit) it = maxit;
  }
  if (iters) *iters = it;
  free(f.ld);
  free(f.lo);
  free(f.dinv);
  free(r);
  free(rh);
  free(pv);
  free(vv);
  free(ph);
  free(sv);
  free(sh);
  free(tv);
  return status;
}

int orc_local_solve(const orc_model* m, const orc_opts* o, const double* p, const double* sw,
                    const double* pn, const double* swn, double dt, const uint8_t* va,
                    double* dp, double* dsw, double* cnv_max, double* dp_max) {
  int32_t n = m->n;
  double* F = (double*)malloc(sizeof(double) * 2 * (n > 0 ? n : 1));
  double* Jd = (double*)malloc(sizeof(double) * 4 * (n > 0 ? n : 1));
  double* Jo = (double*)malloc(sizeof(double) * 4 * (m->n_adj > 0 ? m->n_adj : 1));
  double* cnv = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  orc_assemble(m, p, sw, pn, swn, dt, F, Jd, Jo);
  orc_cnv(m, p, F, dt, cnv);
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int32_t na = 0;
  for (int32_t i = 0; i < n; i++) idx[i] = va[i] ? na++ : -1;
  int32_t* act = (int32_t*)malloc(sizeof(int32_t) * (na > 0 ? na : 1));
  for (int32_t i = 0; i < n; i++)
    if (idx[i] >= 0) act[idx[i]] = i;
  int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * (na + 1));
  int64_t nnz = 0;
  for (int32_t k = 0; k < na; k++)
    for (int32_t e = m->row_ptr[act[k]]; e < m->row_ptr[act[k] + 1]; e++)
      if (idx[m->nbr[e]] >= 0) nnz++;
  int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  double* ob = (double*)malloc(sizeof(double) * 4 * (nnz > 0 ? nnz : 1));
  double* db = (double*)malloc(sizeof(double) * 4 * (na > 0 ? na : 1));
  double* rhs = (double*)malloc(sizeof(double) * 2 * (na > 0 ? na : 1));
  double* x = (double*)malloc(sizeof(double) * 2 * (na > 0 ? na : 1));
  int64_t q = 0;
  double cmax = 0.0;
  for (int32_t k = 0; k < na; k++) {
    int32_t i = act[k];
    rp[k] = (int32_t)q;
    for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; e++) {
      int32_t j = m->nbr[e];
      if (idx[j] < 0) continue;
      cl[q] = idx[j];
      memcpy(ob + 4 * q, Jo + 4 * (int64_t)e, 4 * sizeof(double));
      q++;
    }
    memcpy(db + 4 * (int64_t)k, Jd + 4 * (int64_t)i, 4 * sizeof(double));
    rhs[2 * k] = -F[2 * (int64_t)i];
    rhs[2 * k + 1] = -F[2 * (int64_t)i + 1];
    if (cnv[i] > cmax) cmax = cnv[i];
  }
  rp[na] = (int32_t)q;
  int status;
  if (o->linear == 1) {
    int32_t its = 0;
    status = orc_ilu0_bicgstab(na, rp, cl, db, ob, rhs, x, o->lin_rtol > 0.0 ? o->lin_rtol : 1e-10,
                               o->lin_maxit > 0 ? o->lin_maxit : 5000, &its);
  } else {
    status = orc_lu_solve(na, rp, cl, db, ob, rhs, x, NULL);
  }
  for (int32_t i = 0; i < n; i++) {
    dp[i] = 0.0;
    dsw[i] = 0.0;
  }
  double dmax = 0.0;
  if (status == 0) {
    for (int32_t k = 0; k < na; k++) {
      int32_t i = act[k];
      double ds = x[2 * k + 1];
      if (o->sat_chop > 0.0) {
        if (ds > o->sat_chop) ds = o->sat_chop;
        if (ds < -o->sat_chop) ds = -o->sat_chop;
      }
      dp[i] = x[2 * k];
      dsw[i] = ds;
      if (fabs(dp[i]) > dmax) dmax = fabs(dp[i]);
    }
  }
  *cnv_max = cmax;
  *dp_max = dmax;
  free(F);
  free(Jd);
  free(Jo);
  free(cnv);
  free(idx);
  free(act);
  free(rp);
  free(cl);
  free(ob);
  free(db);
  free(rhs);
  free(x);
  return status;
}

void orc_initial_set(const orc_model* m, const orc_opts* o, const uint8_t* prev_supp,
                     int32_t has_prev, uint8_t* va) {
  int32_t n = m->n;
  if (has_prev) {
    for (int32_t i = 0; i < n; i++) va[i] = (uint8_t)(prev_supp[i] | m->always[i]);
  } else {
    orc_dilate(m, m->always, o->m_layers, va);
  }
}

static void apply_update(int32_t n, const uint8_t* va, double* p, double* sw, const double* dp,
                         const double* dsw) {
  for (int32_t i = 0; i < n; i++)
    if (va[i]) {
      p[i] += dp[i];
      sw[i] += dsw[i];
    }
}

static void or_into(int32_t n, uint8_t* acc, const uint8_t* s) {
  if (!acc) return;
  for (int32_t i = 0; i < n; i++) acc[i] = (uint8_t)(acc[i] | s[i]);
}

static int32_t count_set(int32_t n, const uint8_t* s) {
  int32_t c = 0;
  for (int32_t i = 0; i < n; i++) c += s[i] ? 1 : 0;
  return c;
}

/* Algorithm 2, a subdomain visit beyond its first local solve (the variants the paper names after
 * Algorithm 2 and in Section 6: solving a subproblem further, and exploiting the solution's locality
 * inside a subdomain).  The visit's first step has been taken on V_A^k (converged: its convergence
 * test).  Further steps, up to dd_local_newton in all, stop once a step converges; each solves
 * V_A^k, or with dd_local_shrink only the support of the previous step's update within V_A^k plus
 * the subdomain's always-active cells (none left: the visit ends).  Every step stamps its
 * non-negligible updates with the visit's solve id and can set own_big.  Returns 0, -1 (singular
 * local system) or -4 (iteration limit). */
static int dd_refine(const orc_model* m, const orc_opts* o, double* p, double* sw, const double* pn,
                     const double* swn, double dt, const uint8_t* vak, int converged, int32_t solve_id,
                     int32_t* big_stamp, int32_t* own_big, double* dp, double* dsw, uint8_t* set, int32_t* it,
                     int32_t it_cap, orc_step_stats* st, int32_t* trace, int32_t trace_cap, uint8_t* union_out,
                     double* cnv_max, double* dp_max) {
  int32_t n = m->n;
  for (int32_t j = 2; j <= o->dd_local_newton && !converged; j++) {
    if (o->dd_local_shrink) {
      for (int32_t i = 0; i < n; i++) set[i] = (uint8_t)(vak[i] && (is_big(o, dp[i], dsw[i]) || m->always[i]));
    } else {
      memcpy(set, vak, n);
    }
    int32_t na = count_set(n, set);
    if (na == 0) break;
    if (*it >= it_cap) return -4;
    if (orc_local_solve(m, o, p, sw, pn, swn, dt, set, dp, dsw, cnv_max, dp_max) != 0) return -1;
    apply_update(n, set, p, sw, dp, dsw);
    or_into(n, union_out, set);
    for (int32_t i = 0; i < n; i++)
      if (set[i] && is_big(o, dp[i], dsw[i])) {
        *own_big = 1;
        big_stamp[i] = solve_id;
      }
    if (trace && *it < trace_cap) trace[*it] = na;
    st->cell_updates += na;
    (*it)++;
    converged = *dp_max < o->tol_dp && *cnv_max < o->tol_cnv;
  }
  return 0;
}

int orc_timestep(const orc_model* m, const orc_opts* o, double* p, double* sw, uint8_t* prev_supp,
                 int32_t* has_prev, double dt, orc_step_stats* st, int32_t* trace, int32_t trace_cap,
                 uint8_t* union_out) {
  int32_t n = m->n;
  size_t nn = (size_t)(n > 0 ? n : 1);
  double* pn = (double*)malloc(sizeof(double) * nn);
  double* swn = (double*)malloc(sizeof(double) * nn);
  double* dp = (double*)malloc(sizeof(double) * nn);
  double* dsw = (double*)malloc(sizeof(double) * nn);
  uint8_t* va = (uint8_t*)malloc(nn);
  uint8_t* vb = (uint8_t*)malloc(nn);
  memcpy(pn, p, sizeof(double) * n); /* u^nu = u^n (Algorithm 1 line 1) */
  memcpy(swn, sw, sizeof(double) * n);
  memset(st, 0, sizeof(*st));
  if (union_out) memset(union_out, 0, n);
  int status = 0;
  int32_t it = 0;
  double cnv_max = 0.0, dp_max = 0.0;

  if (o->mode == 0) { /* standard Newton, Section 4.1 */
    memset(va, 1, n);
    int converged = 0;
    while (!converged) {
      if (it >= o->max_newton) {
        status = -4;
        break;
      }
      if (orc_local_solve(m, o, p, sw, pn, swn, dt, va, dp, dsw, &cnv_max, &dp_max) != 0) {
        status = -1;
        break;
      }
      apply_update(n, va, p, sw, dp, dsw);
      or_into(n, union_out, va);
      if (trace && it < trace_cap) trace[it] = n;
      st->cell_updates += n;
      it++;
      converged = dp_max < o->tol_dp && cnv_max < o->tol_cnv;
    }
  } else if (o->mode == 1) { /* Algorithm 1 */
    orc_initial_set(m, o, prev_supp, *has_prev, va);
    int32_t is_expand = 1;
    int converged = 0;
    while (is_expand || !converged) {
      if (it >= o->max_newton) {
        status = -4;
        break;
      }
      int32_t na = count_set(n, va);
      if (orc_local_solve(m, o, p, sw, pn, swn, dt, va, dp, dsw, &cnv_max, &dp_max) != 0) {
        status = -1;
        break;
      }
      apply_update(n, va, p, sw, dp, dsw); /* u^{nu+1} = u^nu + R_A^T du_A */
      or_into(n, union_out, va);
      if (trace && it < trace_cap) trace[it] = na;
      st->cell_updates += na;
      it++;
      converged = dp_max < o->tol_dp && cnv_max < o->tol_cnv; /* check convergence */
      orc_active_set_update(m, o, va, dp, dsw, converged, vb, &is_expand);
    }
  } else if (o->mode == 3) {
    /* Residual-based active set (the Lu-Beckner estimate the paper cites in Section 1 and
     * Section 4.2 as the alternative a-priori strategy): the cells whose scaled residual is not
     * converged (CNV_i >= tol_cnv, the full-domain residual at u^nu), inflated by m layers of
     * neighbours, form the next active set.  Converged when no cell is unconverged and the last
     * update is below tol_dp (at nu = 0: no cell unconverged).  An empty unconverged set before
     * convergence keeps the previous active set. */
    double* F = (double*)malloc(sizeof(double) * 2 * nn);
    double* Jd = (double*)malloc(sizeof(double) * 4 * nn);
    double* Jo = (double*)malloc(sizeof(double) * 4 * (size_t)(m->n_adj > 0 ? m->n_adj : 1));
    double* cnv = (double*)malloc(sizeof(double) * nn);
    uint8_t* unconv = (uint8_t*)malloc(nn);
    memset(va, 0, nn);
    for (;;) {
      orc_assemble(m, p, sw, pn, swn, dt, F, Jd, Jo);
      orc_cnv(m, p, F, dt, cnv);
      int32_t n_unconv = 0;
      for (int32_t i = 0; i < n; i++) {
        unconv[i] = (uint8_t)(cnv[i] >= o->tol_cnv);
        n_unconv += unconv[i];
      }
      if (n_unconv == 0 && (it == 0 || dp_max < o->tol_dp)) break; /* converged */
      if (it >= o->max_newton) {
        status = -4;
        break;
      }
      if (n_unconv > 0) orc_dilate(m, unconv, o->m_layers, va);
      int32_t na = count_set(n, va);
      if (orc_local_solve(m, o, p, sw, pn, swn, dt, va, dp, dsw, &cnv_max, &dp_max) != 0) {
        status = -1;
        break;
      }
      apply_update(n, va, p, sw, dp, dsw);
      or_into(n, union_out, va);
      if (trace && it < trace_cap) trace[it] = na;
      st->cell_updates += na;
      it++;
    }
    free(F);
    free(Jd);
    free(Jo);
    free(cnv);
    free(unconv);
  } else { /* Algorithm 2 */
    int32_t cap = o->max_newton > 0 ? o->max_newton : 1;
    uint8_t** VA = (uint8_t**)calloc(cap + 1, sizeof(uint8_t*));
    uint8_t** VB = (uint8_t**)calloc(cap + 1, sizeof(uint8_t*));
    uint8_t** VD = (uint8_t**)calloc(cap + 1, sizeof(uint8_t*));
    int32_t* last_solve = (int32_t*)calloc(cap + 1, sizeof(int32_t));
    int32_t* own_big = (int32_t*)calloc(cap + 1, sizeof(int32_t));
    int32_t* big_stamp = (int32_t*)calloc(nn, sizeof(int32_t)); /* solve id of the last non-negligible update */
    uint8_t* vt = (uint8_t*)malloc(nn);
    uint8_t* scratch = (uint8_t*)malloc(nn); /* the solved set of a visit's further steps */
    int32_t solve_id = 0;
    VA[0] = (uint8_t*)malloc(nn);
    VB[0] = (uint8_t*)malloc(nn);
    VD[0] = (uint8_t*)malloc(nn);
    orc_initial_set(m, o, prev_supp, *has_prev, VA[0]);
    orc_boundary(m, VA[0], VB[0]);
    orc_outer_halo(m, VA[0], VD[0]);
    memcpy(vt, VA[0], n); /* V_T = V_A^0 */
    int32_t k = 0, is_expand = 1;
    /* expansion phase (Algorithm 2, lines 5-22): solve V_A^k, build V_A^{k+1} */
    while (is_expand) {
      if (k >= cap) {
        status = -4;
        break;
      }
      int32_t na = count_set(n, VA[k]);
      if (orc_local_solve(m, o, p, sw, pn, swn, dt, VA[k], dp, dsw, &cnv_max, &dp_max) != 0) {
        status = -1;
        break;
      }
      apply_update(n, VA[k], p, sw, dp, dsw);
      or_into(n, union_out, VA[k]);
      solve_id++;
      last_solve[k] = solve_id;
      own_big[k] = 0;
      for (int32_t i = 0; i < n; i++)
        if (VA[k][i] && is_big(o, dp[i], dsw[i])) {
          own_big[k] = 1;
          big_stamp[i] = solve_id;
        }
      if (trace && it < trace_cap) trace[it] = na;
      st->cell_updates += na;
      it++;
      VA[k + 1] = (uint8_t*)malloc(nn);
      VB[k + 1] = (uint8_t*)malloc(nn);
      VD[k + 1] = (uint8_t*)malloc(nn);
      const int conv1 = dp_max < o->tol_dp && cnv_max < o->tol_cnv;
      orc_dd_expand(m, o, VB[k], dp, dsw, vt, VA[k + 1], VB[k + 1], VD[k + 1], &is_expand);
      /* the visit's further steps (variants; none with dd_local_newton = 1) */
      int rc = dd_refine(m, o, p, sw, pn, swn, dt, VA[k], conv1, solve_id, big_stamp, &own_big[k], dp, dsw, scratch,
                         &it, o->max_newton * (o->max_dd_outer + 1), st, trace, trace_cap, union_out, &cnv_max,
                         &dp_max);
      k++;
      if (rc != 0) {
        status = rc;
        break;
      }
    }
    int32_t N = k;
    st->n_subdomains = N;
    /* nonlinear DD loop (Algorithm 2, lines 25-37), multiplicative Schwarz */
    int converged = 0;
    int32_t nu = 0;
    while (status == 0 && !converged) {
      if (nu >= o->max_dd_outer) {
        status = -4;
        break;
      }
      int all_ok = 1;
      for (int32_t s = 0; s < N && status == 0; s++) {
        int halo_big = 0;
        for (int32_t i = 0; i < n; i++)
          if (VD[s][i] && big_stamp[i] > last_solve[s]) {
            halo_big = 1;
            break;
          }
        if (!(own_big[s] || halo_big)) continue;
        if (it >= o->max_newton * (o->max_dd_outer + 1)) {
          status = -4;
          break;
        }
        int32_t na = count_set(n, VA[s]);
        if (orc_local_solve(m, o, p, sw, pn, swn, dt, VA[s], dp, dsw, &cnv_max, &dp_max) != 0) {
          status = -1;
          break;
        }
        apply_update(n, VA[s], p, sw, dp, dsw);
        or_into(n, union_out, VA[s]);
        solve_id++;
        last_solve[s] = solve_id;
        own_big[s] = 0;
        for (int32_t i = 0; i < n; i++)
          if (VA[s][i] && is_big(o, dp[i], dsw[i])) {
            own_big[s] = 1;
            big_stamp[i] = solve_id;
          }
        if (trace && it < trace_cap) trace[it] = na;
        st->cell_updates += na;
        it++;
        const int conv1 = dp_max < o->tol_dp && cnv_max < o->tol_cnv;
        if (!conv1) all_ok = 0; /* the pass converges when every visited subdomain was already converged */
        int rc = dd_refine(m, o, p, sw, pn, swn, dt, VA[s], conv1, solve_id, big_stamp, &own_big[s], dp, dsw,
                           scratch, &it, o->max_newton * (o->max_dd_outer + 1), st, trace, trace_cap, union_out,
                           &cnv_max, &dp_max);
        if (rc != 0) status = rc;
      }
      nu++;
      converged = all_ok;
    }
    st->dd_outer = nu;
    for (int32_t s = 0; s <= cap; s++) {
      free(VA[s]);
      free(VB[s]);
      free(VD[s]);
    }
    free(VA);
    free(VB);
    free(VD);
    free(last_solve);
    free(own_big);
    free(big_stamp);
    free(vt);
    free(scratch);
  }
  /* support of the timestep's update: the next step's initial active set (Section 5.2) */
  for (int32_t i = 0; i < n; i++) prev_supp[i] = (uint8_t)is_big(o, p[i] - pn[i], sw[i] - swn[i]);
  *has_prev = 1;
  st->status = status;
  st->iterations = it;
  st->last_max_dp = dp_max;
  st->last_cnv = cnv_max;
  free(pn);
  free(swn);
  free(dp);
  free(dsw);
  free(va);
  free(vb);
  return status;
}
