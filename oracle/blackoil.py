"""CPU FP64 oracle of the three-phase black-oil model with primary-variable switching.

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/``, it exists to check the CUDA path and is
called by the tests, the smoke check and the benchmark's CPU-baseline leg, never by the library.
It shares no code with the CUDA path.  It reuses the oil-water oracle's active-set logic
(Algorithm 1, steps 3-4, and the initial set), which is pinned on its own.

What it computes, in plain vectorised numpy, double precision:

* Appendix A's backward-Euler TPFA residual with phase-potential upwinding, for three phases and
  three components (water, oil, gas; surface volumes), gas dissolving in oil:
      R_c,i = [M_c(u_i) - M_c(u_i^n)] / dt + sum_j F_c,ij + q_c,i
      M_w = PV b_w Sw,  M_o = PV b_o So,  M_g = PV (b_g Sg + Rs b_o So),  So = 1 - Sw - Sg
      F_l,ij = T_ij (lambda_l b_l)_up dPhi_l,ij  for l = w, o, g (free gas),
      F_g,ij += T_ij (Rs lambda_o b_o)_up(o) dPhi_o,ij  (dissolved gas moves with the oil)
      dPhi_l,ij = (p_i - p_j) - g (rho_l,i + rho_l,j) / 2 (z_i - z_j)
      up = i if dPhi > 0, j if dPhi < 0, min(i, j) on a tie
      q_c,i = WI (lambda_c b_c)_i max(p_i - BHP, 0), and q_g += Rs_i q_o.
  Fluid functions: casegen.BlackOilFluid.  Equations in the order (oil, water, gas).
* Primary variables (p, Sw, X) per cell, X = Sg where free gas is present (saturated: Rs =
  Rs_sat(p)) and X = Rs where it is not (undersaturated: Sg = 0).  Section 3.1's variable
  substitution between Newton iterations, in its black-oil form: a cell without free gas whose
  oil holds more gas than Rs_sat(p) splits (free gas appears at Sg = 0, Rs = Rs_sat(p)); a cell
  whose Sg turns negative loses its gas phase (Sg = 0, Rs = Rs_sat(p) at that pressure).
* The Jacobian by forward-mode differentiation (dual numbers carrying d/d(p, Sw, X) of the cell,
  or of both cells of a face), so it is exact up to rounding; blocks 3 x 3, row = equation,
  column = unknown.
* Newton's method (Section 4.1), localized Newton (Section 4.3, Algorithm 1), adaptive nonlinear
  domain decomposition (Section 4.4, Algorithm 2, one Newton step per subdomain visit) and the
  residual-based active sets the paper compares against (mode 3), with the linear step
  J_A du_A = -F_A solved by scipy's sparse direct solver.  A cell whose variable set changed in an
  update counts as a non-negligible update (its unknowns changed meaning); an update that switched
  any cell is not converged.

Parity pins: tests/test_oracle_blackoil.py (reduction to the oil-water oracle at uniform Rs
without free gas; the gas equation equal to Rs times the oil equation there; central
differences; conservation of every component over a closed model; the two switches on a
closed cell whose solution is known; quadratic Newton convergence; planted mistakes).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Model as _SetModel
from . import Options as _SetOptions
from . import active_set_update as _active_set_update
from . import boundary as _boundary
from . import dd_expand as _dd_expand
from . import dilate as _dilate
from . import initial_set as _initial_set
from . import outer_halo as _outer_halo


# ---------------------------------------------------------------------------------------
# Dual numbers over arrays: value v (m,) and derivatives d (m, k)
# ---------------------------------------------------------------------------------------
class D:
    __slots__ = ("v", "d")
    __array_ufunc__ = None  # ndarray (op) D defers to D's reflected operators

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)

    @staticmethod
    def var(v, slot: int, k: int) -> "D":
        d = np.zeros((np.shape(v)[0], k))
        d[:, slot] = 1.0
        return D(v, d)

    def _lift(self, b) -> "D":
        if isinstance(b, D):
            return b
        return D(np.broadcast_to(np.asarray(b, dtype=np.float64), self.v.shape), np.zeros_like(self.d))

    def __add__(self, b):
        b = self._lift(b)
        return D(self.v + b.v, self.d + b.d)

    __radd__ = __add__

    def __neg__(self):
        return D(-self.v, -self.d)

    def __sub__(self, b):
        b = self._lift(b)
        return D(self.v - b.v, self.d - b.d)

    def __rsub__(self, b):
        return self._lift(b) - self

    def __mul__(self, b):
        b = self._lift(b)
        return D(self.v * b.v, self.d * b.v[:, None] + b.d * self.v[:, None])

    __rmul__ = __mul__

    def __truediv__(self, b):
        b = self._lift(b)
        return D(self.v / b.v, (self.d * b.v[:, None] - b.d * self.v[:, None]) / (b.v * b.v)[:, None])

    def __rtruediv__(self, b):
        return self._lift(b) / self

    def powi(self, k: int) -> "D":
        return D(self.v ** k, (k * self.v ** (k - 1))[:, None] * self.d)

    def __getitem__(self, idx) -> "D":
        return D(self.v[idx], self.d[idx])


def where(mask, a: D, b: D) -> D:
    mask = np.asarray(mask, dtype=bool)
    return D(np.where(mask, a.v, b.v), np.where(mask[:, None], a.d, b.d))


def clip01(a: D) -> D:
    """a clamped to [0, 1]; zero derivative outside (as the oil-water oracle's Corey clamps)."""
    lo, hi = a.v <= 0.0, a.v >= 1.0
    v = np.where(lo, 0.0, np.where(hi, 1.0, a.v))
    d = np.where((lo | hi)[:, None], 0.0, a.d)
    return D(v, d)


def widen(a: D, left: bool) -> D:
    """A cell quantity (3 derivative slots) as a face quantity (6 slots: the row cell, then the
    neighbour)."""
    z = np.zeros_like(a.d)
    return D(a.v, np.concatenate([a.d, z], axis=1) if left else np.concatenate([z, a.d], axis=1))


# ---------------------------------------------------------------------------------------
# State and cell properties
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class State:
    """p, Sw, Sg, Rs and the variable set per cell (sat = 1: free gas, X = Sg; 0: X = Rs)."""

    p: np.ndarray
    sw: np.ndarray
    sg: np.ndarray
    rs: np.ndarray
    sat: np.ndarray

    def copy(self) -> "State":
        return State(self.p.copy(), self.sw.copy(), self.sg.copy(), self.rs.copy(), self.sat.copy())

    @property
    def x(self) -> np.ndarray:
        return np.where(self.sat == 1, self.sg, self.rs)


def initial_state(bo) -> State:
    return State(np.array(bo.p0, np.float64), np.array(bo.sw0, np.float64), np.array(bo.sg0, np.float64),
                 np.array(bo.rs0, np.float64), np.array(bo.sat0, np.uint8))


def rs_sat(fl, p):
    """Saturated solution gas-oil ratio, linear in p (rs_max at the bubble point)."""
    return fl.rs_max * p / fl.p_bubble


def cell_props(fl, pv_ref, st: State) -> Dict[str, D]:
    """Per-cell properties as dual numbers in (p, Sw, X)."""
    k = 3
    P = D.var(st.p, 0, k)
    SW = D.var(st.sw, 1, k)
    X = D.var(st.x, 2, k)
    sat = st.sat == 1
    zero = D(np.zeros_like(st.p), np.zeros((st.p.shape[0], k)))
    SG = where(sat, X, zero)
    RS = where(sat, rs_sat(fl, P), X)
    SO = 1.0 - SW - SG
    dpr = P - fl.p_ref
    PV = pv_ref * (1.0 + fl.c_r * dpr)
    BW = fl.b_w_ref * (1.0 + fl.c_w * dpr)
    BO = fl.b_o_ref * (1.0 + fl.c_o * dpr) / (1.0 + fl.kappa * RS)
    BG = fl.b_g_per_pa * P
    span = 1.0 - fl.swc - fl.sor
    krw = clip01((SW - fl.swc) / span).powi(fl.n_w)
    kro = clip01((SO - fl.sor) / span).powi(fl.n_o)
    krg = clip01(SG / span).powi(fl.n_g)
    q = dict(P=P, SW=SW, SG=SG, SO=SO, RS=RS, PV=PV, BW=BW, BO=BO, BG=BG)
    q["rho_w"] = fl.rho_w_sc * BW
    q["rho_o"] = BO * (fl.rho_o_sc + fl.rho_g_sc * RS)
    q["rho_g"] = fl.rho_g_sc * BG
    q["mob_w"] = krw / fl.mu_w * BW
    q["mob_o"] = kro / fl.mu_o * BO
    q["mob_g"] = krg / fl.mu_g * BG
    q["mass_o"] = PV * BO * SO
    q["mass_w"] = PV * BW * SW
    q["mass_g"] = PV * (BG * SG + RS * BO * SO)
    return q


# ---------------------------------------------------------------------------------------
# Residual and Jacobian (Appendix A)
# ---------------------------------------------------------------------------------------
EQ = ("o", "w", "g")  # equation order: oil, water, gas


def _sub(st: State, idx: np.ndarray) -> State:
    return State(st.p[idx], st.sw[idx], st.sg[idx], st.rs[idx], st.sat[idx])


def assemble_cells(bo, st: State, old: State, dt: float, cells) -> Tuple[np.ndarray, np.ndarray, np.ndarray,
                                                                           np.ndarray]:
    """The rows of the given cells (ascending or not, no repeats): residual F (m, 3), diagonal blocks
    (m, 3, 3), the off-diagonal blocks of their adjacency entries (k, 3, 3) and those entries'
    indices e (k,) in CSR order of the given cells (row cells[i] for the entries of row i, column
    nbr[e]), in (p, Sw, X) of the current variable sets.  Only the given cells and their
    neighbours are evaluated, so a sample of rows of a large model costs little."""
    c, fl = bo.case, bo.fluid
    n = c.n
    cells = np.asarray(cells, dtype=np.int64)
    m = cells.shape[0]
    row_ptr = np.asarray(c.row_ptr, dtype=np.int64)
    cnt = row_ptr[cells + 1] - row_ptr[cells]
    first = np.cumsum(cnt) - cnt
    e_idx = np.repeat(row_ptr[cells], cnt) + (np.arange(int(cnt.sum())) - np.repeat(first, cnt))
    loc_row = np.repeat(np.arange(m), cnt)
    rows = cells[loc_row]
    cols = np.asarray(c.nbr, dtype=np.int64)[e_idx]
    need = np.unique(np.concatenate([cells, cols]))
    at = -np.ones(n, np.int64)
    at[need] = np.arange(need.shape[0])
    q = cell_props(fl, c.pv_ref[need], _sub(st, need))
    qn = cell_props(fl, c.pv_ref[cells], _sub(old, cells))
    own = at[cells]
    F = np.zeros((m, 3))
    Jd = np.zeros((m, 3, 3))
    for r, comp in enumerate(EQ):
        acc = (q["mass_" + comp][own] - qn["mass_" + comp].v) / dt
        F[:, r] += acc.v
        Jd[:, r, :] += acc.d
    T = np.asarray(c.trans, dtype=np.float64)[e_idx]
    dz = c.depth[rows] - c.depth[cols]
    g = fl.gravity
    Jo = np.zeros((e_idx.shape[0], 3, 3))
    ai, aj = at[rows], at[cols]

    def face(name):
        a = q[name]
        return widen(a[ai], True), widen(a[aj], False)

    Pi, Pj = face("P")
    up_oil = None
    flux = {}
    for ph in ("o", "w", "g"):
        ri, rj = face("rho_" + ph)
        dphi = (Pi - Pj) - g * dz * (0.5 * (ri + rj))
        up = (dphi.v > 0.0) | ((dphi.v == 0.0) & (rows < cols))
        mi, mj = face("mob_" + ph)
        flux[ph] = T * where(up, mi, mj) * dphi
        if ph == "o":
            up_oil, dphi_oil = up, dphi
    # dissolved gas travels with the oil, upwinded with it
    rs_mob = q["RS"] * q["mob_o"]
    rmi, rmj = widen(rs_mob[ai], True), widen(rs_mob[aj], False)
    flux["dg"] = T * where(up_oil, rmi, rmj) * dphi_oil
    for r, comp in enumerate(EQ):
        f = flux[comp] if comp != "g" else flux["g"] + flux["dg"]
        np.add.at(F[:, r], loc_row, f.v)
        np.add.at(Jd[:, r, :], loc_row, f.d[:, :3])
        Jo[:, r, :] = f.d[:, 3:]
    # producers at fixed bottom-hole pressure
    pos = -np.ones(n, np.int64)
    pos[cells] = np.arange(m)
    for w in range(c.well_cell.shape[0]):
        i = int(c.well_cell[w])
        if pos[i] < 0:
            continue
        k = int(pos[i])
        j = [int(at[i])]
        dpw = q["P"][j] - float(c.well_bhp[w])
        if dpw.v[0] <= 0.0:
            continue
        wi = float(c.well_wi[w])
        qo = wi * q["mob_o"][j] * dpw
        terms = dict(o=qo, w=wi * q["mob_w"][j] * dpw, g=wi * q["mob_g"][j] * dpw + q["RS"][j] * qo)
        for r, comp in enumerate(EQ):
            F[k, r] += terms[comp].v[0]
            Jd[k, r, :] += terms[comp].d[0]
    return F, Jd, Jo, e_idx


def assemble(bo, st: State, old: State, dt: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Full-domain residual F (n, 3) and Jacobian blocks: diagonal (n, 3, 3) and off-diagonal per
    adjacency entry (n_adj, 3, 3) (row i = the entry's row, column nbr[e]), in (p, Sw, X) of the
    current variable sets."""
    F, Jd, Jo, _ = assemble_cells(bo, st, old, dt, np.arange(bo.case.n))
    return F, Jd, Jo


def residual(bo, st: State, old: State, dt: float) -> np.ndarray:
    return assemble(bo, st, old, dt)[0]


def cnv(bo, st: State, F: np.ndarray, dt: float, cells=None) -> np.ndarray:
    """CNV_i = max over components of |R_c,i| dt / (PV_i b_c,i) (b of the phase carrying c); F holds
    the rows of ``cells`` (default: every cell)."""
    if cells is None:
        q = cell_props(bo.fluid, bo.case.pv_ref, st)
    else:
        cells = np.asarray(cells, dtype=np.int64)
        q = cell_props(bo.fluid, bo.case.pv_ref[cells], _sub(st, cells))
    pv = q["PV"].v
    scale = np.stack([q["BO"].v, q["BW"].v, q["BG"].v], axis=1) * pv[:, None]
    return np.max(np.abs(F) * dt / scale, axis=1)


# ---------------------------------------------------------------------------------------
# Newton step on an active set, update with variable switching
# ---------------------------------------------------------------------------------------
def local_solve(bo, st: State, old: State, dt: float, va: np.ndarray, sat_chop: float = 0.2):
    """One Newton step restricted to V_A (J_A du_A = -F_A, Section 4.3; inactive cells are fixed).
    Returns (du (n, 3) in (p, Sw, X), zero outside V_A and chopped, max CNV over V_A at the input
    state, max |dp| over V_A)."""
    c = bo.case
    n = c.n
    F, Jd, Jo = assemble(bo, st, old, dt)
    cv = cnv(bo, st, F, dt)
    act = np.flatnonzero(np.asarray(va) != 0)
    na = act.shape[0]
    du = np.zeros((n, 3))
    if na == 0:
        return du, 0.0, 0.0
    idx = -np.ones(n, np.int64)
    idx[act] = np.arange(na)
    rows = np.repeat(np.arange(n), np.diff(c.row_ptr))
    cols = np.asarray(c.nbr, dtype=np.int64)
    keep = (idx[rows] >= 0) & (idx[cols] >= 0)
    bi = np.concatenate([idx[act], idx[rows[keep]]])
    bj = np.concatenate([idx[act], idx[cols[keep]]])
    blocks = np.concatenate([Jd[act], Jo[keep]])
    # scatter the 3 x 3 blocks into a CSR matrix of order 3 n_A
    r3 = (3 * bi[:, None, None] + np.arange(3)[None, :, None]) + 0 * np.arange(3)[None, None, :]
    c3 = (3 * bj[:, None, None] + np.arange(3)[None, None, :]) + 0 * np.arange(3)[None, :, None]
    A = sp.csr_matrix((blocks.ravel(), (r3.ravel(), c3.ravel())), shape=(3 * na, 3 * na))
    x = spla.spsolve(A.tocsc(), -F[act].ravel())
    x = np.asarray(x).reshape(na, 3)
    if not np.all(np.isfinite(x)):
        raise ArithmeticError("singular local system in the black-oil oracle")
    if sat_chop > 0.0:
        x[:, 1] = np.clip(x[:, 1], -sat_chop, sat_chop)
        s = st.sat[act] == 1
        x[s, 2] = np.clip(x[s, 2], -sat_chop, sat_chop)
    du[act] = x
    return du, float(cv[act].max()), float(np.abs(x[:, 0]).max())


def apply_update(fl, st: State, du: np.ndarray, va: np.ndarray) -> Tuple[State, np.ndarray]:
    """u <- u + du on V_A, then Section 3.1's switch on every updated cell.  Returns the new state
    and the mask of cells whose variable set changed."""
    out = st.copy()
    a = np.asarray(va) != 0
    out.p[a] += du[a, 0]
    out.sw[a] += du[a, 1]
    s = a & (st.sat == 1)
    u = a & (st.sat == 0)
    out.sg[s] += du[s, 2]
    out.rs[s] = rs_sat(fl, out.p[s])
    out.rs[u] += du[u, 2]
    # gas phase disappears: Sg < 0 -> no free gas, the oil holds the saturated amount
    gone = s & (out.sg < 0.0)
    out.sat[gone] = 0
    out.sg[gone] = 0.0
    out.rs[gone] = rs_sat(fl, out.p[gone])
    # gas phase appears: the oil holds more than it can at this pressure -> free gas at Sg = 0
    split = u & (out.rs > rs_sat(fl, out.p))
    out.sat[split] = 1
    out.sg[split] = 0.0
    out.rs[split] = rs_sat(fl, out.p[split])
    return out, gone | split


# ---------------------------------------------------------------------------------------
# Timesteps: standard Newton and Algorithm 1
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    """mode 0 standard Newton, 1 Algorithm 1, 2 Algorithm 2, 3 residual-based sets; cutoffs and
    tolerances as the oil-water oracle's (eps_sw, when > 0, applies to max(|dSw|, |dSg|))."""

    mode: int = 1
    eps_p: float = 0.3 * 6894.757293168
    eps_sw: float = 0.0
    m_layers: int = 2
    tol_dp: float = 0.3 * 6894.757293168
    tol_cnv: float = 1e-6
    max_newton: int = 25
    sat_chop: float = 0.2
    max_dd_outer: int = 25

    def sets(self) -> _SetOptions:
        return _SetOptions(mode=self.mode, eps_p=self.eps_p, eps_sw=self.eps_sw, m_layers=self.m_layers,
                           tol_dp=self.tol_dp, tol_cnv=self.tol_cnv, max_newton=self.max_newton,
                           sat_chop=self.sat_chop, max_dd_outer=self.max_dd_outer)


class Sim:
    """Stateful black-oil oracle simulation: the state and the previous step's support set."""

    def __init__(self, bo, opts: Optional[Options] = None) -> None:
        self.bo = bo
        self.o = opts or Options()
        self.sm = _SetModel(bo.case)
        self.st = initial_state(bo)
        self.prev_supp = np.zeros(bo.n, np.uint8)
        self.has_prev = False

    def _big(self, dp, ds, switched) -> np.ndarray:
        """Non-negligible update: |dp| >= eps_p, or |dS| >= eps_sw when enabled, or a switch."""
        big = np.abs(dp) >= self.o.eps_p
        if self.o.eps_sw > 0.0:
            big |= ds >= self.o.eps_sw
        return big | switched

    def _solve(self, st: State, old: State, dt: float, va: np.ndarray):
        """One step on V_A: returns the new state, the update, the switched cells, the step's
        convergence test and |dp|, |dS| as the set logic reads them (a switch counts as big)."""
        o = self.o
        du, cnv_max, dp_max = local_solve(self.bo, st, old, dt, va, o.sat_chop)
        new, switched = apply_update(self.bo.fluid, st, du, va)
        converged = dp_max < o.tol_dp and cnv_max < o.tol_cnv and not switched.any()
        ds = np.maximum(np.abs(new.sw - st.sw), np.abs(new.sg - st.sg))
        dp_eff = np.where(switched, np.maximum(np.abs(du[:, 0]), o.eps_p), du[:, 0])
        ds_eff = np.where(switched, np.maximum(ds, max(o.eps_sw, 0.0)), ds)
        return new, switched, converged, dp_eff, ds_eff

    def timestep(self, dt: float) -> Dict:
        bo, o, n = self.bo, self.o, self.bo.n
        old = self.st.copy()
        st = self.st.copy()
        stats = dict(status=0, iterations=0, cell_updates=0, switches=0, trace=[], n_subdomains=0, dd_outer=0)

        def count(va, switched):
            na = int(np.count_nonzero(va))
            stats["iterations"] += 1
            stats["cell_updates"] += na
            stats["switches"] += int(switched.sum())
            stats["trace"].append(na)

        if o.mode in (0, 1):  # Section 4.1; Algorithm 1
            va = np.ones(n, np.uint8) if o.mode == 0 else _initial_set(self.sm, o.sets(), self.prev_supp,
                                                                        self.has_prev)
            is_expand, converged = 1, False
            while (o.mode == 1 and is_expand) or not converged:
                if stats["iterations"] >= o.max_newton:
                    stats["status"] = -4
                    break
                st_new, switched, converged, dp_eff, ds_eff = self._solve(st, old, dt, va)
                count(va, switched)
                if o.mode == 1:
                    va, _, is_expand = _active_set_update(self.sm, o.sets(), va, dp_eff, ds_eff, converged)
                st = st_new
        elif o.mode == 3:  # residual-based sets: unconverged cells inflated by m layers
            va = np.zeros(n, np.uint8)
            last_ok = False
            while True:
                F = residual(bo, st, old, dt)
                unconv = (cnv(bo, st, F, dt) >= o.tol_cnv).astype(np.uint8)
                if not unconv.any() and (stats["iterations"] == 0 or last_ok):
                    break
                if stats["iterations"] >= o.max_newton:
                    stats["status"] = -4
                    break
                if unconv.any():
                    va = _dilate(self.sm, unconv, o.m_layers)
                du, _, dp_max = local_solve(bo, st, old, dt, va, o.sat_chop)
                st, switched = apply_update(bo.fluid, st, du, va)
                last_ok = dp_max < o.tol_dp and not switched.any()
                count(va, switched)
        else:  # Algorithm 2: expansion into disjoint subdomains, then multiplicative Schwarz passes
            cap = max(o.max_newton, 1)
            it_cap = o.max_newton * (o.max_dd_outer + 1)
            VA = [_initial_set(self.sm, o.sets(), self.prev_supp, self.has_prev)]
            VB = [_boundary(self.sm, VA[0])]
            VD = [_outer_halo(self.sm, VA[0])]
            vt = VA[0].copy()
            last_solve, own_big = [], []
            big_stamp = np.zeros(n, np.int64)
            solve_id = 0

            def visit(k, st):
                nonlocal solve_id
                st_new, switched, conv1, dp_eff, ds_eff = self._solve(st, old, dt, VA[k])
                count(VA[k], switched)
                solve_id += 1
                big = (VA[k] != 0) & self._big(dp_eff, ds_eff, switched)
                big_stamp[big] = solve_id
                return st_new, conv1, dp_eff, ds_eff, bool(big.any())

            is_expand, k = 1, 0
            while is_expand:
                if k >= cap:
                    stats["status"] = -4
                    break
                st, _, dp_eff, ds_eff, ob = visit(k, st)
                last_solve.append(solve_id)
                own_big.append(ob)
                vt, va_n, vb_n, vd_n, is_expand = _dd_expand(self.sm, o.sets(), VB[k], dp_eff, ds_eff, vt)
                VA.append(va_n)
                VB.append(vb_n)
                VD.append(vd_n)
                k += 1
            N = k
            stats["n_subdomains"] = N
            converged, nu = False, 0
            while stats["status"] == 0 and not converged:
                if nu >= o.max_dd_outer:
                    stats["status"] = -4
                    break
                all_ok = True
                for s_ in range(N):
                    halo_big = bool(np.any((VD[s_] != 0) & (big_stamp > last_solve[s_])))
                    if not (own_big[s_] or halo_big):
                        continue
                    if stats["iterations"] >= it_cap:
                        stats["status"] = -4
                        break
                    st, conv1, _, _, ob = visit(s_, st)
                    last_solve[s_] = solve_id
                    own_big[s_] = ob
                    all_ok = all_ok and conv1
                nu += 1
                converged = all_ok
            stats["dd_outer"] = nu
        self.st = st
        ds = np.maximum(np.abs(st.sw - old.sw), np.abs(st.sg - old.sg))
        self.prev_supp = self._big(st.p - old.p, ds, st.sat != old.sat).astype(np.uint8)
        self.has_prev = True
        return stats

    def run(self, dts) -> list:
        return [self.timestep(float(dt)) for dt in dts]
