"""Seeded synthetic models for the localized Newton solver (matrix + discrete fracture network).

This module builds the *inputs* of the method: the TPFA connection graph with its
transmissibilities, pore volumes, depths, fracture line ids, wells, the fluid
constants and the initial state.  It holds none of the solver's arithmetic
(no residual, no Jacobian, no active-set logic), so both the CPU oracle and the
CUDA path can take their inputs from it.

Geometry follows the paper's description of its test models (Section 5: 2D
matrix with embedded discrete fractures, a fractured producer at fixed BHP,
EDFM connections).  The paper gives no transmissibility formulas, so the standard
EDFM/DFM forms are used:

* matrix-matrix: harmonic TPFA, T = A * 2 k1 k2 / (k1 + k2) / dx;
* matrix-fracture: T = 2 A_f k_m / <d>, A_f = L_piece * h, <d> = (dx + dy) / 8
  (average normal distance of a cell to a fracture through its centre);
* fracture-fracture along a segment: T = k_f w h / L_piece;
* fracture-fracture at an intersection (star-delta):
  T = a_i a_j / (a_i + a_j), a = k_f w h / (L_piece / 2);
* well index (radial flow in the fracture plane, Peaceman radius):
  WI = 2 pi k_f w / ln(r_e / r_w), r_e = 0.14 sqrt(L^2 + h^2), r_w = 0.1 m.

All quantities are SI (Pa, m, m^2, Pa s, s).  Cells of one fracture segment are
numbered consecutively along the segment, after all matrix cells.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

PSI = 6894.757293168
DAY = 86400.0
MD = 9.869233e-16  # m^2 per millidarcy
CP = 1.0e-3  # Pa s per centipoise
GRAVITY = 9.80665


@dataclasses.dataclass
class Fluid:
    """Oil-water fluid and rock constants (SI).

    b_l(p) = b_l_ref (1 + c_l (p - p_ref)) is the inverse formation volume
    factor, rho_l = rho_l_ref b_l the phase density, phi(p) = phi_ref (1 + c_r (p - p_ref)).
    Corey relative permeabilities with integer exponents n_w, n_o.
    """

    p_ref: float = 5000.0 * PSI
    c_r: float = 1.0e-6 / PSI
    b_o_ref: float = 1.0
    c_o: float = 1.0e-5 / PSI
    b_w_ref: float = 1.0
    c_w: float = 3.0e-6 / PSI
    rho_o_ref: float = 800.0
    rho_w_ref: float = 1000.0
    mu_o: float = 2.0 * CP
    mu_w: float = 0.5 * CP
    swc: float = 0.2
    sor: float = 0.2
    n_w: int = 2
    n_o: int = 2
    gravity: float = GRAVITY

    def as_tuple(self) -> Tuple:
        return dataclasses.astuple(self)


@dataclasses.dataclass
class Case:
    """A model description: CSR connection graph (each connection stored at both
    endpoints, neighbours ascending within a row), cell data, wells, fluid, initial
    state and the timestep schedule (seconds)."""

    name: str
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    nbr: np.ndarray  # int32 [n_adj]
    trans: np.ndarray  # float64 [n_adj]
    pv_ref: np.ndarray  # float64 [n]
    depth: np.ndarray  # float64 [n]
    line_id: np.ndarray  # int32 [n]  fracture segment id, -1 for matrix
    always_active: np.ndarray  # uint8 [n] fracture and well cells
    well_cell: np.ndarray  # int32 [n_wells]
    well_wi: np.ndarray  # float64 [n_wells]
    well_bhp: np.ndarray  # float64 [n_wells]
    fluid: Fluid
    p0: np.ndarray  # float64 [n]
    sw0: np.ndarray  # float64 [n]
    dt_schedule: np.ndarray  # float64 [n_steps], seconds
    n_matrix: int = 0
    meta: Dict = dataclasses.field(default_factory=dict)

    @property
    def n_adj(self) -> int:
        return int(self.nbr.shape[0])

    @property
    def n_wells(self) -> int:
        return int(self.well_cell.shape[0])

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


class _Builder:
    """Collects cells and undirected connections, then emits a symmetric CSR graph."""

    def __init__(self) -> None:
        self.pv: List[np.ndarray] = []
        self.depth: List[np.ndarray] = []
        self.line: List[np.ndarray] = []
        self.n = 0
        self.ci: List[np.ndarray] = []
        self.cj: List[np.ndarray] = []
        self.ct: List[np.ndarray] = []
        self.n_lines = 0
        self.wells: List[Tuple[int, float, float]] = []

    def add_cells(self, pv: np.ndarray, depth: np.ndarray, line: Optional[int] = None) -> np.ndarray:
        k = pv.shape[0]
        ids = np.arange(self.n, self.n + k, dtype=np.int64)
        self.pv.append(np.asarray(pv, dtype=np.float64))
        self.depth.append(np.asarray(depth, dtype=np.float64))
        self.line.append(np.full(k, -1 if line is None else line, dtype=np.int32))
        self.n += k
        return ids

    def connect(self, i: np.ndarray, j: np.ndarray, t: np.ndarray) -> None:
        i = np.asarray(i, dtype=np.int64).ravel()
        j = np.asarray(j, dtype=np.int64).ravel()
        t = np.asarray(t, dtype=np.float64).ravel()
        t = np.broadcast_to(t, i.shape) if t.size == 1 else t
        keep = i != j
        self.ci.append(i[keep])
        self.cj.append(j[keep])
        self.ct.append(t[keep].copy())

    def finalize(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        if self.ci:
            i = np.concatenate(self.ci)
            j = np.concatenate(self.cj)
            t = np.concatenate(self.ct)
        else:
            i = np.zeros(0, np.int64)
            j = np.zeros(0, np.int64)
            t = np.zeros(0)
        lo = np.minimum(i, j)
        hi = np.maximum(i, j)
        # merge duplicate undirected connections (parallel transmissibilities add)
        key = lo * self.n + hi
        order = np.argsort(key, kind="stable")
        key = key[order]
        t = t[order]
        uniq, start = np.unique(key, return_index=True)
        tsum = np.add.reduceat(t, start) if t.size else t
        lo = uniq // self.n
        hi = uniq % self.n
        rows = np.concatenate([lo, hi])
        cols = np.concatenate([hi, lo])
        tt = np.concatenate([tsum, tsum])
        order = np.lexsort((cols, rows))
        rows = rows[order]
        cols = cols[order]
        tt = tt[order]
        row_ptr = np.zeros(self.n + 1, dtype=np.int64)
        np.add.at(row_ptr, rows + 1, 1)
        row_ptr = np.cumsum(row_ptr)
        return row_ptr.astype(np.int32), cols.astype(np.int32), tt.astype(np.float64)


def _lognormal_perm(rng: np.random.Generator, shape, mean_md: float, sigma: float) -> np.ndarray:
    return np.exp(np.log(mean_md) + sigma * rng.standard_normal(shape)) * MD


def _add_matrix(b: _Builder, nx: int, ny: int, dx: float, dy: float, h: float, perm: np.ndarray,
                poro: float, depth: float) -> np.ndarray:
    ids = b.add_cells(np.full(nx * ny, dx * dy * h * poro), np.full(nx * ny, depth))
    k = perm.reshape(ny, nx)
    idx = ids.reshape(ny, nx)
    # x-connections
    k1, k2 = k[:, :-1], k[:, 1:]
    tx = (dy * h / dx) * 2.0 * k1 * k2 / (k1 + k2)
    b.connect(idx[:, :-1], idx[:, 1:], tx)
    k1, k2 = k[:-1, :], k[1:, :]
    ty = (dx * h / dy) * 2.0 * k1 * k2 / (k1 + k2)
    b.connect(idx[:-1, :], idx[1:, :], ty)
    return ids


@dataclasses.dataclass
class _Segment:
    x0: float
    y0: float
    x1: float
    y1: float
    n_cells: int
    k_f: float
    w: float
    ids: Optional[np.ndarray] = None

    @property
    def length(self) -> float:
        return math.hypot(self.x1 - self.x0, self.y1 - self.y0)


def _add_segments(b: _Builder, segs: Sequence[_Segment], nx: int, ny: int, dx: float, dy: float,
                  h: float, k_m: np.ndarray, depth: float, phi_f: float = 1.0) -> None:
    """Discretize each segment into equal pieces (consecutive ids), connect the chain,
    connect every piece to the matrix cell holding its midpoint, and connect
    intersecting pieces of different segments (star-delta)."""
    d_avg = (dx + dy) / 8.0
    for s in segs:
        L = s.length / s.n_cells
        line = b.n_lines
        b.n_lines += 1
        s.ids = b.add_cells(np.full(s.n_cells, L * s.w * h * phi_f), np.full(s.n_cells, depth), line=line)
        if s.n_cells > 1:
            b.connect(s.ids[:-1], s.ids[1:], s.k_f * s.w * h / L)
        tmid = (np.arange(s.n_cells) + 0.5) / s.n_cells
        xm = s.x0 + tmid * (s.x1 - s.x0)
        ym = s.y0 + tmid * (s.y1 - s.y0)
        ix = np.clip(np.floor(xm / dx).astype(np.int64), 0, nx - 1)
        iy = np.clip(np.floor(ym / dy).astype(np.int64), 0, ny - 1)
        mcell = iy * nx + ix
        b.connect(s.ids, mcell, 2.0 * L * h * k_m[mcell] / d_avg)
    # intersections between segments
    nseg = len(segs)
    if nseg < 2:
        return
    P = np.array([[s.x0, s.y0] for s in segs])
    Q = np.array([[s.x1, s.y1] for s in segs])
    R = Q - P
    ia, ib = np.triu_indices(nseg, 1)
    r = R[ia]
    s_ = R[ib]
    qp = P[ib] - P[ia]
    den = r[:, 0] * s_[:, 1] - r[:, 1] * s_[:, 0]
    ok = np.abs(den) > 1e-12
    den_safe = np.where(ok, den, 1.0)
    t = (qp[:, 0] * s_[:, 1] - qp[:, 1] * s_[:, 0]) / den_safe
    u = (qp[:, 0] * r[:, 1] - qp[:, 1] * r[:, 0]) / den_safe
    hit = ok & (t >= 0) & (t <= 1) & (u >= 0) & (u <= 1)
    for a, bb, ta, ub in zip(ia[hit], ib[hit], t[hit], u[hit]):
        sa, sb = segs[a], segs[bb]
        pa = min(int(ta * sa.n_cells), sa.n_cells - 1)
        pb = min(int(ub * sb.n_cells), sb.n_cells - 1)
        La = sa.length / sa.n_cells
        Lb = sb.length / sb.n_cells
        al_a = sa.k_f * sa.w * h / (La / 2.0)
        al_b = sb.k_f * sb.w * h / (Lb / 2.0)
        b.connect([sa.ids[pa]], [sb.ids[pb]], al_a * al_b / (al_a + al_b))


def _peaceman_wi(k_f: float, w: float, L: float, h: float, r_w: float = 0.1) -> float:
    r_e = 0.14 * math.sqrt(L * L + h * h)
    return 2.0 * math.pi * k_f * w / math.log(r_e / r_w)


def _finish(b: _Builder, name: str, fluid: Fluid, p_init: float, sw_init: float,
            dts: np.ndarray, n_matrix: int, meta: Dict) -> Case:
    row_ptr, nbr, trans = b.finalize()
    n = b.n
    line = np.concatenate(b.line) if b.line else np.zeros(0, np.int32)
    always = (line >= 0).astype(np.uint8)
    wc = np.array([w[0] for w in b.wells], dtype=np.int32)
    always[wc] = 1
    return Case(
        name=name, n=n, row_ptr=row_ptr, nbr=nbr, trans=trans,
        pv_ref=np.concatenate(b.pv), depth=np.concatenate(b.depth), line_id=line,
        always_active=always, well_cell=wc,
        well_wi=np.array([w[1] for w in b.wells], dtype=np.float64),
        well_bhp=np.array([w[2] for w in b.wells], dtype=np.float64),
        fluid=fluid, p0=np.full(n, p_init), sw0=np.full(n, sw_init),
        dt_schedule=np.asarray(dts, dtype=np.float64), n_matrix=n_matrix, meta=meta)


def geometric_schedule(n_steps: int, total_days: float, dt0_days: float = 0.01,
                       dt_max_days: float = 30.0) -> np.ndarray:
    """dt_k = min(dt0 r^k, dt_max) with r chosen by bisection so the steps sum to total_days."""

    def total(r: float) -> float:
        return float(sum(min(dt0_days * r ** k, dt_max_days) for k in range(n_steps)))

    lo, hi = 1.0, 10.0
    if total(hi) < total_days:
        raise ValueError("schedule cannot reach the requested total")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < total_days:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    return np.array([min(dt0_days * r ** k, dt_max_days) for k in range(n_steps)]) * DAY


def doubling_schedule(n_steps: int, dt0_days: float = 0.01, dt_max_days: float = 30.0) -> np.ndarray:
    return np.array([min(dt0_days * 2.0 ** k, dt_max_days) for k in range(n_steps)]) * DAY


def dfn_case(nx: int, ny: int, dx: float, n_dfn: int, seed: int, *, h: float = 1.0,
             k_mean_md: float = 1e-4, k_sigma: float = 0.5, poro: float = 0.06,
             hf: Optional[Sequence[Tuple[float, float, float, float, int]]] = None,
             hf_k_md: float = 1e4, hf_w: float = 0.01,
             nf_k_md: float = 1e3, nf_w: float = 0.001,
             nf_len: Tuple[float, float] = (20.0, 200.0),
             strikes: Tuple[Tuple[float, float], ...] = ((30.0, 10.0), (120.0, 10.0)),
             wells: Optional[Sequence[Tuple[int, int, float]]] = None,
             p_init: float = 5000.0 * PSI, sw_init: float = 0.25,
             fluid: Optional[Fluid] = None, dts: Optional[np.ndarray] = None,
             depth: float = 2500.0, name: str = "dfn") -> Case:
    """2D matrix of nx x ny square cells plus hydraulic fractures ``hf`` (x0, y0, x1, y1, n_cells)
    and ``n_dfn`` seeded natural fractures in the given strike sets.  ``wells`` lists
    (hf index, piece index, BHP) producers perforated in hydraulic-fracture cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = fluid or Fluid(p_ref=p_init)
    b = _Builder()
    perm = _lognormal_perm(rng, nx * ny, k_mean_md, k_sigma)
    _add_matrix(b, nx, ny, dx, dx, h, perm, poro, depth)
    n_matrix = b.n
    Lx, Ly = nx * dx, ny * dx
    segs: List[_Segment] = []
    for (x0, y0, x1, y1, nc) in (hf or []):
        segs.append(_Segment(x0, y0, x1, y1, nc, hf_k_md * MD, hf_w))
    n_hf = len(segs)
    for s_i in range(n_dfn):
        mean, half = strikes[s_i % len(strikes)]
        ang = math.radians(mean + rng.uniform(-half, half))
        L = rng.uniform(*nf_len)
        cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
        ux, uy = math.cos(ang) * L / 2, math.sin(ang) * L / 2
        x0 = min(max(cx - ux, 1e-6), Lx - 1e-6)
        x1 = min(max(cx + ux, 1e-6), Lx - 1e-6)
        y0 = min(max(cy - uy, 1e-6), Ly - 1e-6)
        y1 = min(max(cy + uy, 1e-6), Ly - 1e-6)
        length = math.hypot(x1 - x0, y1 - y0)
        if length < 0.5 * dx:
            continue
        nc = max(1, int(round(length / dx)))
        segs.append(_Segment(x0, y0, x1, y1, nc, nf_k_md * MD, nf_w))
    _add_segments(b, segs, nx, ny, dx, dx, h, perm, depth)
    for (fi, piece, bhp) in (wells or []):
        s = segs[fi]
        L = s.length / s.n_cells
        b.wells.append((int(s.ids[piece]), _peaceman_wi(s.k_f, s.w, L, h), bhp))
    meta = dict(nx=nx, ny=ny, dx=dx, h=h, n_segments=len(segs), n_hf=n_hf, seed=seed,
                n_fracture_cells=b.n - n_matrix)
    if dts is None:
        dts = doubling_schedule(12)
    return _finish(b, name, fluid, p_init, sw_init, dts, n_matrix, meta)


def config0(seed: int = 0) -> Case:
    """50x50 matrix (10 m cells, 1 m thick), one vertical fracture of 20 cells (1 cm wide,
    1e4 mD) in column 25, rows 15-34; producer in fracture cell 10 at 1000 psi;
    12 steps, dt doubling from 0.01 d."""
    dx = 10.0
    x = 25 * dx + dx / 2
    hf = [(x, 15 * dx, x, 35 * dx, 20)]
    return dfn_case(50, 50, dx, 0, seed, hf=hf, wells=[(0, 10, 1000.0 * PSI)],
                    dts=doubling_schedule(12), name="config0_50x50_1frac")


def config1(seed: int = 1) -> Case:
    """400x400 matrix (5 m cells) + 300 seeded natural fractures in two strike sets +
    4 hydraulic fractures of 80 cells on a horizontal producer at 1500 psi; 40 steps to 365 d."""
    dx = 5.0
    hf = []
    for c in (170, 190, 210, 230):
        x = c * dx + dx / 2
        hf.append((x, 160 * dx, x, 240 * dx, 80))
    wells = [(i, 40, 1500.0 * PSI) for i in range(4)]
    return dfn_case(400, 400, dx, 300, seed, hf=hf, wells=wells,
                    dts=geometric_schedule(40, 365.0), name="config1_400x400_dfn300")


def small_dfn(nx: int = 24, ny: int = 20, n_dfn: int = 6, seed: int = 7, n_steps: int = 6,
              dx: float = 5.0) -> Case:
    """A few-hundred-cell DFN model with one hydraulic fracture and a producer, for fast tests."""
    x = (nx // 2) * dx + dx / 2
    y0 = (ny // 4) * dx
    y1 = (3 * ny // 4) * dx
    nc = max(2, 3 * ny // 4 - ny // 4)
    hf = [(x, y0, x, y1, nc)]
    return dfn_case(nx, ny, dx, n_dfn, seed, hf=hf, wells=[(0, nc // 2, 1500.0 * PSI)],
                    nf_len=(3 * dx, 8 * dx), dts=doubling_schedule(n_steps), name=f"small_{nx}x{ny}")


def chain_1d(n: int, dx: float, k: float, poro: float, area: float, *, p_init: float,
             p_well: float, fluid: Fluid, dts: np.ndarray, wi: float = 1e3,
             depth: float = 1000.0) -> Case:
    """1D chain of n cells (cross-section ``area``) with a producer of huge index in cell 0:
    cell 0 is held at ``p_well`` (a constant-pressure fracture at x = 0)."""
    b = _Builder()
    ids = b.add_cells(np.full(n, dx * area * poro), np.full(n, depth))
    b.connect(ids[:-1], ids[1:], k * area / dx)
    b.wells.append((0, wi, p_well))
    return _finish(b, f"chain_{n}", fluid, p_init, fluid.swc, dts, n, dict(dx=dx, n=n))


def column_1d(n: int, dz: float, k: float, poro: float, area: float, *, top_depth: float,
              fluid: Fluid, dts: np.ndarray) -> Case:
    """Vertical column of n cells (no wells); initial state is set by the caller."""
    b = _Builder()
    ids = b.add_cells(np.full(n, dz * area * poro), top_depth + dz * (np.arange(n) + 0.5))
    b.connect(ids[:-1], ids[1:], k * area / dz)
    return _finish(b, f"column_{n}", fluid, fluid.p_ref, fluid.swc, dts, n, dict(dz=dz, n=n))


def grid_2d(nx: int, ny: int, dx: float = 5.0, seed: int = 3, *, with_well: bool = True,
            n_steps: int = 4) -> Case:
    """Plain matrix grid (no fractures), optional producer in the centre cell."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = Fluid()
    b = _Builder()
    perm = _lognormal_perm(rng, nx * ny, 1.0, 0.5)
    _add_matrix(b, nx, ny, dx, dx, 1.0, perm, 0.1, 2500.0)
    if with_well:
        c = (ny // 2) * nx + nx // 2
        b.wells.append((c, 2.0 * math.pi * perm[c] * 1.0 / math.log(0.2 * dx / 0.1), 3000.0 * PSI))
    return _finish(b, f"grid_{nx}x{ny}", fluid, fluid.p_ref, 0.25, doubling_schedule(n_steps, 0.1),
                   nx * ny, dict(nx=nx, ny=ny))


def realization(index: int, dx: float = 5.0, n_steps: int = 12) -> Case:
    """One member of a seeded ensemble of DFN models of uneven size: an N x N matrix with
    N ~ U{150..500}, U{50..400} natural fractures, and two hydraulic fractures on a producer
    at 1500 psi through the centre (seed = ``index``)."""
    rng = np.random.Generator(np.random.PCG64(10_000 + index))
    nn = int(rng.integers(150, 501))
    n_dfn = int(rng.integers(50, 401))
    half = max(4, nn // 10)
    hf = []
    for c in (nn // 2 - 2, nn // 2 + 2):
        x = c * dx + dx / 2
        hf.append((x, (nn // 2 - half) * dx, x, (nn // 2 + half) * dx, 2 * half))
    wells = [(i, half, 1500.0 * PSI) for i in range(2)]
    return dfn_case(nn, nn, dx, n_dfn, index, hf=hf, wells=wells,
                    dts=geometric_schedule(n_steps, 30.0, dt_max_days=10.0), name=f"real{index}_{nn}x{nn}")


def batch(cases: Sequence[Case], name: str = "batch") -> Case:
    """Disjoint union of models that share the fluid and the timestep schedule: one graph whose
    connected components are the members, cell ranges in member order (member k starts at
    ``meta['offsets'][k]``).  A localized solve of the union advances every member at once."""
    if not cases:
        raise ValueError("empty batch")
    f0, dts = cases[0].fluid, cases[0].dt_schedule
    for c in cases[1:]:
        if c.fluid != f0:
            raise ValueError("batched models must share the fluid")
        if c.dt_schedule.shape != dts.shape or not np.array_equal(c.dt_schedule, dts):
            raise ValueError("batched models must share the timestep schedule")
    offs = np.cumsum([0] + [c.n for c in cases])
    adj = np.cumsum([0] + [c.row_ptr[-1] for c in cases])
    row_ptr = np.concatenate([cases[0].row_ptr[:1]] + [c.row_ptr[1:] + adj[k] for k, c in enumerate(cases)])
    nbr = np.concatenate([c.nbr + offs[k] for k, c in enumerate(cases)]).astype(np.int32)
    line_id, lbase = [], 0
    for c in cases:
        li = c.line_id.astype(np.int64)
        line_id.append(np.where(li >= 0, li + lbase, -1))
        lbase += int(li.max()) + 1 if (li >= 0).any() else 0
    cat = np.concatenate
    return Case(name=name, n=int(offs[-1]), row_ptr=row_ptr.astype(np.int32), nbr=nbr,
                trans=cat([c.trans for c in cases]), pv_ref=cat([c.pv_ref for c in cases]),
                depth=cat([c.depth for c in cases]), line_id=cat(line_id).astype(np.int32),
                always_active=cat([c.always_active for c in cases]).astype(np.uint8),
                well_cell=cat([c.well_cell + offs[k] for k, c in enumerate(cases)]).astype(np.int32),
                well_wi=cat([c.well_wi for c in cases]), well_bhp=cat([c.well_bhp for c in cases]),
                fluid=f0, p0=cat([c.p0 for c in cases]), sw0=cat([c.sw0 for c in cases]),
                dt_schedule=dts.copy(), n_matrix=int(sum(c.n_matrix for c in cases)),
                meta=dict(members=[c.name for c in cases], offsets=offs.tolist()))


def ensemble(n_real: int = 256, first: int = 0, **kw) -> Case:
    """The batched ensemble: realizations first .. first+n_real-1 as one union model."""
    return batch([realization(first + r, **kw) for r in range(n_real)], name=f"ensemble{n_real}")


def serving_model(index: int, cells: int, dx: float = 5.0) -> Case:
    """A resident model of about ``cells`` cells for the serving workload: an N x N matrix
    (N = round(sqrt(cells))) with N * 3/4 natural fractures and two hydraulic fractures on a
    producer at 1500 psi (seed = ``index``); its timestep sizes come with the requests."""
    nn = max(20, int(round(math.sqrt(cells))))
    half = max(3, nn // 10)
    hf = []
    for c in (nn // 2 - 2, nn // 2 + 2):
        x = c * dx + dx / 2
        hf.append((x, (nn // 2 - half) * dx, x, (nn // 2 + half) * dx, 2 * half))
    wells = [(i, half, 1500.0 * PSI) for i in range(2)]
    return dfn_case(nn, nn, dx, (3 * nn) // 4, 20_000 + index, hf=hf, wells=wells,
                    dts=np.array([DAY]), name=f"serve{index}_{nn}x{nn}")


# ---------------------------------------------------------------------------------------
# 3D: a layered matrix with vertical planar fractures (the large HBM-resident case)
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class _Panel:
    """A vertical planar fracture: horizontal trace (x0, y0)-(x1, y1) over layers [k0, k1)."""
    x0: float
    y0: float
    x1: float
    y1: float
    k0: int
    k1: int
    n_cells: int  # cells along the trace
    k_f: float
    w: float


def _add_matrix_3d(b: _Builder, nx: int, ny: int, nz: int, dx: float, dy: float, dz: float, perm: np.ndarray,
                   poro: float, top: float) -> np.ndarray:
    n = nx * ny * nz
    depth = top + (np.arange(nz) + 0.5) * dz
    ids = b.add_cells(np.full(n, dx * dy * dz * poro), np.repeat(depth, nx * ny))
    k = perm.reshape(nz, ny, nx)
    idx = ids.reshape(nz, ny, nx)
    for axis, area_over_d in ((2, dy * dz / dx), (1, dx * dz / dy), (0, dx * dy / dz)):
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[axis] = slice(None, -1)
        sl_b[axis] = slice(1, None)
        k1, k2 = k[tuple(sl_a)], k[tuple(sl_b)]
        b.connect(idx[tuple(sl_a)], idx[tuple(sl_b)], area_over_d * 2.0 * k1 * k2 / (k1 + k2))
    return ids


def _add_panels(b: _Builder, panels: Sequence[_Panel], nx: int, ny: int, dx: float, dy: float, dz: float,
                k_m: np.ndarray, top: float) -> List[np.ndarray]:
    """Each panel is a grid of pieces (along the trace x layers).  Pieces are numbered column by
    column, so each vertical column of a panel is one fracture line (consecutive ids, the strongest
    coupling when L > dz); pieces connect to the piece above and below, to the neighbouring column
    in the same layer, and to the matrix cell holding their centre.  Panels that cross do not
    exchange flow directly (they meet through the matrix).  Returns ids[layer, piece] per panel."""
    d_avg = (dx + dy) / 8.0
    out = []
    for s in panels:
        L = math.hypot(s.x1 - s.x0, s.y1 - s.y0) / s.n_cells
        nl = s.k1 - s.k0
        tmid = (np.arange(s.n_cells) + 0.5) / s.n_cells
        ix = np.clip(np.floor((s.x0 + tmid * (s.x1 - s.x0)) / dx).astype(np.int64), 0, nx - 1)
        iy = np.clip(np.floor((s.y0 + tmid * (s.y1 - s.y0)) / dy).astype(np.int64), 0, ny - 1)
        cols = []
        for a in range(s.n_cells):
            line = b.n_lines
            b.n_lines += 1
            ids = b.add_cells(np.full(nl, L * s.w * dz), top + (np.arange(s.k0, s.k1) + 0.5) * dz, line=line)
            if nl > 1:
                b.connect(ids[:-1], ids[1:], s.k_f * s.w * L / dz)
            mcell = (np.arange(s.k0, s.k1) * ny + iy[a]) * nx + ix[a]
            b.connect(ids, mcell, 2.0 * L * dz * k_m[mcell] / d_avg)
            if cols:
                b.connect(cols[-1], ids, s.k_f * s.w * dz / L)
            cols.append(ids)
        out.append(np.stack(cols, axis=1))  # [layer, piece]
    return out


def dfn3d_case(nx: int, ny: int, nz: int, dx: float, dz: float, n_nf: int, seed: int, *,
               hf: Sequence[Tuple[float, float, float, int, int, int]] = (),
               wells: Sequence[Tuple[int, int, int, float]] = (), k_mean_md: float = 1e-4, k_sigma: float = 0.5,
               poro: float = 0.06, hf_k_md: float = 1e4, hf_w: float = 0.01, nf_k_md: float = 1e3,
               nf_w: float = 0.001, nf_len: Tuple[float, float] = (20.0, 200.0), nf_layers: Tuple[int, int] = (2, 10),
               strikes: Tuple[Tuple[float, float], ...] = ((30.0, 10.0), (120.0, 10.0)), top: float = 2500.0,
               p_top: float = 5000.0 * PSI, sw_init: float = 0.25, dts: Optional[np.ndarray] = None,
               name: str = "dfn3d") -> Case:
    """nx x ny x nz matrix of dx x dx x dz cells (depth grows with the layer index), hydraulic
    fractures ``hf`` = (x, y0, y1, k0, k1, n_cells) as vertical planes at constant x, and ``n_nf``
    seeded natural fractures as vertical panels over U(nf_layers) layers; ``wells`` lists
    (hf index, piece along the trace, layer offset, BHP) producers.  The initial pressure follows
    the oil gradient from p_top at the top (near equilibrium with the dominant phase)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = Fluid(p_ref=p_top)
    b = _Builder()
    perm = _lognormal_perm(rng, nx * ny * nz, k_mean_md, k_sigma)
    _add_matrix_3d(b, nx, ny, nz, dx, dx, dz, perm, poro, top)
    n_matrix = b.n
    Lx, Ly = nx * dx, ny * dx
    panels = [_Panel(x, y0, x, y1, k0, k1, nc, hf_k_md * MD, hf_w) for (x, y0, y1, k0, k1, nc) in hf]
    for s_i in range(n_nf):
        mean, half = strikes[s_i % len(strikes)]
        ang = math.radians(mean + rng.uniform(-half, half))
        L = rng.uniform(*nf_len)
        cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
        ux, uy = math.cos(ang) * L / 2, math.sin(ang) * L / 2
        x0 = min(max(cx - ux, 1e-6), Lx - 1e-6)
        x1 = min(max(cx + ux, 1e-6), Lx - 1e-6)
        y0 = min(max(cy - uy, 1e-6), Ly - 1e-6)
        y1 = min(max(cy + uy, 1e-6), Ly - 1e-6)
        length = math.hypot(x1 - x0, y1 - y0)
        if length < 0.5 * dx:
            continue
        hgt = int(rng.integers(nf_layers[0], nf_layers[1] + 1))
        k0 = int(rng.integers(0, max(1, nz - hgt + 1)))
        panels.append(_Panel(x0, y0, x1, y1, k0, min(nz, k0 + hgt), max(1, int(round(length / dx))),
                             nf_k_md * MD, nf_w))
    ids = _add_panels(b, panels, nx, ny, dx, dx, dz, perm, top)
    for (h, piece, layer, bhp) in wells:
        s = panels[h]
        b.wells.append((int(ids[h][layer, piece]), _peaceman_wi(s.k_f, s.w, dz, dx), bhp))
    dts = dts if dts is not None else geometric_schedule(20, 180.0)
    case = _finish(b, name, fluid, p_top, sw_init, dts, n_matrix,
                   dict(nx=nx, ny=ny, nz=nz, dx=dx, dz=dz, n_panels=len(panels), n_hf=len(hf)))
    case.p0 = p_top + fluid.rho_o_ref * GRAVITY * (case.depth - top)
    return case


def config2(seed: int = 2) -> Case:
    """200 x 200 x 20 matrix of 5 x 5 x 2 m cells, 10 hydraulic-fracture stages (planes of 40 x 12
    cells) on a horizontal producer at 1500 psi along x through the centre, and 2000 natural
    fractures as vertical panels; oil-water (the black-oil variant of this geometry is not built)."""
    nx = ny = 200
    nz, dx, dz = 20, 5.0, 2.0
    yc = ny * dx / 2
    hf = []
    for s in range(10):
        x = (30 + 15 * s) * dx + dx / 2
        hf.append((x, yc - 20 * dx, yc + 20 * dx, 4, 16, 40))
    wells = [(s, 20, 6, 1500.0 * PSI) for s in range(10)]
    return dfn3d_case(nx, ny, nz, dx, dz, 2000, seed, hf=hf, wells=wells, name="config2_200x200x20_dfn2000_oilwater")


def small_dfn3d(nx: int = 10, ny: int = 8, nz: int = 3, n_nf: int = 3, seed: int = 5, n_steps: int = 5) -> Case:
    """A few-hundred-cell 3D model (one hydraulic fracture with a producer, a few panels) for tests."""
    dx, dz = 5.0, 2.0
    hf = [((nx // 2) * dx + dx / 2, 1.0 * dx, (ny - 1) * dx, 0, nz, ny - 2)]
    return dfn3d_case(nx, ny, nz, dx, dz, n_nf, seed, hf=hf, wells=[(0, (ny - 2) // 2, nz // 2, 1500.0 * PSI)],
                      nf_len=(3 * dx, 6 * dx), nf_layers=(1, nz), dts=doubling_schedule(n_steps),
                      name=f"small3d_{nx}x{ny}x{nz}")


def serving_model_3d(index: int, cells: int, dx: float = 5.0, dz: float = 2.0, nz: int = 10) -> Case:
    """A 3D resident model of about ``cells`` cells for the serving workload, built like the
    200x200x20 case: an N x N x nz layered matrix (N = round(sqrt(cells / nz))), two hydraulic-
    fracture stages (vertical planes over the middle layers) with a producer at 1500 psi in each,
    and N / 2 natural-fracture panels (seed = ``index``)."""
    nn = max(12, int(round(math.sqrt(cells / nz))))
    yc = nn * dx / 2
    half = max(3, nn // 8)
    k0, k1 = nz // 4, nz - nz // 4
    hf = [((nn // 2 + o) * dx + dx / 2, yc - half * dx, yc + half * dx, k0, k1, 2 * half) for o in (-3, 3)]
    wells = [(s, half, (k1 - k0) // 2, 1500.0 * PSI) for s in range(2)]
    return dfn3d_case(nn, nn, nz, dx, dz, max(4, nn // 2), 30_000 + index, hf=hf, wells=wells,
                      nf_layers=(2, max(2, nz - 2)), dts=np.array([DAY]), name=f"serve3d{index}_{nn}x{nn}x{nz}")



# ---------------------------------------------------------------------------------------
# Three-phase black-oil inputs (the 3D workload's physics: gas liberation below a bubble
# point, primary variables switched between p/Sw/Sg and p/Sw/Rs)
# ---------------------------------------------------------------------------------------
SCF_PER_STB = 0.028316846592 / 0.158987294928  # m^3 of gas per m^3 of oil, per scf/stb


@dataclasses.dataclass
class BlackOilFluid:
    """Black-oil fluid and rock constants (SI; gas-oil ratios in surface m^3 per surface m^3).

    Water as in ``Fluid``; oil b_o(p, Rs) = b_o_ref (1 + c_o (p - p_ref)) / (1 + kappa Rs) with
    density b_o (rho_o_sc + Rs rho_g_sc); gas b_g(p) = b_g_per_pa p (ideal gas at constant z and
    temperature) with density rho_g_sc b_g; saturated solution gas-oil ratio
    Rs_sat(p) = rs_max p / p_bubble (linear, rs_max at the bubble point); rock
    phi(p) = phi_ref (1 + c_r (p - p_ref)).  Relative permeabilities: Corey in the normalised
    saturations (Sw - swc) / span, (So - sor) / span and Sg / span, span = 1 - swc - sor.
    """

    p_ref: float = 5500.0 * PSI
    c_r: float = 1.0e-6 / PSI
    b_w_ref: float = 1.0
    c_w: float = 3.0e-6 / PSI
    rho_w_sc: float = 1000.0
    mu_w: float = 0.5 * CP
    b_o_ref: float = 1.0
    c_o: float = 1.0e-5 / PSI
    kappa: float = 0.4 / (800.0 * SCF_PER_STB)  # b_o(p_ref, rs_max) = 1 / 1.4
    rho_o_sc: float = 800.0
    mu_o: float = 1.0 * CP
    b_g_per_pa: float = 288.7 / (101325.0 * 0.9 * 350.0)  # T_sc / (p_sc z T)
    rho_g_sc: float = 0.9
    mu_g: float = 0.02 * CP
    rs_max: float = 800.0 * SCF_PER_STB
    p_bubble: float = 3500.0 * PSI
    swc: float = 0.2
    sor: float = 0.2
    n_w: int = 2
    n_o: int = 2
    n_g: int = 2
    gravity: float = GRAVITY


@dataclasses.dataclass
class BlackOilCase:
    """A model (``case``: graph, pore volumes, depths, wells, schedule; its oil-water ``fluid`` is not
    used) with black-oil constants and an initial state: p0, sw0, and per cell either free gas
    (sat0 = 1, sg0 >= 0, rs0 = Rs_sat(p0)) or none (sat0 = 0, sg0 = 0, rs0 <= Rs_sat(p0))."""

    case: Case
    fluid: BlackOilFluid
    p0: np.ndarray
    sw0: np.ndarray
    sg0: np.ndarray
    rs0: np.ndarray
    sat0: np.ndarray  # uint8

    @property
    def n(self) -> int:
        return self.case.n


def blackoil(case: Case, fluid: Optional[BlackOilFluid] = None, *, p_init: float = 5500.0 * PSI,
             bhp: Optional[float] = 2000.0 * PSI, rs_init: Optional[float] = None, sw_init: Optional[float] = None,
             rho_init: float = 640.0) -> BlackOilCase:
    """The black-oil version of a model: undersaturated oil (Rs = rs_init, default the fluid's
    rs_max, i.e. the bubble point at p_bubble) at p_init at the shallowest cell, increasing with depth
    at rho_init g (about the live oil's density), producers at ``bhp`` (None: the model's own)."""
    fl = fluid or BlackOilFluid()
    c = dataclasses.replace(case)
    if bhp is not None:
        c.well_bhp = np.full_like(case.well_bhp, bhp)
    n = case.n
    p0 = p_init + rho_init * fl.gravity * (case.depth - case.depth.min())
    rs = fl.rs_max if rs_init is None else rs_init
    sw0 = np.array(case.sw0, dtype=np.float64) if sw_init is None else np.full(n, sw_init)
    return BlackOilCase(case=c, fluid=fl, p0=p0, sw0=sw0, sg0=np.zeros(n), rs0=np.full(n, rs),
                        sat0=np.zeros(n, np.uint8))


def config2_blackoil(seed: int = 2) -> BlackOilCase:
    """The 3D workload with its black-oil physics: the config-2 geometry (200 x 200 x 20 + 10 hydraulic
    fractures + 2000 natural fractures), 5500 psi initially, producers at 2000 psi, bubble point
    3500 psi, Rs up to 800 scf/stb."""
    return blackoil(config2(seed))


def small_blackoil3d(nx: int = 10, ny: int = 8, nz: int = 3, seed: int = 5, n_steps: int = 5) -> BlackOilCase:
    """A few-hundred-cell 3D black-oil model for tests (the producer draws the fracture below the
    bubble point within the first steps)."""
    return blackoil(small_dfn3d(nx, ny, nz, seed=seed, n_steps=n_steps), p_init=3700.0 * PSI, bhp=2000.0 * PSI)
