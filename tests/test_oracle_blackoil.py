"""Pins of the black-oil oracle (oracle/blackoil.py) against facts that do not come from its own code.

* Without free gas and at one uniform Rs, the model is the oil-water model with a live-oil
  formation factor and density: its oil and water equations and their (p, Sw) derivatives equal
  the C oil-water oracle's (written independently) with b_o_ref = b_o_ref / (1 + kappa Rs) and
  rho_o_ref = rho_o_sc + Rs rho_g_sc, and its gas equation is Rs times its oil equation.
* The Jacobian (forward-mode) equals central differences of the residual in mixed states.
* Over a closed model with no accumulation, the fluxes of every component sum to zero.
* A closed cell has one state for its masses: Newton started on the other side of the bubble point
  comes back to it, through the switch the paper's Section 3.1 describes (phase disappearance or
  appearance).
* A single producing cell depletes at a fixed gas-oil ratio Rs while no free gas forms (the gas it
  produces is the gas dissolved in the oil it produces), and gas appears exactly when p falls below
  the bubble point of that Rs, p_bubble Rs / rs_max (Rs linear in p up to rs_max at the bubble point).
* Newton's method with the exact Jacobian converges quadratically.
Planted mistakes (test_blackoil_mutants_fail_a_pin) each fail one of these.
"""
import dataclasses
import sys
import types

import numpy as np
import pytest

import oracle as O
from oracle import blackoil as B
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    O.build()


def _rs_sat(fl, p):
    # the workload's definition: Rs linear in p, rs_max at the bubble point
    return fl.rs_max * np.asarray(p) / fl.p_bubble


def _model(wells=True):
    bo = cg.blackoil(cg.small_dfn3d(12, 10, 4, seed=9), p_init=3800.0 * PSI, bhp=2000.0 * PSI)
    if not wells:
        c = dataclasses.replace(bo.case, well_cell=np.zeros(0, np.int32), well_wi=np.zeros(0), well_bhp=np.zeros(0))
        bo = dataclasses.replace(bo, case=c)
    return bo


def _pressure(bo, base_psi, seed, noise=5e3):
    rng = np.random.default_rng(seed)
    z = bo.case.depth - bo.case.depth.min()
    return base_psi * PSI + 700.0 * cg.GRAVITY * z + rng.normal(0.0, noise, bo.n)


def _mixed_state(B_, bo, seed, frac_sat=0.5):
    rng = np.random.default_rng(seed + 1000)
    n, fl = bo.n, bo.fluid
    p = _pressure(bo, 3000.0, seed)
    sw = rng.uniform(0.25, 0.5, n)
    sat = (rng.random(n) < frac_sat).astype(np.uint8)
    sg = np.where(sat == 1, rng.uniform(0.02, 0.2, n), 0.0)
    rs = np.where(sat == 1, _rs_sat(fl, p), rng.uniform(0.5, 0.9, n) * _rs_sat(fl, p))
    return B_.State(p, sw, sg, rs, sat)


def _undersaturated(B_, bo, seed, rs0):
    rng = np.random.default_rng(seed + 2000)
    n = bo.n
    return B_.State(_pressure(bo, 4000.0, seed), rng.uniform(0.25, 0.6, n), np.zeros(n), np.full(n, rs0),
                    np.zeros(n, np.uint8))


# ---------------------------------------------------------------------------------------
# pins (each takes the oracle module, so that planted mistakes can be run through them)
# ---------------------------------------------------------------------------------------
def pin_oil_water_reduction(B_):
    bo = _model()
    fl = bo.fluid
    rs0 = 0.6 * fl.rs_max
    st, old = _undersaturated(B_, bo, 1, rs0), _undersaturated(B_, bo, 2, rs0)
    dt = 3.0 * cg.DAY
    F, Jd, Jo = B_.assemble(bo, st, old, dt)
    ow = cg.Fluid(p_ref=fl.p_ref, c_r=fl.c_r, b_o_ref=fl.b_o_ref / (1.0 + fl.kappa * rs0), c_o=fl.c_o,
                  b_w_ref=fl.b_w_ref, c_w=fl.c_w, rho_o_ref=fl.rho_o_sc + fl.rho_g_sc * rs0,
                  rho_w_ref=fl.rho_w_sc, mu_o=fl.mu_o, mu_w=fl.mu_w, swc=fl.swc, sor=fl.sor, n_w=fl.n_w,
                  n_o=fl.n_o, gravity=fl.gravity)
    m = O.Model(dataclasses.replace(bo.case, fluid=ow))
    Fo, Jdo, Joo = O.assemble(m, st.p, st.sw, old.p, old.sw, dt)
    for r in range(2):
        scale = np.max(np.abs(Fo[:, r]))
        assert np.max(np.abs(F[:, r] - Fo[:, r])) <= 1e-11 * scale, r
    assert np.max(np.abs(F[:, 2] - rs0 * F[:, 0])) <= 1e-11 * np.max(np.abs(rs0 * F[:, 0]))
    for J, Jw in ((Jd, Jdo), (Jo, Joo)):
        for r in range(2):
            for c in range(2):
                s = np.max(np.abs(Jw[:, r, c])) + 1e-300
                assert np.max(np.abs(J[:, r, c] - Jw[:, r, c])) <= 1e-10 * s, (r, c)
        s = np.max(np.abs(rs0 * Jw[:, 0, :2])) + 1e-300
        assert np.max(np.abs(J[:, 2, :2] - rs0 * Jw[:, 0, :2])) <= 1e-10 * s


def pin_central_differences(B_):
    bo = _model()
    st, old = _mixed_state(B_, bo, 3), _mixed_state(B_, bo, 4)
    old.sat[:] = st.sat
    dt = 2.0 * cg.DAY
    F, Jd, Jo = B_.assemble(bo, st, old, dt)
    c = bo.case
    rows = np.repeat(np.arange(bo.n), np.diff(c.row_ptr))
    cells = np.random.default_rng(5).choice(bo.n, 30, replace=False)
    for k in cells:
        for a in range(3):
            h = 1e-7 * st.p[k] if a == 0 else 1e-7
            cols = []
            for sgn in (1.0, -1.0):
                s2 = st.copy()
                if a == 0:
                    s2.p[k] += sgn * h
                    if s2.sat[k] == 1:
                        s2.rs[k] = _rs_sat(bo.fluid, s2.p[k])
                elif a == 1:
                    s2.sw[k] += sgn * h
                elif s2.sat[k] == 1:
                    s2.sg[k] += sgn * h
                else:
                    s2.rs[k] += sgn * h * bo.fluid.rs_max
                cols.append(B_.residual(bo, s2, old, dt))
            fd = (cols[0] - cols[1]) / (2.0 * h)
            if a == 2 and st.sat[k] == 0:
                fd = fd / bo.fluid.rs_max
            an = np.zeros_like(fd)
            an[k] = Jd[k][:, a]
            for e in np.flatnonzero(c.nbr == k):
                an[rows[e]] = Jo[e][:, a]
            scale = np.max(np.abs(an)) + 1e-300
            assert np.max(np.abs(fd - an)) <= 1e-5 * scale, (k, a, np.max(np.abs(fd - an)) / scale)


def pin_closed_conservation(B_):
    bo = _model(wells=False)
    st = _mixed_state(B_, bo, 6)
    F, _, _ = B_.assemble(bo, st, st.copy(), 1.0 * cg.DAY)
    for r in range(3):
        assert abs(F[:, r].sum()) <= 1e-11 * np.abs(F[:, r]).sum(), r


def _one_cell(B_, p, sw, sg, rs, sat, wells=()):
    b = cg._Builder()
    b.add_cells(np.array([50.0]), np.array([2500.0]))
    for bhp, wi in wells:
        b.wells.append((0, wi, bhp))
    case = cg._finish(b, "one_cell", cg.Fluid(), p, sw, np.array([cg.DAY]), 1, {})
    bo = cg.BlackOilCase(case=case, fluid=cg.BlackOilFluid(), p0=np.array([p]), sw0=np.array([sw]),
                         sg0=np.array([sg]), rs0=np.array([rs]), sat0=np.array([sat], np.uint8))
    return bo


def _newton(B_, bo, st, old, dt, iters=40):
    switches = 0
    for _ in range(iters):
        du, cmax, dmax = B_.local_solve(bo, st, old, dt, np.ones(bo.n, np.uint8), 0.2)
        st, sw = B_.apply_update(bo.fluid, st, du, np.ones(bo.n, np.uint8))
        switches += int(sw.sum())
        if dmax < 1e-6 and cmax < 1e-13 and not sw.any():
            return st, switches
    raise AssertionError("Newton did not converge")


def pin_closed_cell_switches(B_):
    fl = cg.BlackOilFluid()
    # old state without free gas (bubble point 0.9 p_bubble); start with gas at a lower pressure
    rs_o = 0.9 * fl.rs_max
    bo = _one_cell(B_, 3600.0 * PSI, 0.3, 0.0, rs_o, 0)
    old = B_.initial_state(bo)
    guess = B_.State(np.array([3000.0 * PSI]), np.array([0.3]), np.array([0.05]),
                     np.array([_rs_sat(fl, 3000.0 * PSI)]), np.array([1], np.uint8))
    st, n_sw = _newton(B_, bo, guess, old, cg.DAY)
    assert n_sw >= 1 and st.sat[0] == 0
    assert abs(st.p[0] - old.p[0]) <= 1e-9 * old.p[0] and abs(st.sw[0] - 0.3) <= 1e-12
    assert abs(st.rs[0] - rs_o) <= 1e-9 * rs_o
    # old state with free gas; start without it at a higher pressure and less dissolved gas
    p_o = 3000.0 * PSI
    bo = _one_cell(B_, p_o, 0.3, 0.1, _rs_sat(fl, p_o), 1)
    old = B_.initial_state(bo)
    guess = B_.State(np.array([3600.0 * PSI]), np.array([0.3]), np.array([0.0]), np.array([0.5 * fl.rs_max]),
                     np.array([0], np.uint8))
    st, n_sw = _newton(B_, bo, guess, old, cg.DAY)
    assert n_sw >= 1 and st.sat[0] == 1
    assert abs(st.p[0] - p_o) <= 1e-9 * p_o and abs(st.sg[0] - 0.1) <= 1e-9


def pin_depletion_bubble_point(B_):
    fl = cg.BlackOilFluid()
    rs_o = 0.9 * fl.rs_max
    p_b = fl.p_bubble * rs_o / fl.rs_max
    bo = _one_cell(B_, 3600.0 * PSI, 0.3, 0.0, rs_o, 0, wells=[(2000.0 * PSI, 2e-17)])
    sim = B_.Sim(bo, B_.Options(mode=0, tol_dp=1e-3, tol_cnv=1e-12, max_newton=60))
    seen_above = seen_below = False
    for k in range(40):
        before = sim.st.copy()
        st = sim.timestep(0.5 * cg.DAY * 1.25 ** k)
        assert st["status"] == 0
        s = sim.st
        if s.p[0] > p_b * (1.0 + 1e-9):
            seen_above = True
            assert s.sat[0] == 0 and abs(s.rs[0] - rs_o) <= 1e-9 * rs_o  # gas leaves with the oil
        elif s.p[0] < p_b * (1.0 - 1e-9):
            seen_below = True
            assert s.sat[0] == 1 and s.sg[0] > 0.0
            assert abs(s.rs[0] - _rs_sat(fl, s.p[0])) <= 1e-9 * rs_o
        if before.p[0] > p_b and s.p[0] < p_b:
            assert s.sat[0] == 1
    assert seen_above and seen_below


def pin_quadratic_convergence(B_):
    # a 1D producing chain without gravity: every face carries flow, so the residual is smooth
    # (no upwind direction flips) around the solution and Newton's error squares per step
    fl = dataclasses.replace(cg.BlackOilFluid(), gravity=0.0)
    chain = cg.chain_1d(12, 10.0, 1e-13, 0.1, 10.0, p_init=3800.0 * PSI, p_well=2000.0 * PSI, fluid=cg.Fluid(),
                        dts=np.array([cg.DAY]), wi=1e-12)
    bo = cg.blackoil(chain, fl, p_init=3800.0 * PSI, bhp=2000.0 * PSI, sw_init=0.25)
    sim = B_.Sim(bo, B_.Options(mode=0, tol_dp=1e-3, tol_cnv=1e-11))
    dt = 5.0 * cg.DAY
    old = sim.st.copy()
    assert sim.timestep(dt)["status"] == 0
    star = sim.st
    noise = np.random.default_rng(8).standard_normal(bo.n)
    errs = []
    for delta in (800.0, 400.0):
        st = star.copy()
        st.p = st.p + delta * noise
        du, _, _ = B_.local_solve(bo, st, old, dt, np.ones(bo.n, np.uint8), 0.0)
        new, sw = B_.apply_update(bo.fluid, st, du, np.ones(bo.n, np.uint8))
        assert not sw.any()
        errs.append(np.max(np.abs(new.p - star.p)))
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, (errs, ratio)


PINS = [pin_oil_water_reduction, pin_central_differences, pin_closed_conservation, pin_closed_cell_switches,
        pin_depletion_bubble_point, pin_quadratic_convergence]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_blackoil_pin(pin):
    pin(B)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_local_modes_match_standard_newton_on_3d_model(mode):
    """Algorithm 1, Algorithm 2 and the residual-based sets on the black-oil model reach the fields of
    standard Newton within one pressure cutoff (the methods drop updates below eps_p outside their
    sets), with the same cells holding free gas (gas appears near the producer) and fewer cell
    updates."""
    bo = cg.small_blackoil3d()
    tight = dict(tol_dp=1.0, tol_cnv=1e-10)
    a = B.Sim(bo, B.Options(mode=0, **tight))
    b = B.Sim(bo, B.Options(mode=mode, **tight))
    ua = ub = 0
    for dt in bo.case.dt_schedule:
        sa, sb = a.timestep(dt), b.timestep(dt)
        assert sa["status"] == 0 and sb["status"] == 0
        ua += sa["cell_updates"]
        ub += sb["cell_updates"]
        if mode == 2:
            assert sb["n_subdomains"] >= 1 and sb["dd_outer"] >= 1
    assert a.st.sat.sum() > 0 and np.array_equal(a.st.sat, b.st.sat)
    assert np.max(np.abs(a.st.p - b.st.p)) < B.Options().eps_p
    assert np.max(np.abs(a.st.sg - b.st.sg)) < 1e-3 and np.max(np.abs(a.st.sw - b.st.sw)) < 1e-3
    assert ub < ua


# ---------------------------------------------------------------------------------------
# planted mistakes: each must fail at least one pin
# ---------------------------------------------------------------------------------------
MUTANTS = {
    "dissolved gas flux dropped": ('f = flux[comp] if comp != "g" else flux["g"] + flux["dg"]',
                                   'f = flux[comp] if comp != "g" else flux["g"]'),
    "dissolved gas upwinded with the free gas": ("where(up_oil, rmi, rmj)", "where(up, rmi, rmj)"),
    "producer's dissolved gas dropped": ('g=wi * q["mob_g"][j] * dpw + q["RS"][j] * qo',
                                         'g=wi * q["mob_g"][j] * dpw'),
    "dissolved gas missing from the gas mass": ('q["mass_g"] = PV * (BG * SG + RS * BO * SO)',
                                                'q["mass_g"] = PV * (BG * SG)'),
    "oil density without its dissolved gas": ('q["rho_o"] = BO * (fl.rho_o_sc + fl.rho_g_sc * RS)',
                                              'q["rho_o"] = BO * fl.rho_o_sc'),
    "row cell's density instead of the face mean": ("dphi = (Pi - Pj) - g * dz * (0.5 * (ri + rj))",
                                                    "dphi = (Pi - Pj) - g * dz * ri"),
    "quotient rule sign": ("(self.d * b.v[:, None] - b.d * self.v[:, None])",
                           "(self.d * b.v[:, None] + b.d * self.v[:, None])"),
    "gas appears on the wrong side of Rs_sat": ("split = u & (out.rs > rs_sat(fl, out.p))",
                                                "split = u & (out.rs < rs_sat(fl, out.p))"),
    "gas never disappears": ("gone = s & (out.sg < 0.0)", "gone = s & (out.sg < -1e300)"),
    "Rs_sat quadratic in p": ("return fl.rs_max * p / fl.p_bubble", "return fl.rs_max * p / fl.p_bubble * p / fl.p_bubble"),
}


def _mutant(name):
    old, new = MUTANTS[name]
    src = open(B.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle._blackoil_mutant")
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod  # the dataclasses in it look their module up
    try:
        exec(compile(src.replace(old, new), "blackoil_mutant.py", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


@pytest.mark.parametrize("name", list(MUTANTS))
def test_blackoil_mutants_fail_a_pin(name):
    mod = _mutant(name)
    failed = []
    for pin in PINS:
        try:
            pin(mod)
        except (AssertionError, ArithmeticError, FloatingPointError, ValueError) as e:
            failed.append((pin.__name__, type(e).__name__))
    assert failed, f"planted mistake '{name}' passes every pin"


def test_sampled_rows_equal_the_full_assembly():
    """assemble_cells on a subset of rows (any order) gives those rows of the full assembly, bit for
    bit, with the off-diagonal blocks of their CSR entries."""
    bo = _model()
    st, old = _mixed_state(B, bo, 7), _mixed_state(B, bo, 8)
    F, Jd, Jo = B.assemble(bo, st, old, 2.0 * cg.DAY)
    cells = np.random.default_rng(9).permutation(bo.n)[: bo.n // 3]
    cells = np.concatenate([cells, bo.case.well_cell.astype(np.int64)])
    cells = np.unique(cells)[::-1]
    Fs, Jds, Jos, e = B.assemble_cells(bo, st, old, 2.0 * cg.DAY, cells)
    assert np.array_equal(Fs, F[cells]) and np.array_equal(Jds, Jd[cells]) and np.array_equal(Jos, Jo[e])
    rp = bo.case.row_ptr
    assert np.array_equal(e, np.concatenate([np.arange(rp[i], rp[i + 1]) for i in cells]))

