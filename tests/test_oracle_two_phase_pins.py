"""Pins of the oracle's two-phase fluid terms at interior saturations, and of its scaled
residual (CNV), to values fixed by the definitions and by the mathematics -- not by the
oracle's own code.

- Corey (Appendix A reduced to oil-water): the flux of each phase across one face of a
  two-cell model with no accumulation, no well and no gravity is T kr_l(Se_up) / mu_l b_l dp,
  so with b_l = 1 the water/oil flux ratio is kr_w mu_o / (kr_o mu_w), the fractional-flow
  ratio.  Saturations are chosen so that Se is an exact binary fraction and the expected
  relative permeabilities are literal fractions (Se = 1/4 gives 1/16 and 9/16 at exponent 2).
- Endpoints and invariants: kr_w = 0 and kr_o = 1 at and below connate water, the reverse at
  and above 1 - Sor; with linear relative permeabilities and equal viscosities the total flux
  does not depend on the saturation; the downstream cell's saturation never matters.
- CNV: for a single cell whose state differs from its time level only in Sw by delta, the
  residual is pure accumulation, R_w = PV(p) b_w(p) delta / dt and R_o = -PV(p) b_o(p) delta / dt,
  so the scaled residual |R_l| dt / (PV(p) b_l(p)) equals |delta| for both phases, whatever dt,
  p, c_r or the phases' b.

Each test is chosen so that a mistake in the corresponding oracle term fails it; the planted
mistakes live in tests/test_oracle_mutants.py.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI
SWC, SOR = 0.2, 0.15          # span 1 - Swc - Sor = 0.65 (asymmetric: swapping Swc and Sor changes Se)
MU_O, MU_W = 2.0 * cg.CP, 0.5 * cg.CP


def _two_cells(n_w, n_o, mu_o=MU_O, mu_w=MU_W):
    fl = cg.Fluid(c_r=0.0, c_o=0.0, c_w=0.0, b_o_ref=1.0, b_w_ref=1.0, swc=SWC, sor=SOR,
                  mu_o=mu_o, mu_w=mu_w, n_w=n_w, n_o=n_o, gravity=0.0)
    case = cg.chain_1d(2, 5.0, 1.0 * cg.MD, 0.2, 1.0, p_init=fl.p_ref, p_well=0.0, fluid=fl,
                       dts=np.array([cg.DAY]), wi=0.0)
    return case, O.Model(case)


def _fluxes(m, p, sw):
    """Outflow of each phase from each cell: the residual with u = u^n (no accumulation) and a
    zero well index (no well term)."""
    return O.residual(m, p, sw, p, sw, cg.DAY)


# (Se, n_w, n_o, kr_w, kr_o) with the relative permeabilities written out as fractions.
COREY_POINTS = [
    (0.25, 2, 2, 1 / 16, 9 / 16),
    (0.5, 2, 2, 1 / 4, 1 / 4),
    (0.75, 2, 2, 9 / 16, 1 / 16),
    (0.25, 3, 1, 1 / 64, 3 / 4),
    (0.5, 1, 4, 1 / 2, 1 / 16),
    (0.75, 4, 3, 81 / 256, 1 / 64),
]


@pytest.mark.parametrize("se,n_w,n_o,kr_w,kr_o", COREY_POINTS)
def test_face_flux_is_corey_mobility_of_upstream_cell(se, n_w, n_o, kr_w, kr_o):
    case, m = _two_cells(n_w, n_o)
    T = case.trans[0]
    dp = 40.0 * PSI
    sw_up = SWC + (1.0 - SWC - SOR) * se
    for sw_down in (SWC, 0.5, 1.0 - SOR):   # the downstream saturation must not matter
        p = np.array([case.fluid.p_ref + dp, case.fluid.p_ref])
        F = _fluxes(m, p, np.array([sw_up, sw_down]))
        np.testing.assert_allclose(F[0, 0], T * kr_o / MU_O * dp, rtol=1e-12)
        np.testing.assert_allclose(F[0, 1], T * kr_w / MU_W * dp, rtol=1e-12)
        np.testing.assert_allclose(F[1], -F[0], rtol=0, atol=1e-12 * abs(F[0]).max())
        # fractional flow: water / oil flux ratio = kr_w mu_o / (kr_o mu_w)
        np.testing.assert_allclose(F[0, 1] / F[0, 0], (kr_w * MU_O) / (kr_o * MU_W), rtol=1e-12)
    # reversed pressure difference: the other cell is upstream
    p = np.array([case.fluid.p_ref, case.fluid.p_ref + dp])
    F = _fluxes(m, p, np.array([SWC, sw_up]))
    np.testing.assert_allclose(F[1, 0], T * kr_o / MU_O * dp, rtol=1e-12)
    np.testing.assert_allclose(F[1, 1], T * kr_w / MU_W * dp, rtol=1e-12)


@pytest.mark.parametrize("n_w,n_o", [(2, 2), (3, 1), (1, 4)])
def test_corey_endpoints(n_w, n_o):
    case, m = _two_cells(n_w, n_o)
    T = case.trans[0]
    dp = 25.0 * PSI
    p = np.array([case.fluid.p_ref + dp, case.fluid.p_ref])
    for sw in (SWC - 0.05, SWC):             # connate water and below: water immobile, kr_o = 1
        F = _fluxes(m, p, np.array([sw, 0.5]))
        assert abs(F[0, 1]) <= 1e-12 * F[0, 0]
        np.testing.assert_allclose(F[0, 0], T / MU_O * dp, rtol=1e-12)
    for sw in (1.0 - SOR, 1.0 - SOR + 0.05):  # residual oil and above: oil immobile, kr_w = 1
        F = _fluxes(m, p, np.array([sw, 0.5]))
        assert abs(F[0, 0]) <= 1e-12 * F[0, 1]   # (Sw - Swc) / span rounds to within 1 ulp of 1
        np.testing.assert_allclose(F[0, 1], T / MU_W * dp, rtol=1e-12)


def test_total_flux_is_saturation_independent_for_linear_corey():
    case, m = _two_cells(1, 1, mu_o=1.0 * cg.CP, mu_w=1.0 * cg.CP)
    T = case.trans[0]
    dp = 10.0 * PSI
    p = np.array([case.fluid.p_ref + dp, case.fluid.p_ref])
    for sw in np.linspace(SWC, 1.0 - SOR, 11):
        F = _fluxes(m, p, np.array([sw, SWC]))
        np.testing.assert_allclose(F[0].sum(), T / (1.0 * cg.CP) * dp, rtol=1e-12)


# ---------------------------------------------------------------------------------------
# CNV = max_l |R_l| dt / (PV(p) b_l(p)).
# ---------------------------------------------------------------------------------------
def _one_cell(c_r, b_o_ref, b_w_ref, c_o, c_w):
    fl = cg.Fluid(c_r=c_r, c_o=c_o, c_w=c_w, b_o_ref=b_o_ref, b_w_ref=b_w_ref, gravity=0.0)
    case = cg.chain_1d(1, 10.0, 1.0 * cg.MD, 0.1, 1.0, p_init=fl.p_ref, p_well=0.0, fluid=fl,
                       dts=np.array([cg.DAY]), wi=0.0)
    return case, O.Model(case)


@pytest.mark.parametrize("dt_days", [0.01, 1.0, 30.0])
@pytest.mark.parametrize("dp_psi", [0.0, -1500.0, 800.0])
def test_cnv_of_pure_accumulation_is_the_saturation_change(dt_days, dp_psi):
    case, m = _one_cell(c_r=3e-6 / PSI, b_o_ref=1.0, b_w_ref=0.8, c_o=2e-5 / PSI, c_w=4e-6 / PSI)
    dt = dt_days * cg.DAY
    p = np.array([case.fluid.p_ref + dp_psi * PSI])
    for delta in (1e-7, 3e-3, -0.02):
        swn = np.array([0.4])
        sw = swn + delta
        F = O.residual(m, p, sw, p, swn, dt)
        cnv = O.cnv(m, p, F, dt)
        np.testing.assert_allclose(cnv[0], abs(delta), rtol=1e-8)
        # each phase on its own: the water row scaled by b_w and the oil row by b_o give |delta|
        for phase in (0, 1):
            Fl = F.copy()
            Fl[0, 1 - phase] = 0.0
            np.testing.assert_allclose(O.cnv(m, p, Fl, dt)[0], abs(delta), rtol=1e-8)


def test_cnv_worked_example():
    # PV = 10 m3 and b = (1, 0.5) at p = p_ref; F = (2, 3) per second, dt = 5 s:
    # oil 2 * 5 / (10 * 1) = 1, water 3 * 5 / (10 * 0.5) = 3, CNV = 3
    case, m = _one_cell(c_r=1e-6 / PSI, b_o_ref=1.0, b_w_ref=0.5, c_o=1e-5 / PSI, c_w=1e-6 / PSI)
    case.pv_ref[:] = 10.0
    m = O.Model(case)
    p = np.array([case.fluid.p_ref])
    assert O.cnv(m, p, np.array([[2.0, 3.0]]), 5.0)[0] == 3.0
    assert O.cnv(m, p, np.array([[-4.0, 0.5]]), 5.0)[0] == 2.0
