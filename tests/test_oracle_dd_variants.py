"""Pins of the oracle's Algorithm 2 variants (a subdomain visit solved to local convergence, and
localization inside a subdomain) to standard Newton and to invariants of the definitions.

- One subdomain covering the whole model (m larger than the graph's diameter) and visits solved to
  convergence: the first visit is standard Newton step for step, so each timestep takes standard
  Newton's iterations plus the one Schwarz visit that finds the subdomain converged, every solve is
  the whole model, and the fields agree with standard Newton's within its pressure tolerance.
- With eps = 0 every update is "non-negligible", so the support of an update is the whole solved
  set and localization inside a subdomain changes nothing: bit-identical runs with and without it.
- Every variant converges to standard Newton's discrete solution within the Newton tolerance, and
  localization inside subdomains solves fewer cells than full subdomain visits.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI


def test_single_subdomain_visit_to_convergence_is_standard_newton():
    case = cg.small_dfn(n_steps=4)
    std = O.Sim(case, O.Options(mode=0))
    dd = O.Sim(case, O.Options(mode=2, m_layers=10_000, dd_local_newton=25))
    for dt in case.dt_schedule:
        dd.has_prev.value = 0  # initial set = always-active cells + m layers = the whole (connected) model
        a = std.timestep(dt)
        b = dd.timestep(dt)
        assert a["status"] == 0 and b["status"] == 0
        assert b["n_subdomains"] == 1
        assert b["iterations"] == a["iterations"] + 1, (a, b)
        assert b["trace"] == [case.n] * b["iterations"]
        assert np.max(np.abs(dd.p - std.p)) < O.Options().tol_dp
        assert np.max(np.abs(dd.sw - std.sw)) < 1e-6
        dd.p, dd.sw = std.p.copy(), std.sw.copy()  # next step from the same state


@pytest.mark.parametrize("local_newton", [2, 5])
def test_localization_inside_subdomains_is_void_at_zero_cutoff(local_newton):
    case = cg.small_dfn(n_steps=3)
    base = dict(mode=2, eps_p=0.0, dd_local_newton=local_newton)
    a = O.Sim(case, O.Options(**base, dd_local_shrink=0))
    b = O.Sim(case, O.Options(**base, dd_local_shrink=1))
    for dt in case.dt_schedule:
        sa = a.timestep(dt)
        sb = b.timestep(dt)
        assert (sa["status"], sa["iterations"], sa["cell_updates"]) == (sb["status"], sb["iterations"],
                                                                         sb["cell_updates"])
        assert np.array_equal(a.p, b.p) and np.array_equal(a.sw, b.sw)


def test_variants_reach_the_standard_newton_solution():
    case = cg.config0()
    std = O.Sim(case, O.Options(mode=0))
    std.run(case.dt_schedule)
    updates = {}
    for local_newton, shrink in ((1, 0), (4, 0), (4, 1)):
        sim = O.Sim(case, O.Options(mode=2, dd_local_newton=local_newton, dd_local_shrink=shrink))
        st = sim.run(case.dt_schedule)
        assert all(s["status"] == 0 for s in st)
        assert np.max(np.abs(sim.p - std.p)) < 0.3 * PSI
        assert np.max(np.abs(sim.sw - std.sw)) < 1e-6
        updates[(local_newton, shrink)] = sum(s["cell_updates"] for s in st)
    assert updates[(4, 1)] < updates[(4, 0)]
