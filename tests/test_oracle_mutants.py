"""Plant plausible mistakes in the oracle (on the CPU, in a private copy of its source) and
check that the pins catch each one: a dropped Sor in the Corey span, swapped viscosities, the
wrong Corey exponent or base, and in the scaled residual a missing dt, the other phase's b,
or the reference pore volume in place of PV(p).  The oracle's own build is untouched; each
mutant is compiled into a temporary directory and routed in with oracle.use_library."""
import numpy as np
import pytest

import oracle as O
from tests import test_oracle_two_phase_pins as P

MUTANTS = {
    "span_without_sor": ("double span = 1.0 - f->swc - f->sor;", "double span = 1.0 - f->swc;"),
    "viscosities_swapped": ("double mu[2] = {f->mu_o, f->mu_w};", "double mu[2] = {f->mu_w, f->mu_o};"),
    "water_exponent_from_oil": ("kr[1] = ipow(se, f->n_w);", "kr[1] = ipow(se, f->n_o);"),
    "oil_kr_of_se": ("kr[0] = ipow(1.0 - se, f->n_o);", "kr[0] = ipow(se, f->n_o);"),
    "cnv_without_dt": ("fabs(F[2 * (int64_t)i + 1]) * dt / (q.pv * q.b[1])",
                       "fabs(F[2 * (int64_t)i + 1]) / (q.pv * q.b[1])"),
    "cnv_water_scaled_by_oil_b": ("fabs(F[2 * (int64_t)i + 1]) * dt / (q.pv * q.b[1])",
                                  "fabs(F[2 * (int64_t)i + 1]) * dt / (q.pv * q.b[0])"),
    "cnv_reference_pore_volume": ("fabs(F[2 * (int64_t)i]) * dt / (q.pv * q.b[0])",
                                  "fabs(F[2 * (int64_t)i]) * dt / (m->pv_ref[i] * q.b[0])"),
}


def _pins():
    """Every pin of the two-phase terms and of CNV, as zero-argument calls."""
    calls = [lambda a=a: P.test_face_flux_is_corey_mobility_of_upstream_cell(*a) for a in P.COREY_POINTS]
    calls += [lambda a=a: P.test_corey_endpoints(*a) for a in [(2, 2), (3, 1), (1, 4)]]
    calls += [P.test_total_flux_is_saturation_independent_for_linear_corey, P.test_cnv_worked_example]
    calls += [lambda d=d, q=q: P.test_cnv_of_pure_accumulation_is_the_saturation_change(d, q)
              for d in (0.01, 1.0, 30.0) for q in (0.0, -1500.0, 800.0)]
    return calls


def _failures(calls):
    n = 0
    for c in calls:
        try:
            c()
        except AssertionError:
            n += 1
    return n


def test_pins_pass_on_the_oracle_as_built():
    assert _failures(_pins()) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = O.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    so = O.build_variant(src.replace(old, new), str(tmp_path), name)
    with O.use_library(so):
        failed = _failures(_pins())
    assert failed > 0, f"no pin caught the planted mistake {name}"
