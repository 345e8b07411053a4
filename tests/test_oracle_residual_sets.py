"""Pins of the oracle's residual-based active sets (mode 3: the Lu-Beckner estimate the paper
cites as the alternative a-priori strategy, Section 1 and Section 4.2): unconverged cells
(CNV_i >= tol_cnv on the full-domain residual) inflated by m layers of neighbours."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle as O
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI


def _adjacency(case):
    rows = np.repeat(np.arange(case.n), np.diff(case.row_ptr))
    return sp.csr_matrix((np.ones(case.n_adj), (rows, case.nbr)), shape=(case.n, case.n))


def test_first_set_is_unconverged_cells_within_m_hops():
    """The first solve of a step acts on the cells within m graph hops (scipy distances) of the
    cells whose scaled residual at u^n is not converged."""
    case = cg.small_dfn(n_steps=3)
    sim = O.Sim(case, O.Options(mode=1))
    sim.timestep(case.dt_schedule[0])  # some non-trivial state
    p, sw = sim.p.copy(), sim.sw.copy()
    dt = float(case.dt_schedule[1])
    for m in (1, 2):
        res = O.Sim(case, O.Options(mode=3, m_layers=m))
        res.p, res.sw = p.copy(), sw.copy()
        st = res.timestep(dt)
        assert st["status"] == 0 and st["iterations"] >= 1
        model = O.Model(case)
        F = O.residual(model, p, sw, p, sw, dt)
        unconv = O.cnv(model, p, F, dt) >= O.Options().tol_cnv
        assert unconv.any()
        d = csg.shortest_path(_adjacency(case), unweighted=True, indices=np.flatnonzero(unconv)).min(axis=0)
        assert st["trace"][0] == int(np.count_nonzero(d <= m))


def test_full_inflation_follows_standard_newton_iterates():
    """With m at least the graph diameter every solve covers V, so the iterates are standard
    Newton's, bit for bit, for as many iterations as the residual-based loop runs."""
    case = cg.small_dfn(n_steps=3)
    for dt in case.dt_schedule[:2]:
        res = O.Sim(case, O.Options(mode=3, m_layers=10_000))
        st = res.timestep(dt)
        assert st["status"] == 0 and all(t == case.n for t in st["trace"])
        full = O.Sim(case, O.Options(mode=0, max_newton=st["iterations"]))
        full.timestep(dt)
        assert np.array_equal(full.p, res.p) and np.array_equal(full.sw, res.sw)


def test_equilibrium_takes_no_iteration():
    case = cg.grid_2d(6, 5, with_well=False)
    sim = O.Sim(case, O.Options(mode=3, m_layers=1))
    st = sim.timestep(case.dt_schedule[0])
    assert st["status"] == 0 and st["iterations"] == 0
    assert np.array_equal(sim.p, case.p0) and np.array_equal(sim.sw, case.sw0)


def test_matches_standard_newton_config0():
    """Both converge to the discrete solution: fields within the Newton tolerance, with the
    solves localized (average active fraction well below one)."""
    case = cg.config0()
    full = O.Sim(case, O.Options(mode=0))
    res = O.Sim(case, O.Options(mode=3, m_layers=1))
    s0 = full.run(case.dt_schedule)
    s3 = res.run(case.dt_schedule)
    assert all(s["status"] == 0 for s in s0 + s3)
    assert np.abs(res.p - full.p).max() < 0.3 * PSI
    assert np.abs(res.sw - full.sw).max() < 1e-6
    assert sum(s["cell_updates"] for s in s3) / case.n < 0.5 * sum(s["iterations"] for s in s0)


# ---------------------------------------------------------------------------------------
# The oracle's time-step controller (cut on failure, grow after easy steps)
# ---------------------------------------------------------------------------------------
def test_controller_single_step_equals_plain_timestep():
    case = cg.config0()
    dt = float(case.dt_schedule[3])
    a = O.Sim(case, O.Options(mode=1))
    out = a.advance(dt, dt_init=dt, dt_min=dt / 64, dt_max=dt)
    b = O.Sim(case, O.Options(mode=1))
    st = b.timestep(dt)
    assert out["status"] == 0 and out["steps"] == 1 and out["cuts"] == 0 and out["iterations"] == st["iterations"]
    assert np.array_equal(a.p, b.p) and np.array_equal(a.sw, b.sw)


def test_controller_cuts_then_matches_the_same_steps_taken_plainly():
    """With a small Newton limit a long step fails and is cut; the accepted steps, replayed as
    plain timesteps from the same start, give the same state bit for bit (the undo is exact)."""
    case = cg.config0()
    o = O.Options(mode=1, max_newton=5)
    span = 30.0 * 86400.0
    a = O.Sim(case, o)
    out = a.advance(span, dt_init=span, dt_min=span / 4096, dt_max=span)
    assert out["status"] == 0 and out["cuts"] >= 1 and abs(sum(out["dts"]) - span) <= 1e-6 * span
    b = O.Sim(case, o)
    for h in out["dts"]:
        assert b.timestep(h)["status"] == 0
    assert np.array_equal(a.p, b.p) and np.array_equal(a.sw, b.sw)


def test_controller_gives_up_below_dt_min_with_the_state_unchanged():
    case = cg.config0()
    a = O.Sim(case, O.Options(mode=1, max_newton=1))
    span = 365.0 * 86400.0
    out = a.advance(span, dt_init=span, dt_min=span / 8, dt_max=span)
    assert out["status"] == -4 and out["steps"] == 0 and out["cuts"] >= 3
    assert np.array_equal(a.p, case.p0) and np.array_equal(a.sw, case.sw0)
