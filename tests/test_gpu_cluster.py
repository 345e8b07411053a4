"""The two BiCGStab solvers of the local system J_A du_A = -F_A (Section 4.3) against the oracle's
sparse LU: the thread-block-cluster solver (systems up to its capacity; vectors in distributed
shared memory) and the cooperative grid solver (larger systems, or krylov_cluster = 0).

Sizes span one CTA's chunk, several chunks with ragged ends, and the 400x400 DFN model's sets of
~7k and ~13k rows (the benchmark's range), at every cluster size; both precisions, the
fracture-line preconditioner and the cell-block one.  The solver that ran is reported by the
library (lns_iter_stats.krylov_solver), so each test also checks the size test that picks it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu
PSI = cg.PSI
CLUSTER, GRID = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)
    O.build()


@pytest.fixture(scope="module")
def big():
    return cg.config1()


def _state(case, seed):
    p, sw = case.p0.copy(), case.sw0.copy()
    pn, swn = p.copy(), sw.copy()
    p = p - 30.0 * PSI * np.random.default_rng(seed).random(case.n)
    return p, sw, pn, swn


def _check(case, va, fp32, cluster, precond=lns.LNS_PRECOND_BJAC, expect=None, seed=0):
    om = O.Model(case)
    p, sw, pn, swn = _state(case, seed)
    dt = 2.0 * cg.DAY
    dpo, dso, _, _ = O.local_solve(om, O.Options(), p, sw, pn, swn, dt, va)
    def solve(cl):
        g = lns.Model(case, lns.Options(krylov_fp32=fp32, krylov_rtol=1e-6 if fp32 else 1e-12, krylov_maxit=5000,
                                        krylov_cluster=cl, precond=precond))
        g.lns_set_tuning(cluster_max_rows=-1)  # every system that fits goes to the cluster solver
        g.lns_set_state(p, sw, pn, swn)
        out = g.lns_solve_local(dt, va)
        g.close()
        return out

    dpg, dsg, st = solve(cluster)
    assert st["n_active"] == int(va.sum())
    if expect is not None:
        assert st["krylov_solver"] == expect, st
    # the oracle's tolerance of the local solve, or (ill-conditioned systems, where the Krylov stop
    # on the scaled residual leaves more) no worse than the grid solver on the same system
    tol = 2e-5 if fp32 else 1e-8
    if fp32 and precond == lns.LNS_PRECOND_BJAC_CELL:
        tol = 1e-3  # FP32 with 2x2 cell blocks only: the fracture lines' conditioning limits the error
    err_p = np.max(np.abs(dpg - dpo))
    err_s = np.max(np.abs(dsg - dso))
    lim_p = tol * np.max(np.abs(dpo)) + 1e-9
    lim_s = tol * max(np.max(np.abs(dso)), 1e-12) + 1e-12
    if (err_p > lim_p or err_s > lim_s) and st["krylov_solver"] == CLUSTER:
        dpr, dsr, sr = solve(0)
        assert sr["krylov_solver"] == GRID
        # BiCGStab's recurrence residual drifts from the true one differently with the reduction
        # order, so the two solvers' errors at the same stopping test differ by a small factor
        lim_p = max(lim_p, 10 * np.max(np.abs(dpr - dpo)))
        lim_s = max(lim_s, 10 * np.max(np.abs(dsr - dso)))
        assert err_p <= lim_p and err_s <= lim_s, (err_p, err_s, st, sr)
    assert err_p <= lim_p, (err_p, lim_p, st)
    assert err_s <= lim_s, (err_s, lim_s, st)
    assert np.all(dpg[va == 0] == 0.0)
    return st


def cluster_capacity(ctas, fp32, lines=True):
    """Rows the cluster solver takes: ctas x (rows per CTA - one line block of slack)."""
    return ctas * ((1024 if fp32 else 512) - (128 if lines else 0))


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_cluster_sizes_small_models(fp32, cluster):
    for case in (cg.small_dfn(), cg.config0(), cg.small_dfn3d()):
        om = O.Model(case)
        for va in (np.ones(case.n, np.uint8), O.dilate(om, case.always_active, 2)):
            n = int(va.sum())
            _check(case, va, fp32, cluster, expect=CLUSTER if n <= cluster_capacity(cluster, fp32) else GRID)


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("precond", [lns.LNS_PRECOND_BJAC, lns.LNS_PRECOND_BJAC_CELL])
def test_cluster_and_grid_agree_with_oracle_on_config1_sets(big, fp32, precond):
    """The always-active set of the 400x400 DFN model (6,659 fracture and well cells, the shrink-mode
    floor of every timestep): the cluster solver where it fits (FP32; FP64 with the cell-block
    preconditioner, whose chunks need no line slack), else the grid solver, and the grid solver when
    krylov_cluster = 0."""
    case = big
    va = case.always_active.astype(np.uint8)
    n = int(va.sum())
    assert 6000 < n < 9000
    fits = n <= cluster_capacity(16, fp32, lines=precond == lns.LNS_PRECOND_BJAC)
    _check(case, va, fp32, -1, precond=precond, expect=CLUSTER if fits else GRID, seed=1)
    _check(case, va, fp32, 0, precond=precond, expect=GRID, seed=1)


def test_grid_solver_on_3d_model_fp64():
    """The grid solver on a 3D model of more than five neighbours a cell (3,059 cells, 5.48 a cell;
    fracture cells of seven and eight) in FP64: the whole model and its fracture-support set against
    the oracle's sparse LU.  (Its FP32 solves, whose six-neighbour gathers this model selects, stop
    at the FP32 floor of these systems; they are checked through Newton timesteps against the
    oracle in test_gpu_parity.py.)"""
    case = cg.small_dfn3d(24, 20, 6)
    deg = np.diff(case.row_ptr)
    assert case.n_adj > 5 * case.n and deg.max() > 6
    om = O.Model(case)
    for va in (np.ones(case.n, np.uint8), O.dilate(om, case.always_active, 2)):
        _check(case, va, 0, 0, expect=GRID)


def test_cluster_capacity_boundary(big):
    """FP32 with the line preconditioner: 16 CTAs x (1024 - 128) rows = 14,336.  A set just below
    the capacity runs in the cluster, one just above in the grid solver; both match the oracle."""
    case = big
    rng = np.random.default_rng(3)
    base = case.always_active.astype(np.uint8)
    extra = np.flatnonzero(base == 0)
    cap = cluster_capacity(16, 1)
    for n_target, expect in ((cap, CLUSTER), (cap + 1, GRID)):
        va = base.copy()
        va[rng.choice(extra, n_target - int(base.sum()), replace=False)] = 1
        assert int(va.sum()) == n_target
        _check(case, va, 1, 16, expect=expect, seed=2)


def test_fp64_cluster_capacity(big):
    """FP64: 16 x (512 - 128) = 6,144 rows.  The first 6,144 always-active cells (whole fracture
    lines and a cut one) run in the cluster, one more cell goes to the grid solver."""
    case = big
    cells = np.flatnonzero(case.always_active)
    for n_target, expect in ((6144, CLUSTER), (6145, GRID)):
        va = np.zeros(case.n, np.uint8)
        va[cells[:n_target]] = 1
        _check(case, va, 0, 16, expect=expect, seed=4)


@pytest.mark.parametrize("fp32", [0, 1])
def test_whole_case_cluster_equals_oracle_small(fp32):
    """Whole timesteps at a tight tolerance on the 50x50 case: every solve in the cluster."""
    case = cg.config0()
    tight = dict(tol_dp=1.0, tol_cnv=1e-10)
    ref = O.Sim(case, O.Options(mode=1, **tight))
    g = lns.Model(case, lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-12,
                                    krylov_maxit=5000, krylov_cluster=16, **tight))
    g.lns_set_tuning(cluster_max_rows=-1)
    for dt in case.dt_schedule:
        a = g.lns_timestep(dt)
        b = ref.timestep(dt)
        assert a["status"] == 0 and b["status"] == 0
        if not fp32:
            assert abs(a["iterations"] - b["iterations"]) <= 1
    p, sw = g.lns_get_state()
    g.close()
    tol = 1e-6 if fp32 else 1e-7
    assert np.max(np.abs(p - ref.p) / ref.p) < tol
    assert np.max(np.abs(sw - ref.sw)) < tol * 0.25
