"""Failure paths on the GPU, none of which faults or hangs the device: a bounded device-side wait
that runs out (LNS_ETIMEOUT, context still usable), a forced BiCGStab breakdown, non-finite inputs,
checkpoint and resume (bit-identical), and a cancelled serving request."""
import numpy as np
import pytest

from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)


def _run(case, opts, dts, model=None):
    m = model or lns.Model(case, opts)
    for dt in dts:
        m.lns_timestep(float(dt))
    return m


def test_barrier_wait_runs_out_with_etimeout_and_the_context_survives():
    case = cg.config0()
    m = lns.Model(case, lns.Options(mode=1))
    m.lns_debug_fault(1)  # one block never arrives at the solver's first grid barrier
    with pytest.raises(lns.LnsError) as e:
        m.lns_timestep(case.dt_schedule[0])
    assert e.value.status == lns.LNS_ETIMEOUT
    m.lns_debug_fault(0)
    m.lns_reset()
    _run(case, None, case.dt_schedule[:3], m)
    ref = _run(case, lns.Options(mode=1), case.dt_schedule[:3])
    assert np.array_equal(m.lns_get_state()[0], ref.lns_get_state()[0])
    m.close()
    ref.close()


def test_forced_breakdown_is_reported():
    case = cg.config0()
    m = lns.Model(case, lns.Options(mode=1))
    m.lns_debug_fault(2)
    with pytest.raises(lns.LnsError) as e:
        m.lns_timestep(case.dt_schedule[0])
    assert e.value.status == lns.LNS_EKRYLOV
    m.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_failed_fp32_solve_is_redone_in_fp64(mode):
    """Every FP32 solve breaks down (injected); with fp64_fallback each iteration's solve is redone
    in FP64 from the unchanged state and set, so the run equals an FP64 run bit for bit (both
    models on the same solver choice: the tuning cache of each precision class may pick another)."""
    case = cg.config0()
    base = dict(mode=mode, krylov_rtol=1e-6)
    m = lns.Model(case, lns.Options(**base, krylov_fp32=1))
    m.lns_set_tuning(cluster_max_rows=-1)
    m.lns_debug_fault(3)
    ref = lns.Model(case, lns.Options(**base))
    ref.lns_set_tuning(cluster_max_rows=-1)
    ref.lns_debug_fault(3)  # affects FP32 solves only: the FP64 run is the plain one
    for dt in case.dt_schedule[:3]:
        st = m.lns_timestep(float(dt))
        sr = ref.lns_timestep(float(dt))
        assert st["fp64_retries"] == st["iterations"] == sr["iterations"] > 0
        assert sr["fp64_retries"] == 0
    for a, b in zip(m.lns_get_state(), ref.lns_get_state()):
        assert np.array_equal(a, b)
    m.close()
    ref.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("cluster", [0, -1])
def test_stalled_fp32_solve_is_redone_in_fp64_from_its_iterate(cluster, mode):
    """FP32 solves stop after their first iteration as if stalled (injected), above
    krylov_fail_rtol; each is solved again in FP32 from its iterate (stalling again) and then
    redone in FP64 from the latest iterate (grid and cluster solvers, Algorithm 1 and 2), and the
    steps end at the FP64 run's solution to the Krylov tolerance."""
    case = cg.config0()
    base = dict(mode=mode, krylov_rtol=1e-12, krylov_maxit=5000, tol_dp=1.0, tol_cnv=1e-10)
    m = lns.Model(case, lns.Options(**base, krylov_fp32=1, krylov_fail_rtol=1e-11))
    m.lns_set_tuning(cluster_max_rows=cluster)
    m.lns_debug_fault(4)
    ref = lns.Model(case, lns.Options(**base))
    ref.lns_set_tuning(cluster_max_rows=cluster)
    retries = iters = 0
    for dt in case.dt_schedule[:4]:
        st = m.lns_timestep(float(dt))
        retries += st["fp64_retries"]
        iters += st["iterations"]
        ref.lns_timestep(float(dt))
    assert 0 < retries <= iters  # (a system the first iteration solves is not redone)
    (p, sw), (pr, swr) = m.lns_get_state(), ref.lns_get_state()
    assert np.max(np.abs(p - pr) / pr) < 1e-9
    assert np.max(np.abs(sw - swr)) < 1e-9
    m.close()
    ref.close()


def test_failed_fp32_solve_without_fallback_is_reported():
    case = cg.config0()
    m = lns.Model(case, lns.Options(mode=1, krylov_fp32=1, fp64_fallback=0))
    p0 = m.lns_get_state()[0].copy()
    m.lns_debug_fault(3)
    with pytest.raises(lns.LnsError) as e:
        m.lns_newton_iter(case.dt_schedule[0])
    assert e.value.status == lns.LNS_EKRYLOV
    assert np.array_equal(m.lns_get_state()[0], p0)  # a failed solve scatters nothing
    m.close()


def test_non_finite_inputs_are_rejected():
    case = cg.config0()
    m = lns.Model(case)
    p = case.p0.copy()
    p[7] = np.nan
    with pytest.raises(lns.LnsError) as e:
        m.lns_set_state(p, case.sw0)
    assert e.value.status == lns.LNS_EINVAL
    m.close()
    bad = cg.config0()
    bad.sw0 = bad.sw0.copy()
    bad.sw0[3] = np.inf
    with pytest.raises(lns.LnsError):
        lns.Model(bad)


@pytest.mark.parametrize("fp32", [0, 1])
def test_checkpoint_and_resume_is_bit_identical(fp32):
    case = cg.small_dfn(40, 33, 14, seed=11, n_steps=6)
    opts = lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-6)
    whole = _run(case, opts, case.dt_schedule)
    first = _run(case, opts, case.dt_schedule[:3])
    p, sw = first.lns_get_state()
    supp = lns.mask_to_bits(first.lns_get_support())
    first.close()
    resumed = lns.Model(case, opts)
    resumed.lns_set_state(p, sw)
    resumed.lns_set_support(supp)
    _run(case, opts, case.dt_schedule[3:], resumed)
    pw, sww = whole.lns_get_state()
    pr, swr = resumed.lns_get_state()
    assert np.array_equal(pw, pr) and np.array_equal(sww, swr)
    whole.close()
    resumed.close()


def test_cancelled_request_leaves_its_model_unchanged():
    cases = [cg.config0(), cg.small_dfn(24, 20, 6, seed=7, n_steps=4)]
    opts = lns.Options(mode=1)
    srv = lns.Server(workers=1)
    ids = [srv.add_model(c, opts) for c in cases]
    # one worker: the first request runs while the others wait in the queue
    srv.submit(ids[0], 5.0 * cg.DAY, 0)
    srv.submit(ids[1], 1.0 * cg.DAY, 1)
    srv.submit(ids[1], 2.0 * cg.DAY, 2)
    cancelled = srv.cancel(1)
    srv.drain()
    done = {c["request_id"]: c for c in srv.poll(16, 1.0)}
    assert set(done) == {0, 1, 2}
    ref = lns.Model(cases[1], opts)
    ref.lns_set_tuning(cluster_max_rows=-1)  # as served models: every system that fits in the cluster
    if cancelled:
        assert done[1]["status"] == lns.LNS_ESTATE
        _run(cases[1], opts, [2.0 * cg.DAY], ref)
    else:  # the worker had already taken it
        assert done[1]["status"] == 0
        _run(cases[1], opts, [1.0 * cg.DAY, 2.0 * cg.DAY], ref)
    assert np.array_equal(srv.get_state(ids[1])[0], ref.lns_get_state()[0])
    assert not srv.cancel(0)  # finished requests cannot be cancelled
    srv.close()
    ref.close()
