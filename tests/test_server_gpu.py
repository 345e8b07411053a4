"""The serving loop (lns_server_*): requests for several resident models run concurrently on
worker streams, and every model ends exactly where it ends when run alone; eviction under an HBM
budget restores state and support exactly; a request whose step fails is cut and retried by the
time-step controller, and a request that fails down to the smallest step leaves its model unchanged."""
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


def _models():
    return [cg.config0(), cg.small_dfn(24, 20, 6, seed=7, n_steps=6), cg.small_dfn(40, 33, 14, seed=11, n_steps=6)]


def _schedule(k, n=5):
    rng = np.random.default_rng(100 + k)
    return np.exp(rng.uniform(np.log(0.05), np.log(5.0), n)) * cg.DAY


def _solo(case, opts, dts):
    m = lns.Model(case, opts)
    m.lns_set_tuning(cluster_max_rows=-1)  # as served models: every system that fits in the cluster
    for dt in dts:
        m.lns_timestep(float(dt))
    p, sw = m.lns_get_state()
    m.close()
    return p, sw


@pytest.mark.parametrize("fp32", [0, 1])
def test_mixed_requests_match_solo_runs(fp32):
    cases = _models()
    opts = lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-6)
    scheds = [_schedule(k) for k in range(len(cases))]
    srv = lns.Server(workers=3)
    ids = [srv.add_model(c, opts) for c in cases]
    rid = 0
    for j in range(5):  # interleaved: every model has a request in flight at once
        for k, mid in enumerate(ids):
            srv.submit(mid, scheds[k][j], rid)
            rid += 1
    srv.drain()
    done = []
    while True:
        got = srv.poll(64, 0.0)
        if not got:
            break
        done += got
    assert len(done) == rid and all(c["status"] == 0 for c in done)
    assert all(c["t_submit"] <= c["t_start"] <= c["t_done"] for c in done)
    for k, mid in enumerate(ids):  # per-model order is submission order
        mine = [c["request_id"] for c in sorted(done, key=lambda c: c["t_start"]) if c["model"] == mid]
        assert mine == sorted(mine)
    for k, (c, mid) in enumerate(zip(cases, ids)):
        p, sw = srv.get_state(mid)
        ps, sws = _solo(c, opts, scheds[k])
        assert np.array_equal(p, ps) and np.array_equal(sw, sws), k
    st = srv.stats()
    assert st["completed"] == rid and st["failed"] == 0 and st["resident_models"] == 3
    srv.close()


def test_eviction_under_budget_restores_exactly():
    cases = _models()[1:]
    opts = lns.Options(mode=1)
    scheds = [_schedule(k + 7, 4) for k in range(2)]
    sizes = []
    for k in range(2):  # device bytes of each model alone
        probe = lns.Server(workers=1)
        probe.add_model(cases[k], opts)
        probe.submit(0, scheds[k][0], 0)
        probe.drain()
        sizes.append(probe.stats()["resident_bytes"])
        probe.close()
    budget = int(max(sizes) * 1.05)
    assert sum(sizes) > budget  # one model fits at a time
    srv = lns.Server(workers=2, hbm_budget_bytes=budget)
    ids = [srv.add_model(c, opts) for c in cases]
    rid = 0
    for j in range(4):
        for k, mid in enumerate(ids):
            srv.submit(mid, scheds[k][j], rid)
            rid += 1
    srv.drain()
    st = srv.stats()
    assert st["failed"] == 0 and st["evictions"] >= 2
    for k, (c, mid) in enumerate(zip(cases, ids)):
        p, sw = srv.get_state(mid)
        ps, sws = _solo(c, opts, scheds[k])
        assert np.array_equal(p, ps) and np.array_equal(sw, sws), k
    srv.close()


def _max_krylov(case, opts, dts):
    """Largest BiCGStab iteration count of any solve over the steps dts, and the final fields."""
    m = lns.Model(case, opts)
    m.lns_set_tuning(cluster_max_rows=-1)
    kmax = 0
    for dt in dts:
        while True:
            st = m.lns_newton_iter(float(dt))
            kmax = max(kmax, st["krylov_iters"])
            if st["step_done"]:
                break
    p, sw = m.lns_get_state()
    m.close()
    return kmax, p, sw


def test_failed_step_is_retried_as_halves():
    case = cg.small_dfn(40, 33, 14, seed=11, n_steps=2)
    base = dict(mode=1, krylov_rtol=1e-8, krylov_fail_rtol=1e-14)
    # a step whose linear solves need more BiCGStab iterations than those of its halves
    for days in (30.0, 300.0, 3.0, 3000.0):
        dt = days * cg.DAY
        k_full, _, _ = _max_krylov(case, lns.Options(**base), [dt])
        k_half, p_ref, sw_ref = _max_krylov(case, lns.Options(**base), [dt / 2, dt / 2])
        if k_half < k_full:
            break
    else:
        pytest.fail("no timestep whose halves need fewer BiCGStab iterations")
    opts = lns.Options(**base, krylov_maxit=k_half)  # the whole step fails (LNS_EKRYLOV), the halves pass
    srv = lns.Server(workers=1)
    mid = srv.add_model(case, opts)
    srv.submit(mid, dt, 0)
    srv.drain()
    c = srv.poll(4, 1.0)[0]
    assert c["status"] == 0 and c["stats"]["dd_outer"] == 1, c
    p, sw = srv.get_state(mid)
    assert np.array_equal(p, p_ref) and np.array_equal(sw, sw_ref)  # restored exactly, then two halves
    srv.close()


def test_request_failing_at_every_level_leaves_the_model_unchanged():
    case = cg.config0()
    opts = lns.Options(mode=1, tol_dp=0.0, max_newton=1)  # no step can converge (max |dp| < 0), at any dt
    srv = lns.Server(workers=1)
    mid = srv.add_model(case, opts)
    srv.submit(mid, cg.DAY, 0)
    srv.drain()
    c = srv.poll(4, 1.0)[0]
    # cut down to dt * 2^-16 (17 attempts), then given up
    assert c["status"] == lns.LNS_ENOCONV and c["stats"]["dd_outer"] == 17
    p, sw = srv.get_state(mid)
    assert np.array_equal(p, case.p0) and np.array_equal(sw, case.sw0)
    srv.close()


def test_bad_requests_are_rejected():
    srv = lns.Server(workers=1)
    mid = srv.add_model(cg.config0())
    with pytest.raises(lns.LnsError):
        srv.submit(mid + 1, cg.DAY, 0)
    with pytest.raises(lns.LnsError):
        srv.submit(mid, -1.0, 0)
    srv.close()
