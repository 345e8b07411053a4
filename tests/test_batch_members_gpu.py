"""Batched ensembles (lns_batch_advance): independent realizations advanced together, each with its
own active sets, convergence and time-step controller.

- Every member ends bit for bit as lns_advance leaves it alone with every system that fits in the
  cluster solver sent there (state and statistics: steps, cuts, Newton and Krylov iterations, cell
  updates), in both Krylov precisions, with members of uneven size whose solves go to both solvers
  and whose steps are cut independently.
- Small members at a tight tolerance match the oracle's own controller run per member (same
  accepted and cut steps, fields within 1e-7).
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu
DAY = cg.DAY


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)
    O.build()


def _batch(cases, opts, **adv):
    import torch

    streams = [torch.cuda.Stream() for _ in cases]
    models = [lns.Model(c, opts, stream=s) for c, s in zip(cases, streams)]
    for m in models:
        m.lns_set_tuning(cluster_max_rows=-1)
    outs, bst = lns.lns_batch_advance(models, allow_noconv=True, **adv)
    torch.cuda.synchronize()
    states = [m.lns_get_state() for m in models]
    for m in models:
        m.close()
    return outs, bst, states


@pytest.mark.parametrize("fp32", [0, 1])
def test_members_bit_identical_to_solo_advance(fp32):
    cases = [cg.realization(r) for r in (0, 5, 6, 7)] + [cg.small_dfn(24, 20, 6, seed=7), cg.small_dfn(40, 33, 14, seed=11)]
    opts = lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-6, max_newton=4)
    adv = dict(t_span=20 * DAY, dt_init=20 * DAY, dt_min=0.01 * DAY, dt_max=20 * DAY)
    outs, bst, states = _batch(cases, opts, **adv)
    assert bst["cluster_solves"] > 0 and bst["grid_solves"] > 0, bst
    assert sum(o["cuts"] for o in outs) > 0, outs
    keys = ("status", "steps", "cuts", "iterations", "krylov_iters", "cell_updates", "t_done", "dt_next")
    for c, o, (pb, swb) in zip(cases, outs, states):
        g = lns.Model(c, opts)
        g.lns_set_tuning(cluster_max_rows=-1)  # every system that fits goes to the cluster, as in the batch
        a = g.lns_advance(allow_noconv=True, **adv)
        ps, sws = g.lns_get_state()
        g.close()
        assert {k: o[k] for k in keys} == {k: a[k] for k in keys}, (c.name, o, a)
        assert np.array_equal(pb, ps) and np.array_equal(swb, sws), c.name


def test_small_members_match_oracle_controller():
    cases = [cg.small_dfn(24, 20, 6, seed=7), cg.small_dfn(31, 17, 9, seed=3), cg.config0()]
    tight = dict(tol_dp=1.0, tol_cnv=1e-10, max_newton=8)
    opts = lns.Options(mode=1, krylov_rtol=1e-12, krylov_maxit=5000, **tight)
    adv = dict(t_span=10 * DAY, dt_init=10 * DAY, dt_min=0.001 * DAY, dt_max=10 * DAY)
    outs, bst, states = _batch(cases, opts, **adv)
    for c, o, (pb, swb) in zip(cases, outs, states):
        sim = O.Sim(c, O.Options(mode=1, **tight))
        r = sim.advance(adv["t_span"], adv["dt_init"], adv["dt_min"], adv["dt_max"])
        assert (o["status"], o["steps"], o["cuts"]) == (r["status"], r["steps"], r["cuts"]), (c.name, o, r)
        assert np.max(np.abs(pb - sim.p) / sim.p) < 1e-7
        assert np.max(np.abs(swb - sim.sw)) < 1e-7


def test_batch_rejects_bad_members():
    case = cg.small_dfn()
    a = lns.Model(case, lns.Options(mode=2))
    with pytest.raises(lns.LnsError) as e:
        lns.lns_batch_advance([a], DAY)
    assert e.value.status == lns.LNS_EINVAL
    b = lns.Model(case, lns.Options(mode=1))
    with pytest.raises(lns.LnsError):
        lns.lns_batch_advance([b, b], DAY)
    outs, bst = lns.lns_batch_advance([], DAY)
    assert outs == [] and bst["rounds"] == 0
    a.close()
    b.close()
