"""The autotuner on the GPU: it measures on the model's data and returns a valid tuning; launch
shapes leave every result bit-identical; the choice is cached per device and size class."""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)
    O.build()
    lns.lns_tune_cache_clear()
    yield
    lns.lns_tune_cache_clear()


def _run(case, opts, tuning=None, steps=None):
    g = lns.Model(case, opts)
    if tuning is not None:
        g.lns_set_tuning(tuning)
    stats = [g.lns_timestep(dt) for dt in case.dt_schedule[:steps]]
    p, sw = g.lns_get_state()
    g.close()
    return stats, p, sw


@pytest.mark.parametrize("fp32", [0, 1])
def test_launch_shapes_leave_results_bit_identical(fp32):
    case = cg.small_dfn(40, 33, 14, seed=11, n_steps=5)
    opts = lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-8)
    base = dict(cluster_max_rows=-1, asm_block=64, asm_blocks_per_sm=4, set_blocks_per_sm=4, measured=0)
    ref = _run(case, opts, base)
    for asm_block, am, sm in ((128, 2, 8), (256, 8, 2), (64, 1, 16)):
        got = _run(case, opts, dict(base, asm_block=asm_block, asm_blocks_per_sm=am, set_blocks_per_sm=sm))
        keys = ("iterations", "krylov_iters", "cell_updates")
        assert [[s[k] for k in keys] for s in got[0]] == [[s[k] for k in keys] for s in ref[0]]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("fp32", [0, 1])
def test_autotune_measures_applies_and_caches(fp32):
    case = cg.config1()
    opts = lns.Options(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-6)
    g = lns.Model(case, opts)
    p0, sw0 = g.lns_get_state()
    t = g.lns_autotune()
    assert t["measured"] == 1
    assert t["asm_block"] in (64, 128, 256) and t["asm_blocks_per_sm"] in (2, 4, 8)
    assert t["set_blocks_per_sm"] in (2, 4, 8)
    cap = 16 * ((1024 if fp32 else 512) - 128)
    assert 0 <= t["cluster_max_rows"] <= cap
    assert g.lns_get_tuning() == t
    p1, sw1 = g.lns_get_state()
    assert np.array_equal(p0, p1) and np.array_equal(sw0, sw1)  # the state is untouched
    # a new model of the same size class takes the cached choice
    h = lns.Model(case, opts)
    assert h.lns_get_tuning() == t
    h.lns_set_tuning(cluster_max_rows=0)
    assert h.lns_get_tuning()["cluster_max_rows"] == 0 and h.lns_get_tuning()["measured"] == t["measured"]
    h.lns_set_tuning(None)
    assert h.lns_get_tuning() == t
    # the tuned model runs the first timesteps of the case like the oracle
    ref = O.Sim(case, O.Options(mode=1))
    for dt in case.dt_schedule[:3]:
        a = g.lns_timestep(dt)
        b = ref.timestep(dt)
        assert a["status"] == 0 and b["status"] == 0
    p, sw = g.lns_get_state()
    assert np.max(np.abs(p - ref.p)) < 2 * 0.3 * cg.PSI
    g.close()
    h.close()
