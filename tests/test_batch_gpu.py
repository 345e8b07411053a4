"""Batched realizations: the disjoint union of several DFN models advanced by one solver (one
active set, one BiCGStab launch per Newton iteration for all members) against each member run
alone on the GPU and against the CPU oracle run per member."""
import numpy as np
import pytest

import oracle as O
from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu
TIGHT = dict(tol_dp=1.0, tol_cnv=1e-10)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)
    O.build()


def _members():
    return [cg.small_dfn(24, 20, 6, seed=7, n_steps=5), cg.small_dfn(31, 17, 9, seed=3, n_steps=5),
            cg.small_dfn(40, 33, 14, seed=11, n_steps=5)]


@pytest.mark.parametrize("fp32", [0, 1])
def test_batched_members_match_solo_and_oracle(fp32):
    members = _members()
    union = cg.batch(members)
    opts = dict(mode=1, krylov_fp32=fp32, krylov_rtol=1e-5 if fp32 else 1e-12, krylov_maxit=5000, **TIGHT)
    g = lns.Model(union, lns.Options(**opts))
    for dt in union.dt_schedule:
        assert g.lns_timestep(dt)["status"] == 0
    pb, swb = g.lns_get_state()
    g.close()
    tol = 1e-6 if fp32 else 1e-7
    offs = union.meta["offsets"]
    for k, c in enumerate(members):
        sl = slice(offs[k], offs[k + 1])
        solo = lns.Model(c, lns.Options(**opts))
        ref = O.Sim(c, O.Options(mode=1, **TIGHT))
        for dt in c.dt_schedule:
            assert solo.lns_timestep(dt)["status"] == 0
            ref.timestep(dt)
        ps, sws = solo.lns_get_state()
        solo.close()
        assert np.max(np.abs(pb[sl] - ps) / ps) < tol
        assert np.max(np.abs(swb[sl] - sws)) < tol * 0.25
        assert np.max(np.abs(pb[sl] - ref.p) / ref.p) < tol
        assert np.max(np.abs(swb[sl] - ref.sw)) < tol * 0.25
