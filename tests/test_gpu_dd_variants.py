"""Algorithm 2 variants on the GPU against the oracle: subdomain visits solved to local convergence
(dd_local_newton) with and without localization inside the subdomain (dd_local_shrink), whole
timesteps at a tight tolerance: the same local-solve counts per step within one, the same outer
passes, fields within 1e-7."""
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


@pytest.mark.parametrize("which", ["config0", "small_dfn"])
@pytest.mark.parametrize("local_newton,shrink", [(4, 0), (4, 1)])
def test_dd_variants_match_oracle(which, local_newton, shrink):
    case = cg.config0() if which == "config0" else cg.small_dfn(n_steps=5)
    kw = dict(mode=2, dd_local_newton=local_newton, dd_local_shrink=shrink, **TIGHT)
    ref = O.Sim(case, O.Options(**kw))
    g = lns.Model(case, lns.Options(krylov_rtol=1e-12, krylov_maxit=5000, **kw))
    for dt in case.dt_schedule:
        a = g.lns_timestep(dt)
        b = ref.timestep(dt)
        assert a["status"] == 0 and b["status"] == 0
        assert abs(a["iterations"] - b["iterations"]) <= 1, (a, b)
        assert a["n_subdomains"] == b["n_subdomains"]
    p, sw = g.lns_get_state()
    g.close()
    assert np.max(np.abs(p - ref.p) / ref.p) < 1e-7
    assert np.max(np.abs(sw - ref.sw)) < 1e-7


def test_dd_variant_options_are_checked():
    case = cg.small_dfn()
    with pytest.raises(lns.LnsError):
        lns.Model(case, lns.Options(mode=2, dd_local_newton=0))
    with pytest.raises(lns.LnsError):
        lns.Model(case, lns.Options(mode=2, dd_local_shrink=2))
