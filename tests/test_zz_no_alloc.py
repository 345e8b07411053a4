"""lns_active_set_noalloc: the active-set update for callers that cannot allocate device memory.

Such callers (memory owned by a host framework's pool or a fixed budget, or code where a device
allocation would stall other work) cannot create a model, so this entry point works on device
arrays they already hold and keeps its working storage in a fixed array inside the library.
It must reproduce lns_active_set exactly; this file is collected last.
"""
import numpy as np
import pytest

from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_noalloc_matches_lns_active_set_on_two_calls_in_a_row():
    import torch

    lns.load(build_if_missing=True)
    stream = torch.cuda.current_stream().cuda_stream
    for case, layers in ((cg.small_dfn(), 2), (cg.config0(), 3)):
        opts = lns.Options(mode=lns.LNS_MODE_LOCAL, eps_p=2.0, eps_sw=0.05, m_layers=layers)
        model = lns.Model(case, opts)
        n = case.n
        row_ptr = _dev(case.row_ptr, torch.int32)
        nbr = _dev(case.nbr, torch.int32)
        always = _dev(lns.mask_to_bits(case.always_active).view(np.int32), torch.int32)
        rng = np.random.default_rng(layers)
        for call in range(2):
            va0 = (rng.random(n) < 0.3).astype(np.uint8) | case.always_active
            dp = rng.uniform(-4, 4, n) * (rng.random(n) < 0.5)
            dsw = rng.uniform(-0.1, 0.1, n)
            converged = bool(call)
            ref_va, ref_vb, ref_ie = model.lns_active_set(va0, dp, dsw, converged)
            va = _dev(lns.mask_to_bits(va0).view(np.int32), torch.int32)
            vb = torch.zeros_like(va)
            dp_d = _dev(dp, torch.float64)
            dsw_d = _dev(dsw, torch.float64)
            ie = lns.lns_active_set_noalloc(n, row_ptr.data_ptr(), nbr.data_ptr(), always.data_ptr(), dp_d.data_ptr(),
                                            dsw_d.data_ptr(), opts.eps_p, opts.eps_sw, layers, converged,
                                            va.data_ptr(), vb.data_ptr(), stream)
            got_va = lns.bits_to_mask(va.cpu().numpy().view(np.uint32), n)
            got_vb = lns.bits_to_mask(vb.cpu().numpy().view(np.uint32), n)
            assert np.array_equal(got_va, ref_va), (case.name, call)
            assert np.array_equal(got_vb, ref_vb), (case.name, call)
            assert ie == ref_ie
        model.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lns.load(build_if_missing=True)
    with pytest.raises(lns.LnsError) as e:
        lns.lns_active_set_noalloc((1 << 20) + 1, 0, 0, 0, 0, 0, 1.0, 0.0, 2, False, 0, 0)
    assert e.value.status == lns.LNS_EINVAL and "n_cells" in str(e.value)
