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


@pytest.mark.parametrize("no_always,no_dsw,layers,zero_dp,converged", [
    (True, False, 2, False, False),   # no always-active cells (NULL bitset)
    (False, True, 2, False, True),    # no saturation update (NULL dsw)
    (False, False, 0, False, False),  # m = 0: no expansion beyond the moved boundary cells
    (False, False, 2, True, False),   # zero update, not converged: V_A kept
    (False, False, 2, True, True),    # zero update, converged: shrink to the always-active cells
])
def test_noalloc_edge_cases_match_lns_active_set(no_always, no_dsw, layers, zero_dp, converged):
    import dataclasses

    import torch

    lns.load(build_if_missing=True)
    stream = torch.cuda.current_stream().cuda_stream
    case = cg.small_dfn()
    if no_always:
        case = dataclasses.replace(case, always_active=np.zeros(case.n, np.uint8))
    n = case.n
    opts = lns.Options(mode=lns.LNS_MODE_LOCAL, eps_p=2.0, eps_sw=0.0 if no_dsw else 0.05, m_layers=layers)
    model = lns.Model(case, opts)
    rng = np.random.default_rng(7 + layers)
    va0 = (rng.random(n) < 0.3).astype(np.uint8) | case.always_active
    dp = np.zeros(n) if zero_dp else rng.uniform(-4, 4, n) * (rng.random(n) < 0.5)
    dsw = None if no_dsw else rng.uniform(-0.1, 0.1, n)
    ref_va, ref_vb, ref_ie = model.lns_active_set(va0, dp, dsw, converged)
    model.close()
    va = _dev(lns.mask_to_bits(va0).view(np.int32), torch.int32)
    vb = torch.zeros_like(va)
    dp_d = _dev(dp, torch.float64)
    dsw_d = None if no_dsw else _dev(dsw, torch.float64)
    always = None if no_always else _dev(lns.mask_to_bits(case.always_active).view(np.int32), torch.int32)
    row_ptr = _dev(case.row_ptr, torch.int32)  # kept alive across the call
    nbr = _dev(case.nbr, torch.int32)
    ie = lns.lns_active_set_noalloc(n, row_ptr.data_ptr(), nbr.data_ptr(), 0 if always is None else always.data_ptr(),
                                    dp_d.data_ptr(), 0 if dsw_d is None else dsw_d.data_ptr(), opts.eps_p, opts.eps_sw,
                                    layers, converged, va.data_ptr(), vb.data_ptr(), stream)
    assert np.array_equal(lns.bits_to_mask(va.cpu().numpy().view(np.uint32), n), ref_va)
    assert np.array_equal(lns.bits_to_mask(vb.cpu().numpy().view(np.uint32), n), ref_vb)
    assert ie == ref_ie


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lns.load(build_if_missing=True)
    with pytest.raises(lns.LnsError) as e:
        lns.lns_active_set_noalloc((1 << 20) + 1, 0, 0, 0, 0, 0, 1.0, 0.0, 2, False, 0, 0)
    assert e.value.status == lns.LNS_EINVAL and "n_cells" in str(e.value)
